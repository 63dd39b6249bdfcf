// k_batched.cu -- one Lloyd pass of every problem of lbg_train_batched in a
// single persistent launch.
//
// Paper: the LBG iteration of Sec. 2.2 (and Algorithm 1's Cell Allocation,
// IntegrateDistortions, stop test, Updation and Codebook Splitting), run for
// S independent training sets at once; each set computes exactly what
// lbg_train computes for it alone.
//
// GB300 design.  The phases of a pass depend on one another across the whole
// grid (the cell table needs every row's cell, the offsets every cell's
// count, ...), so they are separated by grid-wide barriers inside one
// cooperative launch (all CTAs resident), instead of one launch per phase:
//   1  codebook preparation (per problem, 32-codevector blocks)
//   2  nearest codevector: each half of a CTA (128 threads, its own named
//      barrier and shared buffers) takes (problem, 64-row tile) items from a
//      counter
//   3  exact re-scoring of the uncertified rows (groups of 8 rows, all problems)
//   4  per-chunk cell counts and distortion partials
//   5  each problem's stop test (sum in chunk order, (D_prev - D)/D <= theta;
//      problem s in CTA s mod grid) and the per-cell prefixes over chunks
//   5b each problem's cell offsets
//   6  stable placement of the rows by cell
//   7  per-warp piece sums of the cells
//   8  centroids, one thread per value (in place), and the split of a
//      finished stage into the spare codebook
//   9  copy back, each problem's stage advance, and the next pass's resets
// A phase's blocks are virtual: CTA b takes blocks b, b + grid, ... of the
// launch-per-phase form and runs the same device body on each, so the bits
// are those of lbg_train.  The per-problem steps (5's stop test, 5b, 9's advance) run in
// one CTA each, after a grid barrier, instead of in whichever block of the
// problem finishes last (a fence and an atomic per block).
//
// Every barrier wait is bounded (%globaltimer, 2 s): a CTA that gives up sets
// the shared abort word and reports LBG_ERR_TIMEOUT in every problem's state;
// every other CTA sees the abort word at its next barrier and returns.  The
// abort word stays set for the rest of the call, so later passes return at
// once and the host stops at its next check.
#include "bodies_assign.cuh"
#include "bodies_update.cuh"
#include "lbg_internal.cuh"

namespace lbg {
namespace {

constexpr int BP_THREADS = 256;
constexpr int BP_TILE = 64;         // rows per assignment tile: two tiles of 128 threads per CTA

// Floats of one assignment tile's dynamic shared memory: the x tile, two codebook chunks.
__host__ __device__ constexpr size_t assign_floats(int Lp, int tbm)
{
    return (size_t)Lp * tbm + 2 * (size_t)(Lp + 1) * BN;
}
constexpr int BP_MAX_SETS = 1024;   // problems the per-CTA state tables hold (more: per-phase launches)

// Per-problem state as of a phase's start, read once per CTA after the barrier
// into shared memory (a virtual block then reads no device state to decide
// whether to run): bit 0 = not finished, bit 1 = the pass updates (stop test
// said UPDATE); the stage size; the exact phase's group prefix.
struct PassTables {
    int *run, *ncur, *gpre;
};

__device__ __forceinline__ void load_states(const BatchSet *__restrict__ sets, int S, const PassTables &t)
{
    for (int s = threadIdx.x; s < S; s += BP_THREADS) {
        const DevState *st = sets[s].st;
        const int fin = st->finished;
        t.run[s] = fin ? 0 : (1 | (st->action == ACT_UPDATE ? 2 : 0));
        t.ncur[s] = st->n_cur;
    }
    __syncthreads();
}

// gpre[s] = flagged groups of problems before s (gpre[S] = all): a thread per
// contiguous range of problems, then the ranges' sums in order.
__device__ __forceinline__ void exact_prefix(const BatchSet *__restrict__ sets, int S, const PassTables &t)
{
    __shared__ int part[BP_THREADS];
    const int per = (S + BP_THREADS - 1) / BP_THREADS;
    const int a = threadIdx.x * per, b = a + per < S ? a + per : S;
    int loc = 0;
    for (int s = a; s < b; ++s) {
        const int g = (t.run[s] & 1) ? (sets[s].st->nflag + EX_R - 1) / EX_R : 0;
        t.gpre[s] = g;
        loc += g;
    }
    part[threadIdx.x] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < BP_THREADS; ++i) {
            const int v = part[i];
            part[i] = run;
            run += v;
        }
        t.gpre[S] = run;
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int s = a; s < b; ++s) {
        const int g = t.gpre[s];
        t.gpre[s] = run;
        run += g;
    }
    __syncthreads();
}

// Rows [r0, r0 + 64) of problem q at a small stage (N codevectors) in the FP32
// direct form, sum over l in index order of fl(x_l - c_l)^2, lowest index on
// ties: the values and the choice the tiled search and its exact re-scoring
// give (as k_assign_direct in the per-step path), without a certificate or
// flagged rows.  The half's 128 threads: two per row, each over one contiguous
// half of the codevectors; the lower half wins a tie.  L <= 64, L % 4 == 0,
// rows 16-byte aligned.
__device__ __forceinline__ void direct_tile(const BatchSet &q, int L, int N, int64_t r0, float *hsm, int t,
                                            int bar_id)
{
    const int r = t & 63, part = t >> 6;
    const int64_t m = r0 + r;
    const int h = (N + 1) >> 1;
    const int n_lo = part ? h : 0, n_hi = part ? N : h;
    const int L4 = L >> 2;
    float best = INFINITY;
    int bi = n_lo;
    bool bad = false;
    if (m < q.M) {
        float x[64];
        const float4 *xr = reinterpret_cast<const float4 *>(q.X + m * L);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float4 v = k < L4 ? __ldg(xr + k) : make_float4(0.f, 0.f, 0.f, 0.f);
            x[4 * k] = v.x;
            x[4 * k + 1] = v.y;
            x[4 * k + 2] = v.z;
            x[4 * k + 3] = v.w;
            bad = bad || !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
        }
        const float4 *C4 = reinterpret_cast<const float4 *>(q.C);
        for (int n = n_lo; n < n_hi; n += 4) {   // four sums at a time (the last ones repeated)
            const float4 *cr[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) cr[j] = C4 + (size_t)(n + j < n_hi ? n + j : n) * L4;
            float d2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if (k < L4) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float4 c = __ldg(cr[j] + k);
                        float d = __fsub_rn(x[4 * k], c.x);
                        d2[j] = fmaf(d, d, d2[j]);
                        d = __fsub_rn(x[4 * k + 1], c.y);
                        d2[j] = fmaf(d, d, d2[j]);
                        d = __fsub_rn(x[4 * k + 2], c.z);
                        d2[j] = fmaf(d, d, d2[j]);
                        d = __fsub_rn(x[4 * k + 3], c.w);
                        d2[j] = fmaf(d, d, d2[j]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)   // in index order: the lowest index wins a tie
                if (n + j < n_hi && d2[j] < best) {
                    best = d2[j];
                    bi = n + j;
                }
        }
    }
    float *sd = hsm;
    int *si = reinterpret_cast<int *>(hsm + 64);
    if (part == 1) {
        sd[r] = best;
        si[r] = bi;
    }
    tile_sync(bar_id, 2 * BP_TILE);
    if (part == 0 && m < q.M) {
        if (bad) flag_error(q.st, ERR_NONFINITE);
        if (sd[r] < best) {
            best = sd[r];
            bi = si[r];
        }
        q.assign[m] = bi;
        q.e[m] = best;
    }
}

// Grid-wide barrier: arrivals counted in bar[0]; the last arrival resets the
// count and bumps the generation bar[1], for which the others wait (bounded).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, const BatchSet *sets, int S)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *gen = bar + 1;
        volatile unsigned *abort_word = bar + 2;
        if (*abort_word) {
            ok = 0;
        } else {
            const unsigned g = *gen;
            __threadfence();
            if (atomicAdd(bar, 1u) == gridDim.x - 1) {
                atomicExch(bar, 0u);
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                const uint64_t t0 = global_ns();
                while (*gen == g) {
                    if (*abort_word) {
                        ok = 0;
                        break;
                    }
                    if (global_ns() - t0 > 2000000000ull) {
                        atomicExch(bar + 2, 1u);
                        for (int s = 0; s < S; ++s) flag_error(sets[s].st, ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(100);
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void abort_all(unsigned *bar) { atomicExch(bar + 2, 1u); }

__global__ void __launch_bounds__(BP_THREADS, 2) kb_pass(const BatchPass a)
{
    extern __shared__ __align__(128) float dsm[];   // each phase's dynamic shared memory, then the tables
    __shared__ AssignSmemT<BP_TILE> ash[2];
    __shared__ __align__(16) ExactSmem esh;
    __shared__ int64_t s_item[2];
    const BatchSet *sets = a.sets;
    const int S = a.S, tid = threadIdx.x;
    const int grid = (int)gridDim.x;
    int *tab = reinterpret_cast<int *>(reinterpret_cast<char *>(dsm) + a.phase_smem);
    const PassTables T{tab, tab + S, tab + 2 * S};

    // 0: the shared-memory barriers of the assignment and exact phases (the work counter
    // and the problems' max ||c~|| were zeroed at the end of the previous pass, or by the
    // host before the first)
    if (tid == 0) {
        for (int h = 0; h < 2; ++h) {
            mbar_init(&ash[h].bar[0], 1);
            mbar_init(&ash[h].bar[1], 1);
            ash[h].abort = 0;
        }
        fence_mbar_init();
    }
    __syncthreads();
    exact_init(esh);

    // 1: codebook preparation
    load_states(sets, S, T);
    for (int vb = blockIdx.x; vb < a.tot_prep; vb += grid) {
        const int s = find_set(a.pre_prep, S, vb);
        const BatchSet &q = sets[s];
        if ((T.run[s] & 1) && T.ncur[s] > a.direct_max)   // the direct tiles read C as it is
            body_prep(q.C, T.ncur[s], a.L, a.Lp, q.mu, q.Cp, q.kn, q.CT, q.st, vb - a.pre_prep[s],
                      *reinterpret_cast<PrepSmem *>(dsm));
        __syncthreads();
    }
    if (!grid_barrier(a.bar, sets, S)) return;

    // 2: nearest codevector.  The two halves of the CTA work independently (named
    // barriers 1 and 2), each taking (problem, 64-row tile) items from the counter
    // into its own shared buffers; a half whose copy timed out stops, and the CTA
    // leaves once both halves are done.
    {
        const int half = tid >> 7;
        uint32_t u0 = 0, u1 = 0;
        float *hsm = dsm + half * assign_floats(a.Lp, BP_TILE);
        bool failed = false;
        for (;;) {
            if ((tid & 127) == 0) s_item[half] = (int64_t)atomicAdd(a.counter, 1);
            tile_sync(1 + half, 2 * BP_TILE);
            const int64_t item = s_item[half];
            if (item >= a.ntiles) break;
            const int s = find_set64(a.pre_tiles, S, item);
            const BatchSet &q = sets[s];
            if ((T.run[s] & 1) && T.ncur[s] <= a.direct_max) {
                direct_tile(q, a.L, T.ncur[s], (item - a.pre_tiles[s]) * BP_TILE, hsm, tid & 127, 1 + half);
            } else if (T.run[s] & 1) {
                const int64_t tile = item - a.pre_tiles[s];
                if (!assign_f32_tile_t<BP_TILE>(q.X, q.M, a.L, a.Lp, q.Cp, q.kn, T.ncur[s], q.mu, q.C, q.st,
                                               q.assign, q.e, q.flags, tile * BP_TILE, hsm, ash[half], u0, u1,
                                               0, half * 2 * BP_TILE, 1 + half)) {
                    failed = true;   // reported by the tile; its copies have been waited for
                    break;
                }
            }
            tile_sync(1 + half, 2 * BP_TILE);   // this item's shared data read before the next
        }
        if (__syncthreads_or(failed)) {
            if (tid == 0) abort_all(a.bar);
            return;
        }
    }
    if (!grid_barrier(a.bar, sets, S)) return;

    // 3: exact re-scoring; the flagged groups of all problems in problem order
    exact_prefix(sets, S, T);
    {
        uint32_t uses[2] = {0u, 0u};
        const int total = T.gpre[S];
        for (int item = blockIdx.x; item < total; item += grid) {
            int lo = 0, hi = S - 1;   // the problem s with gpre[s] <= item < gpre[s + 1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (T.gpre[mid] <= item)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const int s = lo, g = item - T.gpre[s];
            const BatchSet &q = sets[s];
            if (!exact_group(q.X, a.L, a.Lp, q.CT, T.ncur[s], q.st, q.flags, q.st->nflag, q.assign, q.e, g,
                             dsm, esh, uses)) {
                abort_all(a.bar);
                return;
            }
        }
    }
    if (!grid_barrier(a.bar, sets, S)) return;

    // 4: cell counts and distortion partials per chunk
    for (int vb = blockIdx.x; vb < a.tot_hist; vb += grid) {
        const int s = find_set(a.pre_hist, S, vb);
        const BatchSet &q = sets[s];
        if (T.run[s] & 1)
            body_hist(q.assign, q.e, q.M, q.R, T.ncur[s], 1, q.table, q.dpart, q.st, vb - a.pre_hist[s]);
        __syncthreads();
    }
    if (!grid_barrier(a.bar, sets, S)) return;

    // 4b + 5: each problem's stop test (one warp; problem s in CTA s mod grid) and the
    // per-cell prefixes over chunks of every running problem; the two do not depend on each
    // other (the prefixes are used only by an update, which the next phases gate)
    for (int s = blockIdx.x; s < S; s += grid) {
        const BatchSet &q = sets[s];
        if (T.run[s] & 1) body_ctl(q.dpart, q.CH, q.st, MODE_TRAIN, a.theta, a.max_passes, q.N, nullptr, 0);
    }
    for (int vb = blockIdx.x; vb < a.tot_scan; vb += grid) {
        const int s = find_set(a.pre_scan, S, vb);
        const BatchSet &q = sets[s];
        if (T.run[s] & 1) body_scan<BP_THREADS / 32>(q.table, q.CH, T.ncur[s], q.counts, vb - a.pre_scan[s]);
        __syncthreads();
    }
    if (!grid_barrier(a.bar, sets, S)) return;

    // 5b: each problem's cell offsets (problem s in CTA s mod grid)
    load_states(sets, S, T);   // the stop tests of phase 4b
    for (int s = blockIdx.x; s < S; s += grid) {
        const BatchSet &q = sets[s];
        if (T.run[s] & 1) {
            body_offsets<BP_THREADS>(q.counts, T.ncur[s], q.off);
        }
        __syncthreads();
    }
    if (!grid_barrier(a.bar, sets, S)) return;

    // 6: stable placement by cell
    for (int vb = blockIdx.x; vb < a.tot_hist; vb += grid) {
        const int s = find_set(a.pre_hist, S, vb);
        const BatchSet &q = sets[s];
        if (T.run[s] & 2)
            body_scatter(q.assign, q.M, q.R, q.table, q.off, T.ncur[s], q.perm, vb - a.pre_hist[s]);
        __syncthreads();
    }
    if (!grid_barrier(a.bar, sets, S)) return;

    // 7: per-warp piece sums of the cells (the bodies are per warp and use no shared
    // memory: warps take the pieces one by one, piece w of the launch-per-phase form's
    // block w / 8, with no block-wide step)
    {
        constexpr int WPB = BP_THREADS / 32;
        const int64_t nw = (int64_t)grid * WPB, tot = (int64_t)a.tot_cellsum * WPB;
        for (int64_t w = (int64_t)blockIdx.x * WPB + (tid >> 5); w < tot; w += nw) {
            const int vb = (int)(w / WPB);
            const int s = find_set(a.pre_cellsum, S, vb);
            const BatchSet &q = sets[s];
            const int64_t qq = (int64_t)(vb - a.pre_cellsum[s]) * WPB + (w % WPB);
            if (T.run[s] & 2) {
                const int N = T.ncur[s];
                switch (a.vec ? a.L : 0) {
                case 4: body_cellsum_v4<1>(q.X, q.M, q.perm, q.off, N, q.S, q.pieces, 0, qq); break;
                case 8: body_cellsum_v4<2>(q.X, q.M, q.perm, q.off, N, q.S, q.pieces, 0, qq); break;
                case 16: body_cellsum_v4<4>(q.X, q.M, q.perm, q.off, N, q.S, q.pieces, 0, qq); break;
                case 32: body_cellsum_v4<8>(q.X, q.M, q.perm, q.off, N, q.S, q.pieces, 0, qq); break;
                case 64: body_cellsum_v4<16>(q.X, q.M, q.perm, q.off, N, q.S, q.pieces, 0, qq); break;
                case 128: body_cellsum_v4<32>(q.X, q.M, q.perm, q.off, N, q.S, q.pieces, 0, qq); break;
                default: body_cellsum_any(q.X, q.M, a.L, q.perm, q.off, N, q.S, q.pieces, 0, qq);
                }
            }
        }
    }
    if (!grid_barrier(a.bar, sets, S)) return;

    // 7b + 8: centroids of the updating problems, one thread per value (the FP64 sums of
    // the pieces in the order and levels of the fused form, divided by the counts; in
    // place, empty cells keep theirs), and the split of the problems whose stage ended
    // (disjoint problems: an update and a split never meet in one pass)
    for (int vb = blockIdx.x; vb < a.tot_combine; vb += grid) {
        const int s = find_set(a.pre_combine, S, vb);
        const BatchSet &q = sets[s];
        const int b = vb - a.pre_combine[s];
        if ((T.run[s] & 2) && (int64_t)b * BP_THREADS < (int64_t)T.ncur[s] * a.L)
            body_combine(q.pieces, q.off, T.ncur[s], a.L, q.S, q.C, q.C, b);
    }
    for (int vb = blockIdx.x; vb < a.tot_split; vb += grid) {
        const int s = find_set(a.pre_split, S, vb);
        const BatchSet &q = sets[s];
        body_split(q.C, q.Calt, a.L, a.delta, a.mult, q.st, vb - a.pre_split[s]);
    }
    if (!grid_barrier(a.bar, sets, S)) return;

    // 9: copy back (sized by the stage size read at phase 5) and each problem's stage
    // advance (problem s in CTA s mod grid): the copy does not read what the advance writes
    for (int vb = blockIdx.x; vb < a.tot_copy; vb += grid) {
        const int s = find_set(a.pre_copy, S, vb);
        const BatchSet &q = sets[s];
        body_copy_split(q.Calt, q.C, a.L, q.st, vb - a.pre_copy[s], T.ncur[s]);
    }
    for (int s = blockIdx.x; s < S; s += grid) body_stage(sets[s].st);
    // for the next pass: the work counter and the problems' max ||c~|| (phase 1)
    if (blockIdx.x == 0) {
        if (tid == 0) *a.counter = 0;
        for (int s = tid; s < S; s += BP_THREADS) sets[s].st->cmax_bits = 0u;
    }
}

size_t pass_phase_smem(int L, int NMAXB)
{
    const int Lp = round_up(L, 4);
    const size_t assign = 2 * assign_floats(Lp, BP_TILE) * sizeof(float);
    const size_t exact = (size_t)2 * Lp * EX_SW * sizeof(float);
    const size_t hist = (size_t)NMAXB * sizeof(int);
    const size_t scatter = (size_t)NMAXB * (sizeof(int) + 8);
    size_t m = assign;
    if (sizeof(PrepSmem) > m) m = sizeof(PrepSmem);
    if (exact > m) m = exact;
    if (hist > m) m = hist;
    if (scatter > m) m = scatter;
    return (m + 15) / 16 * 16;
}

}  // namespace

int batch_pass_fit(int S, int L, int NMAXB, size_t *phase_smem, size_t *smem)
{
    if (S > BP_MAX_SETS) return 0;
    *phase_smem = pass_phase_smem(L, NMAXB);
    const size_t m = *phase_smem + sizeof(int) * (size_t)(3 * S + 1);
    *smem = m;
    if (cudaFuncSetAttribute(kb_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kb_pass, BP_THREADS, m) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return per;
}

bool launch_b_pass(const BatchPass &a, int ctas_per_sm, size_t smem, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(num_sms() * ctas_per_sm));
    cfg.blockDim = dim3(BP_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kb_pass, a) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    note_launch();
    return true;
}

}  // namespace lbg
