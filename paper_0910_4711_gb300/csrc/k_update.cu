// k_update.cu -- initial centroid, distortion integration, stop test, cell
// table and centroid update, codebook splitting.
//
// Paper: Algorithm 1 -- "compute centroid(input)" (Table 1),
// "IntegratePartialCellTables" / "IntegrateDistortions" (the cell table and
// TD = sum of the per-processor distortions), the stop test
// (D_prev - D)/D <= eps (Sec. 2.2 step 2), "Updation" (ExtractVectors of a
// cell + its centroid), and "Codebook Splitting" ([c + delta], [c - delta]).
//
// GB300 design: the paper's per-processor partial cell tables and round-robin
// centroid updates become a deterministic counting sort of the rows by cell
// followed by a segmented reduction; no floating-point atomics anywhere, and
// every floating-point sum has a fixed order, so two runs give identical bits.
//   k_hist     per-chunk cell counts (integer shared-memory atomics) and
//              per-chunk distortion partials (fixed-order tree, FP64 out);
//   k_ctl      D = fixed-order FP64 sum of the chunk partials, stop test
//              (k_hist_ctl: both in one launch, its last CTA doing k_ctl);
//   k_scan_offsets_q  per cell, exclusive prefix of its chunk counts + cell
//              size; its last CTA: exclusive prefix of the cell sizes (cell
//              start offsets), the cell of each warp piece's first row, empty
//              cells' codevectors copied;
//   k_scatter  stable placement of every row into perm[] (rows grouped by
//              cell, original order inside a cell);
//   k_cellsum_c  one warp per S consecutive perm entries: FP32 sums of the
//              gathered rows per cell piece (coalesced 16-byte row reads); a
//              cell held by one piece is divided by its count at once, the
//              last piece of a longer cell (per-cell counter) sums the cell's
//              pieces in order in FP64 and divides.
// The distortion backward keeps separate cell sums (k_cellsum_v4) and their
// gradient combine (k_combine_grad).
#include "bodies_update.cuh"
#include "lbg_internal.cuh"

#include <math.h>

namespace lbg {
namespace {

__global__ void __launch_bounds__(256) k_mean_part(const float *__restrict__ X, int64_t M, int L,
                                                   double *__restrict__ part, DevState *st)
{
    body_mean_part(X, M, L, part, st, blockIdx.x, gridDim.x);
}

// mu = C0 = fl32(sum of the partials in block order / M).
__global__ void k_mean_final(const double *__restrict__ part, int G, int64_t M, int L,
                             float *__restrict__ mu, float *__restrict__ C0)
{
    const int l = threadIdx.x;
    if (l >= L) return;
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += part[(size_t)b * L + l];
    const float c = (float)(s / (double)M);
    mu[l] = c;
    if (C0) C0[l] = c;
}

__global__ void __launch_bounds__(HIST_THREADS)
    k_hist(const int32_t *__restrict__ assign, const float *__restrict__ e, int64_t M, int64_t R,
           const int32_t *n_dev, int n_host, int do_hist, int32_t *__restrict__ table,
           double *__restrict__ dpart, DevState *st, int train)
{
    if (train && st->finished) return;
    body_hist(assign, e, M, R, cur_n(n_dev, n_host), do_hist, table, dpart, st, blockIdx.x);
}

__global__ void k_ctl(const double *__restrict__ dpart, int CH, DevState *st, int mode, double theta,
                      int max_passes, int N_target, PassRecord *rec, int max_rec)
{
    if (blockIdx.x != 0) return;
    body_ctl(dpart, CH, st, mode, theta, max_passes, N_target, rec, max_rec);
}

__global__ void __launch_bounds__(HIST_THREADS)
    k_hist_ctl(const int32_t *__restrict__ assign, const float *__restrict__ e, int64_t M, int64_t R,
               int N, int do_hist, int32_t *__restrict__ table, double *__restrict__ dpart, DevState *st)
{
    body_hist(assign, e, M, R, N, do_hist, table, dpart, st, blockIdx.x);
    if (!last_cta(st)) return;
    if (threadIdx.x == 0) st->done_ctr = 0u;
    body_ctl(dpart, gridDim.x, st, MODE_STEP, 0.0, 1, N, nullptr, 0);
}

__global__ void __launch_bounds__(1024)
    k_scan_offsets(int32_t *__restrict__ table, int CH, int N, int32_t *__restrict__ counts,
                   int32_t *__restrict__ off, DevState *st)
{
    if ((int)blockIdx.x * 32 < N) body_scan(table, CH, N, counts, blockIdx.x);
    if (!last_cta(st)) return;
    if (threadIdx.x == 0) st->done_ctr = 0u;
    body_offsets(counts, N, off);
}

__global__ void __launch_bounds__(256) k_scatter(const int32_t *__restrict__ assign, int64_t M,
                                                 int64_t R, const int32_t *__restrict__ table,
                                                 const int32_t *__restrict__ off,
                                                 const int32_t *n_dev, int n_host,
                                                 int32_t *__restrict__ perm, DevState *st, int train)
{
    if (skip_update(st, train)) return;
    body_scatter(assign, M, R, table, off, cur_n(n_dev, n_host), perm, blockIdx.x);
}

template <int G>
__global__ void __launch_bounds__(256)
    k_cellsum_v4(const float *__restrict__ X, int64_t M, const int32_t *__restrict__ perm,
                 const int32_t *__restrict__ off, const int32_t *n_dev, int n_host, int64_t S,
                 float *__restrict__ pieces, DevState *st, int train)
{
    if (skip_update(st, train)) return;
    body_cellsum_v4<G>(X, M, perm, off, cur_n(n_dev, n_host), S, pieces, blockIdx.x);
}

__global__ void __launch_bounds__(256)
    k_cellsum_any(const float *__restrict__ X, int64_t M, int L, const int32_t *__restrict__ perm,
                  const int32_t *__restrict__ off, const int32_t *n_dev, int n_host, int64_t S,
                  float *__restrict__ pieces, DevState *st, int train)
{
    if (skip_update(st, train)) return;
    body_cellsum_any(X, M, L, perm, off, cur_n(n_dev, n_host), S, pieces, blockIdx.x);
}

// ---------------------------------------------------------------- fused update (step, train)
// k_scan_offsets_q: per cell, the exclusive prefix of its chunk counts and the
// cell size (body_scan); its last CTA then computes the cell offsets
// (body_offsets) and, in the same pass over each thread's cells, for the centroid
// kernel below, the cell holding the first row of every warp piece (qcell[q] =
// the cell n with off[n] <= q S < off[n+1]), zeroes the per-cell piece counters
// and copies the codevector of every empty cell to C_out (an empty cell keeps
// its codevector) when C_out is not C_in (PieceCells).
__global__ void __launch_bounds__(1024)
    k_scan_offsets_q(int32_t *__restrict__ table, int CH, const int32_t *n_dev, int n_host,
                     int32_t *__restrict__ counts, int32_t *__restrict__ off, int32_t *__restrict__ qcell,
                     int32_t *__restrict__ cell_done, int64_t S, int L, const float *C_in, float *C_out,
                     DevState *st, int train)
{
    if (skip_counts(st, train)) return;
    const int N = cur_n(n_dev, n_host);
    if ((int)blockIdx.x * 32 < N) body_scan(table, CH, N, counts, blockIdx.x);
    if (!last_cta(st)) return;
    if (threadIdx.x == 0) st->done_ctr = 0u;
    body_offsets(counts, N, off, PieceCells{N, S, L, cell_done, C_out != C_in && !skip_update(st, train), C_in, C_out});
    __syncthreads();   // off[] complete (this CTA wrote it)
    // qcell[q] = the cell holding row position q S: the largest n with off[n] <= q S
    const int64_t nq = ((int64_t)off[N] + S - 1) / S;
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) qcell[q] = first_cell(off, N, q * S);
}

template <int G>
__global__ void __launch_bounds__(256)
    k_cellsum_c(const float *__restrict__ X, int64_t M, const int32_t *__restrict__ perm,
                const int32_t *__restrict__ off, const int32_t *__restrict__ qcell, const int32_t *n_dev,
                int n_host, int64_t S, float *__restrict__ pieces, int32_t *__restrict__ cell_done,
                float *__restrict__ C_out, DevState *st, int train)
{
    if (skip_update(st, train)) return;
    body_cellsum_c<G>(X, M, perm, off, qcell, cur_n(n_dev, n_host), S, pieces, cell_done, C_out,
                      (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5));
}

// Any L: as body_cellsum_any, with the pieces finished as above.
__global__ void __launch_bounds__(256)
    k_cellsum_c_any(const float *__restrict__ X, int64_t M, int L, const int32_t *__restrict__ perm,
                    const int32_t *__restrict__ off, const int32_t *__restrict__ qcell,
                    const int32_t *n_dev, int n_host, int64_t S, float *__restrict__ pieces,
                    int32_t *__restrict__ cell_done, float *__restrict__ C_out, DevState *st, int train)
{
    if (skip_update(st, train)) return;
    body_cellsum_c_any(X, M, L, perm, off, qcell, cur_n(n_dev, n_host), S, pieces, cell_done, C_out,
                       (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5));
}

// ---------------------------------------------------------------- backward
// Distortion at a fixed cell table, D = sum_m ||x_m - c_a(m)||^2, and its
// gradients (the differentiable form of the paper's distortion).  One warp
// per row group: G lanes read a row with float4 loads (L = 4G), lane sums in
// index order within its float4, a fixed shuffle tree across the G lanes.
//   e[m]  = ||x_m - c_a(m)||^2            (for D through k_hist / k_ctl)
//   dX[m] = 2 gD (x_m - c_a(m))           (nullable)
__global__ void __launch_bounds__(256) k_grad_x(const float *__restrict__ X, int64_t M, int L,
                                                const float *__restrict__ C, int N,
                                                const int32_t *__restrict__ assign, float gD,
                                                const float *__restrict__ gD_dev,
                                                float *__restrict__ e, float *__restrict__ dX,
                                                DevState *st)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    int a = assign[m];
    if (a < 0 || a >= N) {
        flag_error(st, ERR_INTERNAL);
        a = a < 0 ? 0 : N - 1;
    }
    const float *xr = X + m * L;
    const float *cr = C + (int64_t)a * L;
    float *gr = dX ? dX + m * L : nullptr;
    const float g2 = 2.0f * (gD_dev ? *gD_dev : gD);
    float d2 = 0.f;
    for (int l = 0; l < L; ++l) {
        const float d = xr[l] - cr[l];
        d2 = fmaf(d, d, d2);
        if (gr) gr[l] = g2 * d;
    }
    e[m] = d2;
}

// dC_n = 2 gD (count_n c_n - sum_{a(m)=n} x_m): the cell sums come from the
// same deterministic pieces as the centroid update (FP64 combine in order).
__global__ void k_combine_grad(const float *__restrict__ pieces, const int32_t *__restrict__ off,
                               int N, int L, int64_t S, const float *__restrict__ C, float gD,
                               const float *__restrict__ gD_dev, float *__restrict__ dC)
{
    if (gD_dev) gD = *gD_dev;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * L) return;
    const int n = (int)(i / L), l = (int)(i - (int64_t)n * L);
    const int64_t a = off[n], b = off[n + 1];
    double s = 0.0;
    if (b > a) {
        const int64_t q0 = a / S, q1 = (b - 1) / S;
        for (int64_t q = q0; q <= q1; ++q) s += (double)pieces[(size_t)(n + q) * L + l];
    }
    dC[i] = (float)(2.0 * (double)gD * ((double)(b - a) * (double)C[i] - s));
}

__global__ void k_split(const float *__restrict__ C_cur, float *__restrict__ C_alt, int L,
                        double delta, int mult, DevState *st)
{
    body_split(C_cur, C_alt, L, delta, mult, st, blockIdx.x);
}

// Empty-cell re-seeding (opt-in variant) after an update: every empty cell e,
// in increasing index order, takes c_b + delta from the cell b with the
// largest count (lowest index on ties), c_b becomes c_b - delta, and e takes
// half of b's count.  One CTA: integer counts in shared memory, a fixed-order
// argmax per empty cell.
__global__ void __launch_bounds__(1024) k_reseed(const int32_t *__restrict__ off,
                                                 const int32_t *n_dev, int n_host, int L,
                                                 double delta, float *__restrict__ C, DevState *st,
                                                 int train)
{
    if (skip_update(st, train)) return;
    extern __shared__ int cnt[];
    __shared__ int wbest[32], wcount[32];
    __shared__ int s_b;
    const int N = cur_n(n_dev, n_host);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int n = t; n < N; n += 1024) cnt[n] = off[n + 1] - off[n];
    __syncthreads();
    for (int e = 0; e < N; ++e) {
        if (cnt[e] != 0) continue;   // uniform: every thread reads the same shared value
        int bi = 0x7fffffff, bc = -1;
        for (int n = t; n < N; n += 1024)
            if (cnt[n] > bc) {
                bc = cnt[n];
                bi = n;
            }
        for (int o = 16; o > 0; o >>= 1) {
            const int oc = __shfl_xor_sync(0xffffffffu, bc, o), oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oc > bc || (oc == bc && oi < bi)) {
                bc = oc;
                bi = oi;
            }
        }
        if (lane == 0) {
            wbest[w] = bi;
            wcount[w] = bc;
        }
        __syncthreads();
        if (t == 0) {
            int b = wbest[0], c = wcount[0];
            for (int q = 1; q < 32; ++q)
                if (wcount[q] > c || (wcount[q] == c && wbest[q] < b)) {
                    c = wcount[q];
                    b = wbest[q];
                }
            s_b = c >= 2 ? b : -1;
        }
        __syncthreads();
        const int b = s_b;
        if (b < 0) break;
        for (int l = t; l < L; l += 1024) {
            const double c = (double)C[(int64_t)b * L + l];
            C[(int64_t)e * L + l] = (float)(c + delta);
            C[(int64_t)b * L + l] = (float)(c - delta);
        }
        if (t == 0) {
            cnt[e] = cnt[b] / 2;
            cnt[b] -= cnt[e];
        }
        __syncthreads();
    }
}

__global__ void k_copy_split(const float *__restrict__ C_alt, float *__restrict__ C_cur, int L,
                             DevState *st)
{
    body_copy_split(C_alt, C_cur, L, st, blockIdx.x);
}

__global__ void k_stage(DevState *st) { body_stage(st); }

// ---------------------------------------------------------------- pass trace
// Start of a pass of lbg_train with a trace: marks whether the pass runs (a
// pass issued after training ended does not), stamps its start and copies the
// codebook its allocation uses (the stage's n_cur rows) to trace slot
// st->total (the pass's index over the run).
__global__ void __launch_bounds__(256) k_trace_begin(DevState *st, const float *__restrict__ C, int N,
                                                     int L, float *__restrict__ trace_C, int cap)
{
    const bool run = !st->finished;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->trace_on = run ? 1 : 0;
        if (run) st->t_pass0 = global_ns();
    }
    if (!run || !trace_C) return;
    const int slot = st->total;
    if (slot >= cap) return;
    const int64_t n = (int64_t)st->n_cur * L;
    float *dst = trace_C + (int64_t)slot * N * L;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = C[i];
}

// End of a traced pass (its record is slot st->total - 1): the pass's cell
// table to its trace slot; block 0 counts the stage's empty cells and writes
// them and the pass's device time into the record.
__global__ void __launch_bounds__(256) k_trace_end(DevState *st, const int32_t *__restrict__ assign,
                                                   int64_t M, const int32_t *__restrict__ counts,
                                                   PassRecord *rec, int max_rec,
                                                   int32_t *__restrict__ trace_A, int cap)
{
    if (!st->trace_on) return;
    const int slot = st->total - 1;
    if (slot < 0) return;
    if (trace_A && slot < cap) {
        int32_t *dst = trace_A + (int64_t)slot * M;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
            dst[i] = assign[i];
    }
    if (blockIdx.x != 0 || !rec || slot >= max_rec) return;
    __shared__ int wsum[8];
    const int n = rec[slot].stage_n;
    int empty = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) empty += counts[i] == 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) empty += __shfl_xor_sync(0xffffffffu, empty, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = empty;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < 8; ++w) t += wsum[w];
        rec[slot].n_empty = t;
        rec[slot].ms = (float)((double)(global_ns() - st->t_pass0) * 1e-6);
    }
}

// ---------------------------------------------------------------- batched
// One launch per step for every problem of a batched call: block b serves
// problem s = find_set(pre, S, b), local block b - pre[s]; problems that
// have finished training (or whose step is skipped) return at once.
__device__ __forceinline__ int set_of(const int32_t *pre, int S, int &local)
{
    const int s = find_set(pre, S, blockIdx.x);
    local = blockIdx.x - pre[s];
    return s;
}

__global__ void __launch_bounds__(256) kb_mean(const BatchSet *__restrict__ sets, int S,
                                               const int32_t *__restrict__ pre, int L)
{
    int b;
    const int s = set_of(pre, S, b);
    const BatchSet &q = sets[s];
    body_mean_part(q.X, q.M, L, q.mpart, q.st, b, q.G);
}

__global__ void kb_mean_final(const BatchSet *__restrict__ sets, int L)
{
    const BatchSet &q = sets[blockIdx.x];
    const int l = threadIdx.x;
    if (l >= L) return;
    double acc = 0.0;
    for (int b = 0; b < q.G; ++b) acc += q.mpart[(size_t)b * L + l];
    const float c = (float)(acc / (double)q.M);
    q.mu[l] = c;
    q.C[l] = c;
}

__global__ void __launch_bounds__(HIST_THREADS) kb_hist(const BatchSet *__restrict__ sets, int S,
                                                        const int32_t *__restrict__ pre)
{
    int b;
    const int s = set_of(pre, S, b);
    const BatchSet &q = sets[s];
    if (q.st->finished) return;
    body_hist(q.assign, q.e, q.M, q.R, q.st->n_cur, 1, q.table, q.dpart, q.st, b);
}

__global__ void kb_ctl(const BatchSet *__restrict__ sets, double theta, int max_passes)
{
    const BatchSet &q = sets[blockIdx.x];
    if (q.st->finished) return;
    body_ctl(q.dpart, q.CH, q.st, MODE_TRAIN, theta, max_passes, q.N, nullptr, 0);
}

__global__ void __launch_bounds__(1024) kb_scan(const BatchSet *__restrict__ sets, int S,
                                                const int32_t *__restrict__ pre)
{
    int b;
    const int s = set_of(pre, S, b);
    const BatchSet &q = sets[s];
    if (skip_update(q.st, 1)) return;
    body_scan(q.table, q.CH, q.st->n_cur, q.counts, b);
}

__global__ void __launch_bounds__(1024) kb_offsets(const BatchSet *__restrict__ sets)
{
    const BatchSet &q = sets[blockIdx.x];
    if (skip_update(q.st, 1)) return;
    body_offsets(q.counts, q.st->n_cur, q.off);
}

__global__ void __launch_bounds__(256) kb_scatter(const BatchSet *__restrict__ sets, int S,
                                                  const int32_t *__restrict__ pre)
{
    int b;
    const int s = set_of(pre, S, b);
    const BatchSet &q = sets[s];
    if (skip_update(q.st, 1)) return;
    body_scatter(q.assign, q.M, q.R, q.table, q.off, q.st->n_cur, q.perm, b);
}

template <int G>
__global__ void __launch_bounds__(256) kb_cellsum_v4(const BatchSet *__restrict__ sets, int S,
                                                     const int32_t *__restrict__ pre)
{
    int b;
    const int s = set_of(pre, S, b);
    const BatchSet &q = sets[s];
    if (skip_update(q.st, 1)) return;
    body_cellsum_v4<G>(q.X, q.M, q.perm, q.off, q.st->n_cur, q.S, q.pieces, b);
}

__global__ void __launch_bounds__(256) kb_cellsum_any(const BatchSet *__restrict__ sets, int S,
                                                      const int32_t *__restrict__ pre, int L)
{
    int b;
    const int s = set_of(pre, S, b);
    const BatchSet &q = sets[s];
    if (skip_update(q.st, 1)) return;
    body_cellsum_any(q.X, q.M, L, q.perm, q.off, q.st->n_cur, q.S, q.pieces, b);
}

__global__ void kb_combine(const BatchSet *__restrict__ sets, int S, const int32_t *__restrict__ pre,
                           int L)
{
    int b;
    const int s = set_of(pre, S, b);
    const BatchSet &q = sets[s];
    if (skip_update(q.st, 1)) return;
    const int N = q.st->n_cur;
    if ((int64_t)b * blockDim.x >= (int64_t)N * L) return;
    body_combine(q.pieces, q.off, N, L, q.S, q.C, q.C, b);
}

__global__ void kb_split(const BatchSet *__restrict__ sets, int S, const int32_t *__restrict__ pre,
                         int L, double delta, int mult)
{
    int b;
    const int s = set_of(pre, S, b);
    const BatchSet &q = sets[s];
    body_split(q.C, q.Calt, L, delta, mult, q.st, b);
}

__global__ void kb_copy_split(const BatchSet *__restrict__ sets, int S,
                              const int32_t *__restrict__ pre, int L)
{
    int b;
    const int s = set_of(pre, S, b);
    const BatchSet &q = sets[s];
    body_copy_split(q.Calt, q.C, L, q.st, b);
}

__global__ void kb_stage(const BatchSet *__restrict__ sets) { body_stage(sets[blockIdx.x].st); }

}  // namespace

void launch_mean(const float *X, int64_t M, int L, double *part, int G, float *mu, float *C0,
                 DevState *st, cudaStream_t s)
{
    LBG_COUNTED k_mean_part<<<G, 256, 0, s>>>(X, M, L, part, st);
    LBG_COUNTED k_mean_final<<<1, 128, 0, s>>>(part, G, M, L, mu, C0);
}

void launch_hist(const int32_t *assign, const float *e, int64_t M, int64_t R, int CH,
                 const int32_t *n_dev, int n_host, bool do_hist, int32_t *table, double *dpart,
                 DevState *st, bool train, cudaStream_t s)
{
    const size_t smem = do_hist ? (size_t)n_host * sizeof(int) : 0;
    cudaFuncSetAttribute(k_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LBG_COUNTED k_hist<<<CH, HIST_THREADS, smem, s>>>(assign, e, M, R, n_dev, n_host, do_hist ? 1 : 0, table,
                                          dpart, st, train ? 1 : 0);
}

void launch_ctl(const double *dpart, int CH, DevState *st, int mode, double theta, int max_passes,
                int N_target, PassRecord *records, int max_records, cudaStream_t s)
{
    LBG_COUNTED k_ctl<<<1, 32, 0, s>>>(dpart, CH, st, mode, theta, max_passes, N_target, records, max_records);
}

void launch_hist_ctl(const int32_t *assign, const float *e, int64_t M, int64_t R, int CH, int N,
                     bool do_hist, int32_t *table, double *dpart, DevState *st, cudaStream_t s)
{
    const size_t smem = do_hist ? (size_t)N * sizeof(int) : 0;
    cudaFuncSetAttribute(k_hist_ctl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LBG_COUNTED k_hist_ctl<<<CH, HIST_THREADS, smem, s>>>(assign, e, M, R, N, do_hist ? 1 : 0, table, dpart, st);
}

void launch_scan_offsets(int32_t *table, int CH, int N, int32_t *counts, int32_t *off, DevState *st,
                         cudaStream_t s)
{
    LBG_COUNTED k_scan_offsets<<<(N + 31) / 32, 1024, 0, s>>>(table, CH, N, counts, off, st);
}

void launch_scatter(const int32_t *assign, int64_t M, int64_t R, int CH, const int32_t *table,
                    const int32_t *off, const int32_t *n_dev, int n_host, int32_t *perm,
                    DevState *st, bool train, cudaStream_t s)
{
    const size_t smem = (size_t)n_host * (sizeof(int) + 8);
    cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LBG_COUNTED k_scatter<<<CH, 256, smem, s>>>(assign, M, R, table, off, n_dev, n_host, perm, st,
                                    train ? 1 : 0);
}

void launch_cellsum(const float *X, int64_t M, int L, const int32_t *perm, const int32_t *off,
                    const int32_t *n_dev, int n_host, int64_t S, float *pieces, DevState *st,
                    bool train, cudaStream_t s)
{
    const int64_t warps = (M + S - 1) / S;
    if (warps == 0) return;
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    const int t = train ? 1 : 0;
    const bool al = (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
    switch (al ? L : 0) {
    case 4: LBG_COUNTED k_cellsum_v4<1><<<blocks, 256, 0, s>>>(X, M, perm, off, n_dev, n_host, S, pieces, st, t); break;
    case 8: LBG_COUNTED k_cellsum_v4<2><<<blocks, 256, 0, s>>>(X, M, perm, off, n_dev, n_host, S, pieces, st, t); break;
    case 16: LBG_COUNTED k_cellsum_v4<4><<<blocks, 256, 0, s>>>(X, M, perm, off, n_dev, n_host, S, pieces, st, t); break;
    case 32: LBG_COUNTED k_cellsum_v4<8><<<blocks, 256, 0, s>>>(X, M, perm, off, n_dev, n_host, S, pieces, st, t); break;
    case 64: LBG_COUNTED k_cellsum_v4<16><<<blocks, 256, 0, s>>>(X, M, perm, off, n_dev, n_host, S, pieces, st, t); break;
    case 128: LBG_COUNTED k_cellsum_v4<32><<<blocks, 256, 0, s>>>(X, M, perm, off, n_dev, n_host, S, pieces, st, t); break;
    default:
        LBG_COUNTED k_cellsum_any<<<blocks, 256, 0, s>>>(X, M, L, perm, off, n_dev, n_host, S, pieces, st, t);
    }
}

void launch_scan_offsets_q(int32_t *table, int CH, const int32_t *n_dev, int n_host, int32_t *counts,
                           int32_t *off, int32_t *qcell, int32_t *cell_done, int64_t S, int L,
                           const float *C_in, float *C_out, DevState *st, bool train, cudaStream_t s)
{
    LBG_COUNTED k_scan_offsets_q<<<(n_host + 31) / 32, 1024, 0, s>>>(table, CH, n_dev, n_host, counts, off, qcell,
                                                                   cell_done, S, L, C_in, C_out, st,
                                                                   train ? 1 : 0);
}
void launch_cellsum_c(const float *X, int64_t M, int L, const int32_t *perm, const int32_t *off,
                      const int32_t *qcell, const int32_t *n_dev, int n_host, int64_t S, float *pieces,
                      int32_t *cell_done, float *C_out, DevState *st, bool train, cudaStream_t s)
{
    const int64_t warps = (M + S - 1) / S;
    if (warps == 0) return;
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    const int t = train ? 1 : 0;
    const bool al = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(C_out)) & 15u) == 0;
    switch (al ? L : 0) {
    case 4: LBG_COUNTED k_cellsum_c<1><<<blocks, 256, 0, s>>>(X, M, perm, off, qcell, n_dev, n_host, S, pieces, cell_done, C_out, st, t); break;
    case 8: LBG_COUNTED k_cellsum_c<2><<<blocks, 256, 0, s>>>(X, M, perm, off, qcell, n_dev, n_host, S, pieces, cell_done, C_out, st, t); break;
    case 16: LBG_COUNTED k_cellsum_c<4><<<blocks, 256, 0, s>>>(X, M, perm, off, qcell, n_dev, n_host, S, pieces, cell_done, C_out, st, t); break;
    case 32: LBG_COUNTED k_cellsum_c<8><<<blocks, 256, 0, s>>>(X, M, perm, off, qcell, n_dev, n_host, S, pieces, cell_done, C_out, st, t); break;
    case 64: LBG_COUNTED k_cellsum_c<16><<<blocks, 256, 0, s>>>(X, M, perm, off, qcell, n_dev, n_host, S, pieces, cell_done, C_out, st, t); break;
    case 128: LBG_COUNTED k_cellsum_c<32><<<blocks, 256, 0, s>>>(X, M, perm, off, qcell, n_dev, n_host, S, pieces, cell_done, C_out, st, t); break;
    default:
        LBG_COUNTED k_cellsum_c_any<<<blocks, 256, 0, s>>>(X, M, L, perm, off, qcell, n_dev, n_host, S, pieces, cell_done, C_out, st, t);
    }
}

void launch_b_mean(const BatchSet *sets, int S, const int32_t *pre_mean, int total_blocks, int L,
                   cudaStream_t s)
{
    LBG_COUNTED kb_mean<<<total_blocks, 256, 0, s>>>(sets, S, pre_mean, L);
    LBG_COUNTED kb_mean_final<<<S, 128, 0, s>>>(sets, L);
}

void launch_b_hist(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int NMAXB,
                   cudaStream_t s)
{
    const size_t smem = (size_t)NMAXB * sizeof(int);
    cudaFuncSetAttribute(kb_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LBG_COUNTED kb_hist<<<total_blocks, HIST_THREADS, smem, s>>>(sets, S, pre);
}

void launch_b_ctl(const BatchSet *sets, int S, double theta, int max_passes, cudaStream_t s)
{
    LBG_COUNTED kb_ctl<<<S, 32, 0, s>>>(sets, theta, max_passes);
}

void launch_b_scan(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, cudaStream_t s)
{
    LBG_COUNTED kb_scan<<<total_blocks, 1024, 0, s>>>(sets, S, pre);
}

void launch_b_offsets(const BatchSet *sets, int S, cudaStream_t s)
{
    LBG_COUNTED kb_offsets<<<S, 1024, 0, s>>>(sets);
}

void launch_b_scatter(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int NMAXB,
                      cudaStream_t s)
{
    const size_t smem = (size_t)NMAXB * (sizeof(int) + 8);
    cudaFuncSetAttribute(kb_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LBG_COUNTED kb_scatter<<<total_blocks, 256, smem, s>>>(sets, S, pre);
}

void launch_b_cellsum(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int L,
                      bool vec, cudaStream_t s)
{
    switch (vec ? L : 0) {
    case 4: LBG_COUNTED kb_cellsum_v4<1><<<total_blocks, 256, 0, s>>>(sets, S, pre); break;
    case 8: LBG_COUNTED kb_cellsum_v4<2><<<total_blocks, 256, 0, s>>>(sets, S, pre); break;
    case 16: LBG_COUNTED kb_cellsum_v4<4><<<total_blocks, 256, 0, s>>>(sets, S, pre); break;
    case 32: LBG_COUNTED kb_cellsum_v4<8><<<total_blocks, 256, 0, s>>>(sets, S, pre); break;
    case 64: LBG_COUNTED kb_cellsum_v4<16><<<total_blocks, 256, 0, s>>>(sets, S, pre); break;
    case 128: LBG_COUNTED kb_cellsum_v4<32><<<total_blocks, 256, 0, s>>>(sets, S, pre); break;
    default: LBG_COUNTED kb_cellsum_any<<<total_blocks, 256, 0, s>>>(sets, S, pre, L);
    }
}

void launch_b_combine(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int L,
                      cudaStream_t s)
{
    LBG_COUNTED kb_combine<<<total_blocks, 256, 0, s>>>(sets, S, pre, L);
}

void launch_b_split(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int L,
                    double delta, bool mult, cudaStream_t s)
{
    LBG_COUNTED kb_split<<<total_blocks, 256, 0, s>>>(sets, S, pre, L, delta, mult ? 1 : 0);
}

void launch_b_advance(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int L,
                      cudaStream_t s)
{
    LBG_COUNTED kb_copy_split<<<total_blocks, 256, 0, s>>>(sets, S, pre, L);
    LBG_COUNTED kb_stage<<<S, 32, 0, s>>>(sets);
}

void launch_grad_x(const float *X, int64_t M, int L, const float *C, int N, const int32_t *assign,
                   float gD, const float *gD_dev, float *e, float *dX, DevState *st, cudaStream_t s)
{
    if (M == 0) return;
    LBG_COUNTED k_grad_x<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(X, M, L, C, N, assign, gD, gD_dev, e, dX, st);
}

void launch_combine_grad(const float *pieces, const int32_t *off, int N, int L, int64_t S,
                         const float *C, float gD, const float *gD_dev, float *dC, cudaStream_t s)
{
    const int64_t total = (int64_t)N * L;
    LBG_COUNTED k_combine_grad<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(pieces, off, N, L, S, C, gD, gD_dev, dC);
}

void launch_split(const float *C_cur, float *C_alt, int N_alloc, int L, double delta, bool mult,
                  DevState *st, cudaStream_t s)
{
    const int64_t total = (int64_t)(N_alloc / 2 > 0 ? N_alloc / 2 : 1) * L;
    LBG_COUNTED k_split<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(C_cur, C_alt, L, delta, mult ? 1 : 0, st);
}

void launch_reseed(const int32_t *off, const int32_t *n_dev, int n_host, int L, double delta,
                   float *C, DevState *st, bool train, cudaStream_t s)
{
    const size_t smem = (size_t)n_host * sizeof(int);
    cudaFuncSetAttribute(k_reseed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LBG_COUNTED k_reseed<<<1, 1024, smem, s>>>(off, n_dev, n_host, L, delta, C, st, train ? 1 : 0);
}

void launch_trace_begin(DevState *st, const float *C, int N, int L, float *trace_C, int cap,
                        cudaStream_t s)
{
    int blocks = (int)(((int64_t)N * L + 1023) / 1024);
    if (blocks < 1) blocks = 1;
    LBG_COUNTED k_trace_begin<<<blocks, 256, 0, s>>>(st, C, N, L, trace_C, cap);
}

void launch_trace_end(DevState *st, const int32_t *assign, int64_t M, const int32_t *counts,
                      PassRecord *rec, int max_rec, int32_t *trace_A, int cap, cudaStream_t s)
{
    int64_t blocks = trace_A ? (M + 1023) / 1024 : 1;
    if (blocks > 2 * (int64_t)num_sms()) blocks = 2 * (int64_t)num_sms();
    if (blocks < 1) blocks = 1;
    LBG_COUNTED k_trace_end<<<(unsigned)blocks, 256, 0, s>>>(st, assign, M, counts, rec, max_rec, trace_A, cap);
}

void launch_advance(const float *C_alt, float *C_cur, int N_alloc, int L, DevState *st,
                    cudaStream_t s)
{
    const int64_t total = (int64_t)N_alloc * L;
    LBG_COUNTED k_copy_split<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(C_alt, C_cur, L, st);
    LBG_COUNTED k_stage<<<1, 32, 0, s>>>(st);
}

}  // namespace lbg
