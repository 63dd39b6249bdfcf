// k_assign.cu -- cell allocation (nearest codevector) kernels.
//
// Paper: Algorithm 1 "Cell Allocation" and Sec. 2.2 step 1 (minimum
// distortion partition): every training vector gets the index of the
// codevector at the smallest squared Euclidean distance (ties: lowest
// index) and its distance is added to the distortion.  The same kernels
// serve encoding (Abstract: replacement by the nearest codevector).
//
// GB300 design.  The search is the contraction -2 x.c over L plus the
// per-codevector norm, done with FP32 FFMA:
//   * a CTA owns BM = 128 rows of X (centred by mu, staged once in shared
//     memory, k-major) and streams the whole prepared codebook through two
//     shared-memory buffers of BN = 128 codevectors, each filled by one TMA
//     bulk copy (cp.async.bulk + mbarrier, bounded waits);
//   * every thread keeps an 8 x 8 register tile of accumulators whose FMA
//     chain starts at a per-codevector constant, so the tile needs no
//     epilogue arithmetic besides a running top-2 over split pairs (the
//     minimum of codevectors 2k, 2k + 1, then 3 FMNMX: 2 per distance);
//   * the index of the minimum is recovered after the sweep by recomputing
//     the one winning 8-codevector group bit-identically;
//   * a rigorous rounding-error bound certifies the minimum; rows it cannot
//     certify (about 0.2% on image blocks) are re-scored exactly in FP32
//     direct form by k_assign_exact_split (k_assign_exact in the batched and
//     no-allocation paths).
//
// Certification.  Let x~ = fl(x - mu), c~_n = fl(c_n - mu), u = 2^-24 and
//   k_n = 2 (L+2) u ||c~_n||^2,  R = (L+2) u ||x~||^2.
// The chain computes v_n ~ f_n - k_n with f_n = ||c~_n||^2 - 2 x~.c~_n and
// |v_n - (f_n - k_n)| <= (L+1)(1+Lu) u (||c~_n||^2 + 2||x~|| ||c~_n||)
//                     <= k_n + R          (2ab <= a^2 + b^2),
// hence v_n - R <= f_n <= v_n + 2 k_n + R.  The codevectors are taken in pairs
// P = (2k, 2k + 1) -- the two children of a split.  If V1 = v_i1 is the minimum,
// P* its pair and V2 the smallest value outside P*, V2 - V1 > 2R + 2k_P*
// (k_P* the larger k of the pair) proves f_n > f_i1 for all n outside P*, i.e.
// ||x~ - c~_n|| > ||x~ - c~_i1||.  Centring moves each distance ||x - c_n|| by
// at most eta = u (||x~|| + max ||c~||); the extra term 4 eta (g1 + eta),
// g1 >= ||x~ - c~_i1||, keeps the proof valid for the original x and c_n.  The
// exact argmin is then i1 or its partner: the one whose FP32 direct-form
// distance is smaller by more than that form's rounding bound (else the row
// is not certified).  Right after a split a row's two nearest codevectors are
// often such twins; they are told apart exactly here instead of failing the
// bound.
#include "bodies_assign.cuh"
#include "lbg_internal.cuh"

#include <math.h>

namespace lbg {
namespace {

// mu[l] = mean over the N codevectors (fixed-order FP32 tree); the centring
// vector of lbg_lloyd_step / vq_encode.  One CTA of 256 threads per dimension.
__global__ void __launch_bounds__(256) k_codebook_mean(const float *__restrict__ C, int N, int L,
                                                       float *__restrict__ mu)
{
    __shared__ float part[256];
    const int l = blockIdx.x, t = threadIdx.x;
    float s = 0.f;
    for (int n = t; n < N; n += 256) s += C[(size_t)n * L + l];
    part[t] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) part[t] += part[t + h];
        __syncthreads();
    }
    if (t == 0) mu[l] = part[0] / (float)N;
}

// Start of a Lloyd step / encode in one launch: the codebook mean mu (CTA l sums
// column l as k_codebook_mean does), rounded to integers for the tensor-core
// form, and the initial device state (CTA 0; st may be null).
__global__ void __launch_bounds__(256) k_begin(const float *__restrict__ C, int N, int L,
                                               float *__restrict__ mu, int round_mu, DevState *st,
                                               int n_cur)
{
    __shared__ float part[256];
    const int l = blockIdx.x, t = threadIdx.x;
    float s = 0.f;
    for (int n = t; n < N; n += 256) s += C[(size_t)n * L + l];
    part[t] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) part[t] += part[t + h];
        __syncthreads();
    }
    if (t == 0) {
        const float m = part[0] / (float)N;
        mu[l] = round_mu ? rintf(m) : m;
        if (l == 0 && st) {
            DevState h0 = {};
            h0.n_cur = n_cur;
            h0.D_prev = INFINITY;
            *st = h0;
        }
    }
}

__global__ void __launch_bounds__(256)
    k_prep(const float *__restrict__ C, const int32_t *n_dev, int n_host, int L, int Lp,
           const float *__restrict__ mu, float *__restrict__ Cp, float *__restrict__ kn,
           float *__restrict__ CT, int NP, DevState *st)
{
    if (st->finished || cur_n(n_dev, n_host) <= st->direct_max) return;
    (void)NP;
    __shared__ PrepSmem ps;
    body_prep(C, cur_n(n_dev, n_host), L, Lp, mu, Cp, kn, CT, st, blockIdx.x, ps);
}

// Small codebooks (the early stages of lbg_train, N <= DevState::direct_max):
// every row against all N codevectors in the FP32 direct form, the sum over l
// in index order of fl(x_l - c_l)^2 (an fmaf chain from 0), lowest index on
// ties.  These are the values and the choice the certified search and its
// exact re-scoring produce for every row (a certified winner beats every other
// codevector by more than the rounding of these sums, and a flagged row is
// re-scored this way), so the results do not depend on which kernel ran; at a
// few codevectors the search's tiles, certificate and re-scoring cost far more
// than this arithmetic, which reads X once.  One row per thread (x in
// registers after a coalesced staging of the CTA's 256 rows, L <= LK,
// L % 4 == 0), codevectors read by broadcast loads (the same address in every
// lane), four codevectors' sums at a time.
template <int LK>
__global__ void __launch_bounds__(256)
    k_assign_direct(const float *__restrict__ X, int64_t M, int L, const float *__restrict__ C,
                    const int32_t *n_dev, int n_host, DevState *st, int32_t *__restrict__ assign,
                    float *__restrict__ e)
{
    if (st->finished) return;
    const int N = cur_n(n_dev, n_host);
    if (N > st->direct_max) return;
    if (blockIdx.x == 0) {   // non-finite codevectors (the preparation that checks them is skipped)
        bool bad = false;
        for (int i = threadIdx.x; i < N * L; i += blockDim.x) bad = bad || !isfinite(C[i]);
        if (bad) flag_error(st, ERR_NONFINITE);
    }
    // the CTA's rows, staged through shared memory with coalesced loads (row
    // stride L + 4 floats: a warp's reads of its 32 rows are conflict-free)
    extern __shared__ float4 xs4[];
    const int L4 = L >> 2, rs4 = L4 + 1;
    const int64_t m0 = (int64_t)blockIdx.x * 256;
    const int rows = M - m0 < 256 ? (int)(M - m0) : 256;
    const float4 *Xt = reinterpret_cast<const float4 *>(X + m0 * L);
    const int total4 = rows * L4;
    for (int i0 = threadIdx.x; i0 < total4; i0 += 8 * 256) {   // eight loads in flight per thread
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + 256 * u;
            v[u] = i < total4 ? __ldg(Xt + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + 256 * u, r = i / L4;
            if (i < total4) xs4[r * rs4 + (i - r * L4)] = v[u];
        }
    }
    __syncthreads();
    const int64_t m = m0 + threadIdx.x;
    if (m >= M) return;
    float x[LK];
    bool bad = false;
    const float4 *xr = xs4 + threadIdx.x * rs4;
#pragma unroll
    for (int q = 0; q < LK / 4; ++q) {
        const float4 v = q < L4 ? xr[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        x[4 * q] = v.x;
        x[4 * q + 1] = v.y;
        x[4 * q + 2] = v.z;
        x[4 * q + 3] = v.w;
        bad = bad || !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
    }
    if (bad) flag_error(st, ERR_NONFINITE);
    const float4 *C4 = reinterpret_cast<const float4 *>(C);
    float best = INFINITY;
    int bi = 0;
    for (int n = 0; n < N; n += 4) {   // four codevectors' sums at a time (the last ones repeated)
        const float4 *cp[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) cp[k] = C4 + (size_t)(n + k < N ? n + k : n) * L4;
        float dk[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < LK / 4; ++q) {
            if (q < L4) {
                float4 c[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) c[k] = __ldg(cp[k] + q);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float d = __fsub_rn(x[4 * q], c[k].x);
                    dk[k] = fmaf(d, d, dk[k]);
                    d = __fsub_rn(x[4 * q + 1], c[k].y);
                    dk[k] = fmaf(d, d, dk[k]);
                    d = __fsub_rn(x[4 * q + 2], c[k].z);
                    dk[k] = fmaf(d, d, dk[k]);
                    d = __fsub_rn(x[4 * q + 3], c[k].w);
                    dk[k] = fmaf(d, d, dk[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)   // in index order: the lowest index wins a tie
            if (n + k < N && dk[k] < best) {
                best = dk[k];
                bi = n + k;
            }
    }
    assign[m] = bi;
    e[m] = best;
}

__global__ void __launch_bounds__(ASSIGN_THREADS, 2)
    k_assign_f32(const float *__restrict__ X, int64_t M, int L, int Lp, const float *__restrict__ Cp,
                 const float *__restrict__ kn, const int32_t *n_dev, int n_host,
                 const float *__restrict__ mu, const float *__restrict__ C, DevState *st,
                 int32_t *__restrict__ assign, float *__restrict__ e, int32_t *__restrict__ flags,
                 int64_t m_lo, int expire)
{
    if (st->finished || cur_n(n_dev, n_host) <= st->direct_max) return;   // k_assign_direct's stages
    extern __shared__ __align__(128) float smem[];
    __shared__ AssignSmem sh;
    if (threadIdx.x == 0) {
        mbar_init(&sh.bar[0], 1);
        mbar_init(&sh.bar[1], 1);
        fence_mbar_init();
        sh.abort = 0;
    }
    __syncthreads();
    uint32_t u0 = 0, u1 = 0;
    (void)assign_f32_tile_t<BM>(X, M, L, Lp, Cp, kn, cur_n(n_dev, n_host), mu, C, st, assign, e, flags,
                                m_lo + (int64_t)blockIdx.x * BM, smem, sh, u0, u1, expire);
}

// Batched problems: a persistent CTA takes (problem, row tile) work items from
// a global counter until all are done; finished problems are skipped.
template <int TBM>
__global__ void __launch_bounds__(2 * TBM, TBM == 128 ? 2 : 4)
    kb_assign_f32(const BatchSet *__restrict__ sets, int S, const int64_t *__restrict__ pre_tiles,
                  int64_t total, int L, int Lp, int *counter)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ AssignSmemT<TBM> sh;
    __shared__ int64_t s_item;
    if (threadIdx.x == 0) {
        mbar_init(&sh.bar[0], 1);
        mbar_init(&sh.bar[1], 1);
        fence_mbar_init();
        sh.abort = 0;
    }
    __syncthreads();
    uint32_t u0 = 0, u1 = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(counter, 1);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const int s = find_set64(pre_tiles, S, item);
        const BatchSet &q = sets[s];
        if (!q.st->finished) {
            const int64_t tile = item - pre_tiles[s];
            if (!assign_f32_tile_t<TBM>(q.X, q.M, L, Lp, q.Cp, q.kn, q.st->n_cur, q.mu, q.C, q.st,
                                        q.assign, q.e, q.flags, tile * TBM, smem, sh, u0, u1))
                break;
        }
        __syncthreads();   // all reads of this item's shared data before the next item
    }
}

__global__ void __launch_bounds__(EX_THREADS)
    k_assign_exact(const float *__restrict__ X, int L, int Lp, const float *__restrict__ CT,
                   const int32_t *n_dev, int n_host, DevState *st, const int32_t *__restrict__ flags,
                   int32_t *__restrict__ assign, float *__restrict__ e)
{
    if (st->finished) return;
    const int nflag = st->nflag;
    const int ngroups = (nflag + EX_R - 1) / EX_R;
    if ((int)blockIdx.x >= ngroups) return;
    extern __shared__ __align__(128) float cbuf[];   // [2][Lp][EX_SW]
    __shared__ __align__(16) ExactSmem sh;
    exact_init(sh);
    uint32_t uses[2] = {0u, 0u};
    const int N = cur_n(n_dev, n_host);
    for (int g = blockIdx.x; g < ngroups; g += gridDim.x)
        if (!exact_group(X, L, Lp, CT, N, st, flags, nflag, assign, e, g, cbuf, sh, uses)) return;
}

// Exact re-scoring spread evenly over the CTAs.  The work is U = groups x
// nchunk units (a group of XS_R flagged rows against one chunk of EX_SW
// codevectors), ordered group-major; CTA b takes the contiguous units
// [b U / G, (b + 1) U / G) of G = min(launched CTAs, U), so every CTA streams about
// the same number of chunks whatever the flagged count (the count is known
// only on the device).  Thread t scores codevector t % EX_SW of each chunk
// against rows 16 (t / EX_SW) .. + 15, d = sum_l (x_l - c_l)^2 in index order
// (terms beyond L are (0 - 0)^2 and leave the sum unchanged), with the
// operands of dimension l + 1 loaded while dimension l is scored.  A CTA keeps
// its rows and running minima while consecutive units share a group.  A group
// that lies in one CTA is finished in place; a group cut by CTA boundaries has
// one segment per CTA it touches: each writes its per-row (d, index) minima to
// its slot (0 for the CTA's first group, 1 for its last), and the last
// segment to arrive (atomic count on the group's first CTA, reset by itself)
// merges them in CTA order, i.e. in codevector order, so ties keep the lowest
// index and the result does not depend on which CTA finishes last.
constexpr int XS_R = 32;
constexpr int XS_HALF = XS_R / 2;
// two resident CTAs per SM: one wave
int xs_ctas() { return 2 * num_sms(); }

struct ExactSplitSmem {
    float xs[LMAX][XS_R];
    uint64_t bar[2];
    int abort, last;
    float rb[EX_THREADS / 32][XS_HALF];
    int ri[EX_THREADS / 32][XS_HALF];
    float rowb[XS_R];
    int rowi[XS_R];
};

// first unit of CTA b; the CTA that takes unit u (the largest b with
// first unit <= u, which is never an empty CTA)
__device__ __forceinline__ int64_t xs_first_unit(int64_t b, int64_t U, int G) { return b * U / G; }
__device__ __forceinline__ int xs_cta_of(int64_t u, int64_t U, int G) { return (int)(((u + 1) * G - 1) / U); }

// d[q] += (x_q - c)^2 for the 16 rows of a thread at one dimension, two rows
// per packed instruction
__device__ __forceinline__ void xs_step(float (&d2)[XS_HALF], const float4 (&x)[4], float c)
{
    uint64_t cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
        sqdiff2(x[q4].x, x[q4].y, cc, d2[4 * q4], d2[4 * q4 + 1]);
        sqdiff2(x[q4].z, x[q4].w, cc, d2[4 * q4 + 2], d2[4 * q4 + 3]);
    }
}

__global__ void __launch_bounds__(EX_THREADS)
    k_assign_exact_split(const float *__restrict__ X, int L, int Lp, const float *__restrict__ CT,
                         const int32_t *n_dev, int n_host, DevState *st, const int32_t *__restrict__ flags,
                         int32_t *__restrict__ assign, float *__restrict__ e, float *__restrict__ part_d,
                         int32_t *__restrict__ part_i, int32_t *__restrict__ cnt)
{
    if (st->finished) return;
    const int nflag = st->nflag;
    const int groups = (nflag + XS_R - 1) / XS_R;
    if (groups == 0) return;
    const int N = cur_n(n_dev, n_host);
    const int nchunk = (N + EX_SW - 1) / EX_SW;
    const int64_t U = (int64_t)groups * nchunk;
    const int G = (int)min((int64_t)gridDim.x, U), b = (int)blockIdx.x;   // G <= U: no CTA is empty
    if (b >= G) return;
    const int64_t u0 = xs_first_unit(b, U, G), u1 = xs_first_unit(b + 1, U, G);
    const int g_first = (int)(u0 / nchunk);

    extern __shared__ __align__(128) float cbuf[];   // [2][Lp][EX_SW]
    __shared__ __align__(16) ExactSplitSmem sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int j = tid % EX_SW, h = tid / EX_SW;
    const uint32_t chunk_floats = (uint32_t)Lp * EX_SW;
    const uint32_t chunk_bytes = chunk_floats * 4u;
    if (tid == 0) {
        mbar_init(&sh.bar[0], 1);
        mbar_init(&sh.bar[1], 1);
        fence_mbar_init();
        sh.abort = 0;
        for (int64_t u = u0; u < u0 + 2 && u < u1; ++u) {   // in flight while the rows are staged
            const int bb = (int)(u - u0) & 1;
            mbar_expect_tx(&sh.bar[bb], chunk_bytes);
            bulk_load(cbuf + bb * chunk_floats, CT + (size_t)(u % nchunk) * chunk_floats, chunk_bytes,
                      &sh.bar[bb]);
        }
    }
    uint32_t uses[2] = {0u, 0u};
    float best[XS_HALF];
    int bi[XS_HALF];
    int g = -1, nr = 0;
    for (int64_t u = u0;; ++u) {
        const int gu = u < u1 ? (int)(u / nchunk) : -1;
        if (gu != g) {
            if (g >= 0) {
                // ---- the segment of group g in this CTA is done: per-row minima ----
#pragma unroll
                for (int q = 0; q < XS_HALF; ++q) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const float ob = __shfl_xor_sync(0xffffffffu, best[q], o);
                        const int oi = __shfl_xor_sync(0xffffffffu, bi[q], o);
                        if (ob < best[q] || (ob == best[q] && oi < bi[q])) {
                            best[q] = ob;
                            bi[q] = oi;
                        }
                    }
                    if (lane == 0) {
                        sh.rb[warp][q] = best[q];
                        sh.ri[warp][q] = bi[q];
                    }
                }
                __syncthreads();
                const int fb = xs_cta_of((int64_t)g * nchunk, U, G);
                const int lb = xs_cta_of((int64_t)(g + 1) * nchunk - 1, U, G);
                const int slot = g == g_first ? 0 : 1;
                if (tid < XS_R) {
                    const int hh = tid / XS_HALF, q = tid % XS_HALF, w0 = hh * (EX_SW / 32);
                    float bb = sh.rb[w0][q];
                    int ii = sh.ri[w0][q];
                    for (int ww = w0 + 1; ww < w0 + EX_SW / 32; ++ww)
                        if (sh.rb[ww][q] < bb || (sh.rb[ww][q] == bb && sh.ri[ww][q] < ii)) {
                            bb = sh.rb[ww][q];
                            ii = sh.ri[ww][q];
                        }
                    sh.rowb[tid] = bb;
                    sh.rowi[tid] = ii;
                    if (fb != lb) {
                        part_d[((size_t)b * 2 + slot) * XS_R + tid] = bb;
                        part_i[((size_t)b * 2 + slot) * XS_R + tid] = ii;
                    }
                }
                bool fin = fb == lb;
                if (!fin) {
                    if (tid < XS_R) __threadfence();   // the partial minima written above
                    __syncthreads();
                    if (tid == 0) sh.last = atomicAdd(&cnt[fb], 1) == lb - fb;
                    __syncthreads();
                    fin = sh.last != 0;
                    if (fin) {
                        if (tid < nr) {   // segments in CTA order = codevector order, 8 loads in flight
                            __threadfence();
                            float bb = INFINITY;
                            int ii = 0x7fffffff;
                            for (int c0 = fb; c0 <= lb; c0 += 8) {
                                float ob[8];
                                int oi[8];
#pragma unroll
                                for (int k = 0; k < 8; ++k) {
                                    const int c = c0 + k;
                                    const int s = c <= lb && (int)(xs_first_unit(c, U, G) / nchunk) != g ? 1 : 0;
                                    ob[k] = c <= lb ? __ldcg(part_d + ((size_t)c * 2 + s) * XS_R + tid) : INFINITY;
                                    oi[k] = c <= lb ? __ldcg(part_i + ((size_t)c * 2 + s) * XS_R + tid) : 0x7fffffff;
                                }
#pragma unroll
                                for (int k = 0; k < 8; ++k)
                                    if (ob[k] < bb || (ob[k] == bb && oi[k] < ii)) {
                                        bb = ob[k];
                                        ii = oi[k];
                                    }
                            }
                            sh.rowb[tid] = bb;
                            sh.rowi[tid] = ii;
                        }
                        if (tid == 0) cnt[fb] = 0;
                    }
                }
                if (fin && tid < nr) {
                    const float bb = sh.rowb[tid];
                    const int ii = sh.rowi[tid];
                    const int row = flags[g * XS_R + tid];
                    const bool valid = ii >= 0 && ii < N;
                    if (!valid) flag_error(st, ERR_NONFINITE);   // only NaN rows compare false everywhere
                    assign[row] = valid ? ii : 0;
                    e[row] = valid ? bb : 0.f;
                }
                __syncthreads();   // rb/ri/rowb and xs are reused
            }
            if (gu < 0) break;
            // ---- stage the rows of group gu, zero beyond L: lane r reads the r-th flag, then
            // each warp loads its rows (coalesced) with every load in flight before the stores ----
            g = gu;
            nr = min(XS_R, nflag - g * XS_R);
            {
                constexpr int RPW = XS_R / (EX_THREADS / 32), VPL = LMAX / 32;
                const int frow = lane < nr ? flags[g * XS_R + lane] : -1;
                float v[RPW][VPL];
#pragma unroll
                for (int k = 0; k < RPW; ++k) {
                    const int row = __shfl_sync(0xffffffffu, frow, warp + k * (EX_THREADS / 32));
#pragma unroll
                    for (int i = 0; i < VPL; ++i) {
                        const int l = lane + 32 * i;
                        v[k][i] = row >= 0 && l < L ? X[(int64_t)row * L + l] : 0.f;
                    }
                }
#pragma unroll
                for (int k = 0; k < RPW; ++k)
#pragma unroll
                    for (int i = 0; i < VPL; ++i)
                        if (lane + 32 * i < Lp) sh.xs[lane + 32 * i][warp + k * (EX_THREADS / 32)] = v[k][i];
            }
#pragma unroll
            for (int q = 0; q < XS_HALF; ++q) {
                best[q] = INFINITY;
                bi[q] = 0x7fffffff;
            }
            __syncthreads();
        }
        // ---- unit u: chunk u % nchunk against the staged rows ----
        const int bsel = (int)(u - u0) & 1;
        const bool ok = mbar_wait_bounded(&sh.bar[bsel], uses[bsel] & 1u);
        uses[bsel] += 1u;
        if (!ok) sh.abort = 1;
        const int n = (int)(u % nchunk) * EX_SW + j;
        if (ok && n < N) {
            const float *cq = cbuf + bsel * chunk_floats + j;
            const float *xq = &sh.xs[0][h * XS_HALF];
            float d2[XS_HALF];
#pragma unroll
            for (int q = 0; q < XS_HALF; ++q) d2[q] = 0.f;
            float4 xa[4], xb[4];
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) xa[q4] = lds4(xq + 4 * q4);
            float ca = cq[0];
            for (int l = 0; l < Lp; l += 2) {   // Lp is a multiple of 4
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) xb[q4] = lds4(xq + (l + 1) * XS_R + 4 * q4);
                const float cb2 = cq[(l + 1) * EX_SW];
                xs_step(d2, xa, ca);
                if (l + 2 < Lp) {
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) xa[q4] = lds4(xq + (l + 2) * XS_R + 4 * q4);
                    ca = cq[(l + 2) * EX_SW];
                }
                xs_step(d2, xb, cb2);
            }
#pragma unroll
            for (int q = 0; q < XS_HALF; ++q)
                if (d2[q] < best[q]) {
                    best[q] = d2[q];
                    bi[q] = n;
                }
        }
        __syncthreads();
        if (sh.abort) {
            if (tid == 0) {
                if (u + 1 < u1)
                    (void)mbar_wait_bounded(&sh.bar[bsel ^ 1], uses[bsel ^ 1] & 1u);
                flag_error(st, ERR_TIMEOUT);
            }
            return;
        }
        if (tid == 0 && u + 2 < u1) {
            mbar_expect_tx(&sh.bar[bsel], chunk_bytes);
            bulk_load(cbuf + bsel * chunk_floats, CT + (size_t)((u + 2) % nchunk) * chunk_floats, chunk_bytes,
                      &sh.bar[bsel]);
        }
    }
}

// Batched problems: the flagged groups of all problems form one work list
// (problem order, then group order); a persistent grid strides through it.
__global__ void __launch_bounds__(EX_THREADS)
    kb_assign_exact(const BatchSet *__restrict__ sets, int S, int L, int Lp)
{
    extern __shared__ __align__(128) float cbuf[];
    __shared__ __align__(16) ExactSmem sh;
    __shared__ int s_total;
    if (threadIdx.x == 0) {
        int t = 0;
        for (int s = 0; s < S; ++s)
            if (!sets[s].st->finished) t += (sets[s].st->nflag + EX_R - 1) / EX_R;
        s_total = t;
    }
    __syncthreads();
    const int total = s_total;
    if ((int)blockIdx.x >= total) return;
    exact_init(sh);
    uint32_t uses[2] = {0u, 0u};
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int s = 0, g = item;
        for (; s < S; ++s) {
            if (sets[s].st->finished) continue;
            const int ng = (sets[s].st->nflag + EX_R - 1) / EX_R;
            if (g < ng) break;
            g -= ng;
        }
        const BatchSet &q = sets[s];
        if (!exact_group(q.X, L, Lp, q.CT, q.st->n_cur, q.st, q.flags, q.st->nflag, q.assign, q.e, g,
                         cbuf, sh, uses))
            return;
    }
}

__global__ void __launch_bounds__(256) kb_prep(const BatchSet *__restrict__ sets, int S,
                                               const int32_t *__restrict__ pre, int L, int Lp)
{
    const int s = find_set(pre, S, blockIdx.x);
    const int b = blockIdx.x - pre[s];
    const BatchSet &q = sets[s];
    if (q.st->finished) return;
    __shared__ PrepSmem ps;
    body_prep(q.C, q.st->n_cur, L, Lp, q.mu, q.Cp, q.kn, q.CT, q.st, b, ps);
}

__global__ void kb_reset(const BatchSet *__restrict__ sets, int S, int *counter)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) *counter = 0;
    if (s < S) sets[s].st->cmax_bits = 0u;
}

__global__ void k_decode(const int32_t *__restrict__ assign, int64_t M, int L,
                         const float *__restrict__ C, float *__restrict__ Xhat)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * L) return;
    const int64_t m = i / L;
    const int l = (int)(i - m * L);
    Xhat[i] = C[(size_t)assign[m] * L + l];
}

}  // namespace

void launch_begin(const float *C, int N, int L, float *mu, bool round_mu, DevState *st, cudaStream_t s)
{
    LBG_COUNTED k_begin<<<L, 256, 0, s>>>(C, N, L, mu, round_mu ? 1 : 0, st, N);
}

void launch_codebook_mean(const float *C, int N, int L, float *mu, cudaStream_t s)
{
    LBG_COUNTED k_codebook_mean<<<L, 256, 0, s>>>(C, N, L, mu);
}

// k_assign_direct serves rows of L % 4 == 0, L <= 64 with X and C 16-byte aligned.
bool direct_supported(int L, const void *X, const void *C)
{
    return (L & 3) == 0 && L <= 64 && ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(C)) & 15u) == 0;
}

void launch_assign_direct(const float *X, int64_t M, int L, const float *C, const int32_t *n_dev, int n_host,
                          DevState *st, int32_t *assign, float *e, cudaStream_t s)
{
    const int64_t grid = (M + 255) / 256;
    if (grid <= 0) return;
    const size_t smem = (size_t)256 * (L / 4 + 1) * sizeof(float4);
#define LBG_DIRECT(LK)                                                                                      \
    cudaFuncSetAttribute(k_assign_direct<LK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
    LBG_COUNTED k_assign_direct<LK><<<(unsigned)grid, 256, smem, s>>>(X, M, L, C, n_dev, n_host, st, assign, e)
    switch (round_up(L, 16)) {
    case 16: LBG_DIRECT(16); break;
    case 32: LBG_DIRECT(32); break;
    case 48: LBG_DIRECT(48); break;
    default: LBG_DIRECT(64); break;
    }
#undef LBG_DIRECT
}

void launch_prep(const float *C, int N_alloc, const int32_t *n_dev, int n_host, int L, int Lp,
                 const float *mu, float *Cp, float *kn, float *CT, int NP, DevState *st,
                 cudaStream_t s)
{
    const int total = round_up(N_alloc, BN);
    LBG_COUNTED k_prep<<<total / PREP_TILE, 256, 0, s>>>(C, n_dev, n_host, L, Lp, mu, Cp, kn, CT, NP, st);
}

size_t assign_smem_bytes(int Lp) { return (size_t)(Lp * BM + 2 * (Lp + 1) * BN) * sizeof(float); }

void launch_assign(const float *X, int64_t M, int L, int Lp, const float *Cp, const float *kn,
                   const int32_t *n_dev, int n_host, const float *mu, const float *C, DevState *st,
                   int32_t *assign, float *e, int32_t *flags, cudaStream_t s, int64_t m_lo, int expire)
{
    const size_t smem = assign_smem_bytes(Lp);
    cudaFuncSetAttribute(k_assign_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t grid = (M - m_lo + BM - 1) / BM;
    if (grid <= 0) return;
    LBG_COUNTED k_assign_f32<<<(unsigned)grid, ASSIGN_THREADS, smem, s>>>(X, M, L, Lp, Cp, kn, n_dev, n_host, mu,
                                                              C, st, assign, e, flags, m_lo, expire);
}

void launch_exact(const float *X, int L, int Lp, const float *CT, const int32_t *n_dev, int n_host,
                  DevState *st, const int32_t *flags, int32_t *assign, float *e, int64_t M,
                  cudaStream_t s)
{
    // CTAs loop over groups of EX_R flagged rows; at most 3 CTAs per SM (the
    // count of flagged rows is only known on the device; spare CTAs exit).
    const size_t smem = (size_t)2 * Lp * EX_SW * sizeof(float);
    cudaFuncSetAttribute(k_assign_exact, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int64_t groups = (M + EX_R - 1) / EX_R;
    const int64_t cap = 3 * (int64_t)num_sms();
    int64_t blocks = groups < cap ? groups : cap;
    if (blocks < 1) blocks = 1;
    LBG_COUNTED k_assign_exact<<<(unsigned)blocks, EX_THREADS, smem, s>>>(X, L, Lp, CT, n_dev, n_host, st, flags,
                                                             assign, e);
}

int exact_split_ctas() { return xs_ctas(); }
int exact_split_rows() { return XS_R; }

void launch_exact_split(const float *X, int L, int Lp, const float *CT, const int32_t *n_dev, int n_host,
                        DevState *st, const int32_t *flags, int32_t *assign, float *e, float *part_d,
                        int32_t *part_i, int32_t *cnt, int64_t M, cudaStream_t s)
{
    const size_t smem = (size_t)2 * Lp * EX_SW * sizeof(float);
    cudaFuncSetAttribute(k_assign_exact_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // the flagged count is known only on the device: up to one wave, at least 16 CTAs per
    // possible group of rows when M is small (CTAs beyond the units exit at once)
    int64_t blocks = (M + XS_R - 1) / XS_R;
    const int64_t wave = xs_ctas();
    blocks = blocks * 16 < wave ? blocks * 16 : wave;
    if (blocks < 1) blocks = 1;
    LBG_COUNTED k_assign_exact_split<<<(unsigned)blocks, EX_THREADS, smem, s>>>(X, L, Lp, CT, n_dev, n_host, st, flags,
                                                                   assign, e, part_d, part_i, cnt);
}

void launch_b_prep(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int L, int Lp,
                   cudaStream_t s)
{
    LBG_COUNTED kb_prep<<<total_blocks, 256, 0, s>>>(sets, S, pre, L, Lp);
}

void launch_b_assign(const BatchSet *sets, int S, const int64_t *pre_tiles, int64_t total_tiles,
                     int L, int Lp, int *counter, int tile_rows, int ctas_per_sm, cudaStream_t s)
{
    // the work counter and the per-problem codebook norms are reset by
    // kb_reset, which runs before kb_prep in the pass (see lbg_train_batched)
    int64_t grid = num_sms() * (int64_t)ctas_per_sm;
    if (grid > total_tiles) grid = total_tiles;
    if (grid < 1) return;
    if (tile_rows == 64) {
        const size_t smem = (size_t)(Lp * 64 + 2 * (Lp + 1) * BN) * sizeof(float);
        cudaFuncSetAttribute(kb_assign_f32<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LBG_COUNTED kb_assign_f32<64><<<(unsigned)grid, 128, smem, s>>>(sets, S, pre_tiles, total_tiles, L, Lp, counter);
    } else {
        const size_t smem = assign_smem_bytes(Lp);
        cudaFuncSetAttribute(kb_assign_f32<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LBG_COUNTED kb_assign_f32<128><<<(unsigned)grid, 256, smem, s>>>(sets, S, pre_tiles, total_tiles, L, Lp, counter);
    }
}

void launch_b_reset(const BatchSet *sets, int S, int *counter, cudaStream_t s)
{
    LBG_COUNTED kb_reset<<<(S + 255) / 256, 256, 0, s>>>(sets, S, counter);
}

void launch_b_exact(const BatchSet *sets, int S, int L, int Lp, int max_ngroups, cudaStream_t s)
{
    const size_t smem = (size_t)2 * Lp * EX_SW * sizeof(float);
    cudaFuncSetAttribute(kb_assign_exact, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int cap = 3 * num_sms();
    int grid = max_ngroups < cap ? max_ngroups : cap;
    if (grid < 1) grid = 1;
    LBG_COUNTED kb_assign_exact<<<grid, EX_THREADS, smem, s>>>(sets, S, L, Lp);
}

void launch_decode(const int32_t *assign, int64_t M, int L, const float *C, float *Xhat,
                   cudaStream_t s)
{
    const int64_t total = M * L;
    if (total == 0) return;
    LBG_COUNTED k_decode<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(assign, M, L, C, Xhat);
}

}  // namespace lbg
