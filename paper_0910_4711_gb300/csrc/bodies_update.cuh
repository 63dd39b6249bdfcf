// bodies_update.cuh -- device bodies of the cell-table, distortion, stop-test,
// centroid-update and split steps, shared by the per-step kernels (k_update.cu)
// and the persistent batched pass (k_batched.cu).  Internal.
#pragma once
#include "lbg_internal.cuh"

#include <math.h>

namespace lbg {
namespace {

__device__ __forceinline__ bool skip_update(const DevState *st, int train)
{
    return train && (st->finished || st->action != ACT_UPDATE);
}

// The cell sizes and offsets (k_scan_offsets_q) are computed on every pass of
// a training run, also on a pass that ends its stage: the pass trace reports
// the empty cells of every allocation.
__device__ __forceinline__ bool skip_counts(const DevState *st, int train)
{
    return train && st->finished;
}

// ---------------------------------------------------------------- mean
// Column sums of X per CTA over a contiguous row range: FP32 runs of 8 rows
// accumulated in FP64, then a fixed-order reduction.  part[b*L + l].
__device__ __forceinline__ void body_mean_part(const float *__restrict__ X, int64_t M, int L,
                                               double *__restrict__ part, DevState *st, int blk,
                                               int nblk)
{
    __shared__ double red[256];
    const int per = 256 / L;   // rows in parallel
    const int t = threadIdx.x;
    const int l = t % L, rr = t / L;
    const int64_t R = (M + nblk - 1) / nblk;
    const int64_t m0 = (int64_t)blk * R, m1 = m0 + R < M ? m0 + R : M;
    double acc = 0.0;
    bool bad = false;
    if (rr < per) {
        float run = 0.f;
        int cnt = 0;
        for (int64_t m = m0 + rr; m < m1; m += per) {
            const float v = X[m * L + l];
            bad = bad || !isfinite(v);
            run += v;
            if (++cnt == 8) {
                acc += run;
                run = 0.f;
                cnt = 0;
            }
        }
        acc += run;
    }
    if (bad) flag_error(st, ERR_NONFINITE);
    red[t] = acc;
    __syncthreads();
    if (t < L) {
        double s = 0.0;
        for (int q = 0; q < per; ++q) s += red[q * L + t];
        part[(size_t)blk * L + t] = s;
    }
}

// ---------------------------------------------------------------- hist
// CTA per chunk of R rows: cell counts of the chunk -> table[chunk][n]
// (stride n_cur) and the chunk's distortion partial -> dpart[chunk].
__device__ __forceinline__ void body_hist(const int32_t *__restrict__ assign,
                                          const float *__restrict__ e, int64_t M, int64_t R, int N,
                                          int do_hist, int32_t *__restrict__ table,
                                          double *__restrict__ dpart, DevState *st, int blk)
{
    extern __shared__ int h[];
    __shared__ double red[HIST_THREADS / 32];
    const int tid = threadIdx.x;
    const int64_t m0 = (int64_t)blk * R, m1 = m0 + R < M ? m0 + R : M;
    if (do_hist)
        for (int n = tid; n < N; n += HIST_THREADS) h[n] = 0;
    __syncthreads();
    // a thread's rows m0 + tid, + 256, ... in batches of eight (all loads in
    // flight at once); each batch is one FP32 run of eight added to the FP64 sum
    double acc = 0.0;
    bool clamped = false;
    for (int64_t base = m0 + tid; base < m1; base += 8 * HIST_THREADS) {
        int a[8];
        float ev[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t m = base + (int64_t)u * HIST_THREADS;
            const bool ok = m < m1;
            a[u] = (ok && do_hist) ? assign[m] : 0;
            ev[u] = ok ? e[m] : 0.f;
        }
        float run = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (base + (int64_t)u * HIST_THREADS >= m1) break;
            if (do_hist) {
                int c = a[u];
                if (c < 0 || c >= N) {
                    clamped = true;
                    c = c < 0 ? 0 : N - 1;
                }
                atomicAdd(&h[c], 1);
            }
            run += ev[u];
        }
        acc += run;
    }
    if (clamped) flag_error(st, ERR_INTERNAL);
    // the chunk's distortion: a fixed xor tree in each warp, then the warp sums in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();   // also: every histogram atomic done
    if (tid == 0) {
        double d = 0.0;
#pragma unroll
        for (int w = 0; w < HIST_THREADS / 32; ++w) d += red[w];
        dpart[blk] = d;
    }
    if (do_hist)
        for (int n = tid; n < N; n += HIST_THREADS) table[(size_t)blk * N + n] = h[n];
}

// ---------------------------------------------------------------- control
// D = sum of the chunk partials in chunk order.  In MODE_TRAIN also the
// stop test of Sec. 2.2 with the readings of the library: the stage ends if
// D == 0 or (D_prev - D)/D <= theta, or when it has run max_passes passes.
__device__ __forceinline__ void body_ctl(const double *__restrict__ dpart, int CH, DevState *st,
                                         int mode, double theta, int max_passes, int N_target,
                                         PassRecord *rec, int max_rec)
{
    if (threadIdx.x >= 32) return;
    if (mode == MODE_TRAIN && st->finished) return;
    // lane partials over chunks lane, lane + 32, ... (all loads in flight, then added
    // in that order), then a fixed shuffle tree
    constexpr int PER = (HIST_CHUNKS_MAX + 31) / 32;
    double pv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int c = (int)threadIdx.x + 32 * u;
        pv[u] = c < CH ? dpart[c] : 0.0;
    }
    double D = 0.0;
#pragma unroll
    for (int u = 0; u < PER; ++u)
        if ((int)threadIdx.x + 32 * u < CH) D += pv[u];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) D += __shfl_xor_sync(0xffffffffu, D, o);
    if (threadIdx.x != 0) return;
    const int nflag = st->nflag;
    st->n_exact_last = nflag;
    st->nflag = 0;
    st->D = D;
    if (mode != MODE_TRAIN) {
        st->action = ACT_UPDATE;
        return;
    }
    bool done = (D == 0.0) || ((st->D_prev - D) / D <= theta);
    if (!done && st->pass + 1 >= max_passes) {
        done = true;
        st->warn = 1;
    }
    const int act = !done ? ACT_UPDATE : (st->n_cur >= N_target ? ACT_FINISH : ACT_SPLIT);
    if (rec && st->total < max_rec) {
        PassRecord r;
        r.stage_n = st->n_cur;
        r.pass = st->pass;
        r.action = act;
        r.n_exact = nflag;
        r.D = D;
        r.n_empty = -1;   // filled in at the end of a traced pass
        r.ms = 0.f;
        rec[st->total] = r;
    }
    st->total += 1;
    st->action = act;
    if (act == ACT_UPDATE) {
        st->D_prev = D;
        st->pass += 1;
    }
}

// ---------------------------------------------------------------- scan
// CTA of 32 WARPS threads per 32 cells: lane = cell, warp w covers a range of
// chunks.  table[c][n] becomes the exclusive prefix over c; counts[n] = total.
template <int WARPS = 32>
__device__ __forceinline__ void body_scan(int32_t *__restrict__ table, int CH, int N,
                                          int32_t *__restrict__ counts, int blk)
{
    if (blk * 32 >= N) return;
    // a warp's chunk counts are loaded at once and kept in registers (CH <= HIST_CHUNKS_MAX)
    constexpr int MAXPER = (HIST_CHUNKS_MAX + WARPS - 1) / WARPS;
    __shared__ int part[WARPS][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = blk * 32 + lane;
    const int per = (CH + WARPS - 1) / WARPS;
    const int c0 = w * per, c1 = c0 + per < CH ? c0 + per : CH;
    int v[MAXPER];
#pragma unroll
    for (int u = 0; u < MAXPER; ++u) v[u] = (c0 + u < c1 && n < N) ? table[(size_t)(c0 + u) * N + n] : 0;
    int s = 0;
#pragma unroll
    for (int u = 0; u < MAXPER; ++u) s += v[u];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0) {
        int run = 0;
        for (int q = 0; q < WARPS; ++q) {
            const int v = part[q][lane];
            part[q][lane] = run;
            run += v;
        }
        if (n < N) counts[n] = run;
    }
    __syncthreads();
    int run = part[w][lane];
#pragma unroll
    for (int u = 0; u < MAXPER; ++u)
        if (c0 + u < c1 && n < N) {
            table[(size_t)(c0 + u) * N + n] = run;
            run += v[u];
        }
}

// One CTA of NT threads: off[n] = sum_{n' < n} counts[n'], off[N] = total.
// Thread t takes the cells [t per, (t + 1) per); with per <= OFF_REG their
// counts stay in registers (all loads in flight).  `cell(n, a, b)` is then
// called for each of the thread's cells with its rows [a, b) = [off[n], off[n+1]).
constexpr int OFF_REG = 8;
struct NoCell {
    __device__ void operator()(int, int64_t, int64_t) const {}
};
template <int NT = 1024, class Cell = NoCell>
__device__ __forceinline__ void body_offsets(const int32_t *__restrict__ counts, int N,
                                             int32_t *__restrict__ off, Cell cell = Cell())
{
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (N + NT - 1) / NT;
    const int a = t * per, b = a + per < N ? a + per : N;
    const bool in_reg = per <= OFF_REG;
    int cv[OFF_REG];
    int loc = 0;
    if (in_reg) {
#pragma unroll
        for (int u = 0; u < OFF_REG; ++u) cv[u] = a + u < b ? counts[a + u] : 0;
#pragma unroll
        for (int u = 0; u < OFF_REG; ++u) loc += cv[u];
    } else {
        for (int i = a; i < b; ++i) loc += counts[i];
    }
    int inc = loc;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int v = lane < NT / 32 ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int run = inc - loc + (w > 0 ? wsum[w - 1] : 0);
    if (in_reg) {
#pragma unroll
        for (int u = 0; u < OFF_REG; ++u)
            if (a + u < b) {
                off[a + u] = run;
                cell(a + u, run, run + cv[u]);
                run += cv[u];
            }
    } else {
        for (int i = a; i < b; ++i) {
            const int c = counts[i];
            off[i] = run;
            cell(i, run, run + c);
            run += c;
        }
    }
    if (t == NT - 1) off[N] = run;
}

// ---------------------------------------------------------------- fused (step forms)
// The last CTA to finish (a counter in the state; __threadfence before it, so
// that every CTA's partials are visible to it) runs the second kernel's body
// and resets the counter.
__device__ __forceinline__ bool last_cta(DevState *st)
{
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&st->done_ctr, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    return true;
}

// ---------------------------------------------------------------- scatter
// CTA per chunk (same chunks as k_hist).  Rows are taken in rounds of 256 in
// index order; inside a round a row's slot is
//   run[cell] + (rows of that cell in lower warps of the round) + (rank among
//   equal cells in its warp, __match_any_sync),
// which is the stable counting-sort position.  run[] starts at the cell
// offset plus the chunk's exclusive prefix.  Integer atomics only.
__device__ __forceinline__ void body_scatter(const int32_t *__restrict__ assign, int64_t M,
                                             int64_t R, const int32_t *__restrict__ table,
                                             const int32_t *__restrict__ off, int N,
                                             int32_t *__restrict__ perm, int blk)
{
    extern __shared__ int sm[];
    int *run = sm;                                                   // [N]
    unsigned char *wcnt = reinterpret_cast<unsigned char *>(sm + N);  // [8][N]
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blk * R, m1 = m0 + R < M ? m0 + R : M;
    // run[] in rounds of eight cells per thread, every load of a round in flight
    for (int n0 = tid; n0 < N; n0 += 8 * 256) {
        int o[8], c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int n = n0 + 256 * u;
            o[u] = n < N ? off[n] : 0;
            c[u] = n < N ? table[(size_t)blk * N + n] : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (n0 + 256 * u < N) run[n0 + 256 * u] = o[u] + c[u];
    }
    for (int i = tid; i < 2 * N; i += 256) reinterpret_cast<int *>(wcnt)[i] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int a_next = (m0 + tid < m1) ? assign[m0 + tid] : 0;   // the next round's cell, loaded ahead
    for (int64_t base = m0; base < m1; base += 256) {
        const int64_t m = base + tid;
        const bool valid = m < m1;
        int a = valid ? a_next : -1 - w;
        a_next = (m + 256 < m1) ? assign[m + 256] : 0;
        if (valid && (a < 0 || a >= N)) a = a < 0 ? 0 : N - 1;   // same clamp as k_hist
        const unsigned peers = __match_any_sync(0xffffffffu, a);
        const int rank = __popc(peers & lt);
        const bool leader = (peers & lt) == 0u;
        const int cnt = __popc(peers);
        if (valid && leader) wcnt[w * N + a] = (unsigned char)cnt;
        __syncthreads();
        if (valid) {
            int pre = 0;
            for (int q = 0; q < w; ++q) pre += wcnt[q * N + a];
            perm[run[a] + pre + rank] = (int32_t)m;
        }
        __syncthreads();
        if (valid && leader) {
            atomicAdd(&run[a], cnt);
            wcnt[w * N + a] = 0;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- cellsum
__device__ __forceinline__ int first_cell(const int32_t *off, int N, int64_t p)
{
    // largest n with off[n] <= p (then off[n + 1] > p because off[N] = M > p)
    int lo = 0, hi = N - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= p)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void add4(float4 &a, const float4 &b)
{
    a.x += b.x;
    a.y += b.y;
    a.z += b.z;
    a.w += b.w;
}

// Warp q sums perm[q*S, (q+1)*S) cell piece by cell piece; G lanes cover a
// row with float4 loads (L = 4G), 32/G rows per step, four steps in flight.
// Piece (cell n, warp q) -> pieces[(n + q) * L ...] (unique slot per piece).
// acc += the rows pp, pp + RPG, ... < pe (RPG = 32 / G; row r = perm[.] of X,
// this lane's float4 qd), in that order: batches of B rows in flight per lane,
// the next batch's perm entries loaded while the current rows are in flight,
// and the last (fewer than B) rows in one predicated batch.
template <int G, int B = 8>
__device__ __forceinline__ void sum_rows_v4(const float4 *__restrict__ X4, const int32_t *__restrict__ perm,
                                            int64_t pp, int64_t pe, int qd, float4 &acc)
{
    constexpr int RPG = 32 / G;
    if (pp + (B - 1) * RPG < pe) {
        int r[B];
#pragma unroll
        for (int u = 0; u < B; ++u) r[u] = perm[pp + u * RPG];
        for (;;) {
            float4 v[B];
#pragma unroll
            for (int u = 0; u < B; ++u) v[u] = __ldg(X4 + (int64_t)r[u] * G + qd);
            pp += B * RPG;
            const bool more = pp + (B - 1) * RPG < pe;
            if (more)
#pragma unroll
                for (int u = 0; u < B; ++u) r[u] = perm[pp + u * RPG];
#pragma unroll
            for (int u = 0; u < B; ++u) add4(acc, v[u]);
            if (!more) break;
        }
    }
    if (pp < pe) {
        int r[B];
#pragma unroll
        for (int u = 0; u < B; ++u) r[u] = pp + u * RPG < pe ? perm[pp + u * RPG] : -1;
        float4 v[B];
#pragma unroll
        for (int u = 0; u < B; ++u)
            v[u] = r[u] >= 0 ? __ldg(X4 + (int64_t)r[u] * G + qd) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < B; ++u)
            if (r[u] >= 0) add4(acc, v[u]);
    }
}

template <int G>
__device__ __forceinline__ void body_cellsum_v4(const float *__restrict__ X, int64_t M,
                                                const int32_t *__restrict__ perm,
                                                const int32_t *__restrict__ off, int N, int64_t S,
                                                float *__restrict__ pieces, int blk, int64_t qw = -1)
{
    constexpr int L = 4 * G;
    const int64_t q = qw >= 0 ? qw : (int64_t)blk * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t p0 = q * S;
    if (p0 >= M) return;
    const int64_t p1 = p0 + S < M ? p0 + S : M;
    const int rs = lane / G, qd = lane % G;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    int n = first_cell(off, N, p0);
    int64_t p = p0;
    while (p < p1) {
        const int64_t pe = (int64_t)off[n + 1] < p1 ? (int64_t)off[n + 1] : p1;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        sum_rows_v4<G>(X4, perm, p + rs, pe, qd, acc);
#pragma unroll
        for (int o = G; o < 32; o <<= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
            acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
        }
        if (rs == 0) reinterpret_cast<float4 *>(pieces + (size_t)(n + q) * L)[qd] = acc;
        p = pe;
        while (n + 1 < N && off[n + 1] <= p) ++n;
    }
}

// Any L: lanes own dims l = lane, lane + 32, ...; rows in order.
__device__ __forceinline__ void body_cellsum_any(const float *__restrict__ X, int64_t M, int L,
                                                 const int32_t *__restrict__ perm,
                                                 const int32_t *__restrict__ off, int N, int64_t S,
                                                 float *__restrict__ pieces, int blk, int64_t qw = -1)
{
    const int64_t q = qw >= 0 ? qw : (int64_t)blk * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t p0 = q * S;
    if (p0 >= M) return;
    const int64_t p1 = p0 + S < M ? p0 + S : M;
    int n = first_cell(off, N, p0);
    int64_t p = p0;
    while (p < p1) {
        const int64_t pe = (int64_t)off[n + 1] < p1 ? (int64_t)off[n + 1] : p1;
        float acc[LMAX / 32] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t pp = p; pp < pe; ++pp) {
            const int64_t r = perm[pp];
#pragma unroll
            for (int k = 0; k < LMAX / 32; ++k) {
                const int l = lane + 32 * k;
                if (l < L) acc[k] += __ldg(X + r * L + l);
            }
        }
#pragma unroll
        for (int k = 0; k < LMAX / 32; ++k) {
            const int l = lane + 32 * k;
            if (l < L) pieces[(size_t)(n + q) * L + l] = acc[k];
        }
        p = pe;
        while (n + 1 < N && off[n + 1] <= p) ++n;
    }
}

// Combining a cell's pieces (FP32 sums of up to S rows each, pieces q0 .. q1 of
// cell n in slots n + q0 .. n + q1).  A cell of at most COMBINE_GROUP pieces:
// the FP64 sum of its pieces in order.  A larger cell (small codebooks: up to
// M / S pieces in one cell) is combined in two levels so that no warp sums
// thousands of pieces alone: group k = pieces q0 + CG k .. q0 + CG k + CG - 1
// is summed in order in FP64 and kept as hi = fl32(s), lo = fl32(s - hi)
// (exact for the sums of integer pixel rows, and within 2^-48 of s
// otherwise) in the group's first two piece slots; the cell is the FP64 sum,
// in group order, of hi then lo of each group.  The same arithmetic runs in
// the fused form (the warp completing a group or the cell does the sums) and
// in body_combine (one thread per value), so both give the same bits.
constexpr int COMBINE_GROUP = 32;

__device__ __forceinline__ int64_t combine_groups(int64_t q0, int64_t q1)
{
    return q1 - q0 < COMBINE_GROUP ? 1 : (q1 - q0) / COMBINE_GROUP + 1;
}

// FP64 sum of pieces [ga, gb] of cell n, component l, in order.
__device__ __forceinline__ double sum_pieces(const float *__restrict__ pieces, int n, int64_t ga, int64_t gb,
                                             int L, int l)
{
    double s = 0.0;
    int64_t q = ga;
    for (; q + 7 <= gb; q += 8) {   // eight loads in flight, added in order
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(pieces + (size_t)(n + q + u) * L + l);
#pragma unroll
        for (int u = 0; u < 8; ++u) s += (double)v[u];
    }
    for (; q <= gb; ++q) s += (double)__ldcg(pieces + (size_t)(n + q) * L + l);
    return s;
}

// Component l of the centroid of a cell (pieces q0 .. q1, count b - a).  With
// more than one group, each group's (hi, lo) are in its first two slots (a
// one-piece group: its piece, lo = 0).
__device__ __forceinline__ float cell_value(const float *__restrict__ pieces, int n, int64_t q0, int64_t q1,
                                            int64_t count, int L, int l)
{
    double s;
    if (q1 - q0 < COMBINE_GROUP) {
        s = sum_pieces(pieces, n, q0, q1, L, l);
    } else {
        s = 0.0;
        for (int64_t g = q0; g <= q1; g += COMBINE_GROUP) {
            s += (double)__ldcg(pieces + (size_t)(n + g) * L + l);
            if (g < q1) s += (double)__ldcg(pieces + (size_t)(n + g + 1) * L + l);
        }
    }
    // FP32 division of the rounded sum (two roundings, ~1.2e-7 relative; FP64
    // division is slow on this part)
    return (float)s / (float)count;
}

// c_n = (FP64 sum of its pieces, in the order and levels of piece_done) /
// count_n, one thread per value; an empty cell copies C_in (may alias C_out).
__device__ __forceinline__ void body_combine(const float *__restrict__ pieces,
                                             const int32_t *__restrict__ off, int N, int L, int64_t S,
                                             const float *C_in, float *C_out, int blk)
{
    const int64_t i = (int64_t)blk * blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * L) return;
    const int n = (int)(i / L), l = (int)(i - (int64_t)n * L);
    const int64_t a = off[n], b = off[n + 1];
    if (b == a) {
        C_out[i] = C_in[i];
        return;
    }
    const int64_t q0 = a / S, q1 = (b - 1) / S;
    double s = 0.0;
    if (q1 - q0 < COMBINE_GROUP) {
        s = sum_pieces(pieces, n, q0, q1, L, l);
    } else {   // the two levels of piece_done, with (hi, lo) of each group in registers
        for (int64_t g = q0; g <= q1; g += COMBINE_GROUP) {
            const int64_t g1 = g + COMBINE_GROUP - 1 < q1 ? g + COMBINE_GROUP - 1 : q1;
            if (g1 == g) {
                s += (double)__ldcg(pieces + (size_t)(n + g) * L + l);
            } else {
                const double sg = sum_pieces(pieces, n, g, g1, L, l);
                const float hi = (float)sg;
                s += (double)hi;
                s += (double)(float)(sg - (double)hi);
            }
        }
    }
    // FP32 division of the rounded sum (two roundings, ~1.2e-7 relative; FP64
    // division is slow on this part)
    C_out[i] = (float)s / (float)(b - a);
}

// ---------------------------------------------------------------- split
// [c + delta], [c - delta] per centroid (or c (1 + delta), c (1 - delta) when
// mult), interleaved, rounded once from FP64.
__device__ __forceinline__ void body_split(const float *__restrict__ C_cur, float *__restrict__ C_alt,
                                           int L, double delta, int mult, DevState *st, int blk)
{
    if (st->finished || st->action != ACT_SPLIT) return;
    const int n = st->n_cur;
    const int64_t i = (int64_t)blk * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * L) return;
    const int64_t c = i / L, l = i - c * L;
    const double v = (double)C_cur[i];
    C_alt[(2 * c) * L + l] = (float)(mult ? v * (1.0 + delta) : v + delta);
    C_alt[(2 * c + 1) * L + l] = (float)(mult ? v * (1.0 - delta) : v - delta);
}

// n_cur: the stage size before the split (the state's, unless the caller holds
// it from before a concurrent stage advance).
__device__ __forceinline__ void body_copy_split(const float *__restrict__ C_alt,
                                                float *__restrict__ C_cur, int L, DevState *st,
                                                int blk, int n_cur = -1)
{
    if (st->finished || st->action != ACT_SPLIT) return;
    const int64_t n = n_cur >= 0 ? n_cur : st->n_cur;
    const int64_t i = (int64_t)blk * blockDim.x + threadIdx.x;
    if (i < 2 * n * L) C_cur[i] = C_alt[i];
}

// End of a training pass: a split doubles the stage size and resets the
// stage (D_prev = +inf, reading of the library); a finish ends training.
__device__ __forceinline__ void body_stage(DevState *st)
{
    if (threadIdx.x != 0 || st->finished) return;
    if (st->action == ACT_SPLIT) {
        st->n_cur *= 2;
        st->pass = 0;
        st->D_prev = INFINITY;
    } else if (st->action == ACT_FINISH) {
        st->finished = 1;
    }
}

// The warp that has stored piece q of cell n (rows [a, b)): counts it; the
// warp completing a group stores the group's (hi, lo), and the warp completing
// the cell writes its centroid.  cell_done[0 .. N) counts finished pieces (a
// cell of one group) or finished groups per cell, gdone = cell_done + N counts finished pieces per group (indexed by the
// slot of the group's first piece); each counter is reset by the warp that
// completes it.
__device__ __forceinline__ void piece_done(float *__restrict__ pieces, int32_t *__restrict__ cell_done, int N,
                                           int n, int64_t q, int64_t a, int64_t b, int64_t S, int L,
                                           float *__restrict__ C_out, int lane)
{
    const int64_t q0 = a / S, q1 = (b - 1) / S;
    const int64_t ng = combine_groups(q0, q1);
    __threadfence();
    __syncwarp();
    if (ng > 1) {
        int32_t *gdone = cell_done + N;
        const int64_t g0 = q0 + (q - q0) / COMBINE_GROUP * COMBINE_GROUP;
        const int64_t g1 = g0 + COMBINE_GROUP - 1 < q1 ? g0 + COMBINE_GROUP - 1 : q1;
        int last = 0;
        if (lane == 0) last = atomicAdd(&gdone[n + g0], 1) == (int)(g1 - g0);
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) return;
        __threadfence();
        if (g1 > g0)
            for (int l = lane; l < L; l += 32) {
                const double sg = sum_pieces(pieces, n, g0, g1, L, l);
                const float hi = (float)sg;
                pieces[(size_t)(n + g0) * L + l] = hi;
                pieces[(size_t)(n + g0 + 1) * L + l] = (float)(sg - (double)hi);
            }
        if (lane == 0) gdone[n + g0] = 0;
        __threadfence();
        __syncwarp();
    }
    // the cell counter counts pieces (one group) or completed groups
    const int expect = ng > 1 ? (int)(ng - 1) : (int)(q1 - q0);
    int last = 0;
    if (lane == 0) last = atomicAdd(&cell_done[n], 1) == expect;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    for (int l = lane; l < L; l += 32) C_out[(int64_t)n * L + l] = cell_value(pieces, n, q0, q1, b - a, L, l);
    if (lane == 0) cell_done[n] = 0;
}

// End of the warp's piece of cell n (rows [a, b), L = 4 G, lanes (rs, qd) hold
// the reduced sums in rs == 0): a cell that lies in this one piece gets its
// centroid at once; else the piece is stored and piece_done combines.
template <int G>
__device__ __forceinline__ void finish_piece_v4(float4 acc, int n, int64_t q, int64_t a, int64_t b, int64_t S,
                                                float *__restrict__ pieces, int32_t *__restrict__ cell_done, int N,
                                                float *__restrict__ C_out, int lane)
{
    constexpr int L = 4 * G;
    const int rs = lane / G, qd = lane % G;
    const int64_t q0 = a / S, q1 = (b - 1) / S;
    if (q0 == q1) {
        if (rs == 0) {
            const float cnt = (float)(b - a);
            reinterpret_cast<float4 *>(C_out + (size_t)n * L)[qd] =
                make_float4(acc.x / cnt, acc.y / cnt, acc.z / cnt, acc.w / cnt);
        }
        return;
    }
    if (rs == 0) reinterpret_cast<float4 *>(pieces + (size_t)(n + q) * L)[qd] = acc;
    piece_done(pieces, cell_done, N, n, q, a, b, S, L, C_out, lane);
}

// Warp q sums perm[q S, (q + 1) S) cell piece by cell piece, as
// body_cellsum_v4 (same order, same bits), starting from qcell[q] instead of a
// search of the offsets, and finishes every piece with finish_piece_v4.
template <int G>
__device__ __forceinline__ void body_cellsum_c(const float *__restrict__ X, int64_t M,
                                               const int32_t *__restrict__ perm,
                                               const int32_t *__restrict__ off,
                                               const int32_t *__restrict__ qcell, int N, int64_t S,
                                               float *__restrict__ pieces, int32_t *__restrict__ cell_done,
                                               float *__restrict__ C_out, int64_t q)
{
    const int lane = threadIdx.x & 31;
    const int64_t p0 = q * S;
    if (p0 >= M) return;
    const int64_t p1 = p0 + S < M ? p0 + S : M;
    const int rs = lane / G, qd = lane % G;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    int n = qcell[q];
    int64_t p = p0;
    while (p < p1) {
        const int64_t a = off[n], b = off[n + 1];
        const int64_t pe = b < p1 ? b : p1;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        sum_rows_v4<G>(X4, perm, p + rs, pe, qd, acc);
#pragma unroll
        for (int o = G; o < 32; o <<= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
            acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
        }
        finish_piece_v4<G>(acc, n, q, a, b, S, pieces, cell_done, N, C_out, lane);
        p = pe;
        while (n + 1 < N && off[n + 1] <= p) ++n;
    }
}

// Per cell, given its rows [a, b) after the offsets (the `cell` step of
// body_offsets): the cell's piece counters zeroed and, when `copy`, an empty
// cell's codevector copied from C_in to C_out.  (The cell of each piece is
// found afterwards by all threads at once: one thread per large cell writing
// thousands of entries was the longest step of a pass at small N.)
struct PieceCells {
    int N;
    int64_t S;
    int L;
    int32_t *cell_done;
    bool copy;
    const float *C_in;
    float *C_out;
    __device__ __forceinline__ void operator()(int n, int64_t a, int64_t b) const
    {
        cell_done[n] = 0;
        if (b == a) {
            if (copy)
                for (int l = 0; l < L; ++l) C_out[(int64_t)n * L + l] = C_in[(int64_t)n * L + l];
            return;
        }
        const int64_t q0 = a / S, q1 = (b - 1) / S;   // group counters of a large cell
        if (combine_groups(q0, q1) > 1)
            for (int64_t g = q0; g <= q1; g += COMBINE_GROUP) cell_done[N + n + g] = 0;
    }
};

// Any L: the cell sums of body_cellsum_any (lanes own dims l = lane, lane + 32,
// ...; rows in order) with the pieces finished as in finish_piece_v4.
__device__ __forceinline__ void body_cellsum_c_any(const float *__restrict__ X, int64_t M, int L,
                                                   const int32_t *__restrict__ perm,
                                                   const int32_t *__restrict__ off,
                                                   const int32_t *__restrict__ qcell, int N, int64_t S,
                                                   float *__restrict__ pieces, int32_t *__restrict__ cell_done,
                                                   float *__restrict__ C_out, int64_t q)
{
    const int lane = threadIdx.x & 31;
    const int64_t p0 = q * S;
    if (p0 >= M) return;
    const int64_t p1 = p0 + S < M ? p0 + S : M;
    int n = qcell[q];
    int64_t p = p0;
    while (p < p1) {
        const int64_t a = off[n], b = off[n + 1];
        const int64_t pe = b < p1 ? b : p1;
        float acc[LMAX / 32] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t pp = p; pp < pe; ++pp) {
            const int64_t r = perm[pp];
#pragma unroll
            for (int k = 0; k < LMAX / 32; ++k) {
                const int l = lane + 32 * k;
                if (l < L) acc[k] += __ldg(X + r * L + l);
            }
        }
        const int64_t q0 = a / S, q1 = (b - 1) / S;
        if (q0 == q1) {
            const float cnt = (float)(b - a);
#pragma unroll
            for (int k = 0; k < LMAX / 32; ++k) {
                const int l = lane + 32 * k;
                if (l < L) C_out[(int64_t)n * L + l] = acc[k] / cnt;
            }
        } else {
#pragma unroll
            for (int k = 0; k < LMAX / 32; ++k) {
                const int l = lane + 32 * k;
                if (l < L) pieces[(size_t)(n + q) * L + l] = acc[k];
            }
            piece_done(pieces, cell_done, N, n, q, a, b, S, L, C_out, lane);
        }
        p = pe;
        while (n + 1 < N && off[n + 1] <= p) ++n;
    }
}

}  // namespace
}  // namespace lbg
