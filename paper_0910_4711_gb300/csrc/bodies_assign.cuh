// bodies_assign.cuh -- device bodies of the FP32 nearest-codevector search
// (codebook preparation, the certified tile search, the exact re-scoring of a
// group of flagged rows), shared by the per-step kernels (k_assign.cu) and the
// persistent batched pass (k_batched.cu).  Internal; the certificate is proved
// in the header of k_assign.cu.
#pragma once
#include "lbg_internal.cuh"

#include <math.h>

namespace lbg {
namespace {

constexpr float U32 = 5.9604644775390625e-8f;   // 2^-24
constexpr float SLOP = 1.0000305175781250f;     // 1 + 2^-15, covers FP32 evaluation of bounds
constexpr int EX_R = 8;                         // flagged rows per CTA group in k_assign_exact
constexpr int EX_SW = EXACT_SW;                 // codevectors per staged chunk
constexpr int EX_THREADS = 256;

// Prepared codebook, chunk-major: chunk k holds (Lp + 1) x BN floats; row 0
// is the chain start s0_n = fl(||c~_n||^2 - k_n) (+inf for padding), rows
// 1..Lp are -2 c~_{n,l} (0 for l >= L or padding).  Also writes k_n, the
// original codebook in chunks of EX_SW codevectors, k-major inside a chunk
// (CT[(n / EX_SW) * Lp + l][n % EX_SW]) for the exact fallback, max ||c~_n||
// into st->cmax_bits, and flags non-finite entries.
// A CTA takes PREP_TILE codevectors: coalesced row loads into shared memory,
// FP64 norms (warp per codevector, fixed shuffle tree), coalesced transposed
// stores.
constexpr int PREP_TILE = 32;

// Shared memory of body_prep (static in its own kernels, in the phase buffer of
// the persistent batched pass).
struct PrepSmem {
    float orig[PREP_TILE][LMAX + 1];
    float cen[PREP_TILE][LMAX + 1];
    double sqs[PREP_TILE];
};

__device__ __forceinline__ void body_prep(const float *__restrict__ C, int N, int L, int Lp,
                                          const float *__restrict__ mu, float *__restrict__ Cp,
                                          float *__restrict__ kn, float *__restrict__ CT,
                                          DevState *st, int blk, PrepSmem &ps)
{
    auto &orig = ps.orig;
    auto &cen = ps.cen;
    auto &sqs = ps.sqs;
    const int npad = round_up(N, BN);
    const int n0 = blk * PREP_TILE;
    if (n0 >= npad) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    bool finite = true;
    for (int i = tid; i < PREP_TILE * L; i += 256) {
        const int j = i / L, l = i - (i / L) * L;
        const int n = n0 + j;
        float c = 0.f, v = 0.f;
        if (n < N) {
            c = C[(size_t)n * L + l];
            finite = finite && isfinite(c);
            v = c - mu[l];
        }
        orig[j][l] = c;
        cen[j][l] = v;
    }
    if (!finite) flag_error(st, ERR_NONFINITE);
    __syncthreads();
    for (int j = warp; j < PREP_TILE; j += 8) {
        double sq = 0.0;
        for (int l = lane; l < L; l += 32) {
            const double v = cen[j][l];
            sq += v * v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) sqs[j] = sq;
    }
    __syncthreads();
    if (tid < PREP_TILE) {   // warp 0: one codevector per lane
        const int n = n0 + tid;
        uint32_t cbits = 0u;
        float *blk = Cp + (size_t)(n / BN) * (Lp + 1) * BN;
        if (n < N) {
            const double sq = sqs[tid];
            const double k = 2.0 * (double)(L + 2) * 5.9604644775390625e-8 * sq;
            const float kf = __double2float_ru(k);
            blk[n % BN] = __double2float_rn(sq - (double)kf);
            kn[n] = kf;
            cbits = __float_as_uint(__fsqrt_ru(__double2float_ru(sq)));   // >= ||c~_n||
        } else if (n < npad) {
            blk[n % BN] = INFINITY;
            kn[n] = 0.f;
        }
        // max ||c~_n|| of the tile (bits of non-negative floats order as integers): one atomic per CTA
        cbits = __reduce_max_sync(0xffffffffu, cbits);
        if (tid == 0 && cbits) atomicMax(&st->cmax_bits, cbits);
    }
    for (int i = tid; i < Lp * PREP_TILE; i += 256) {
        const int l = i / PREP_TILE, j = i % PREP_TILE;
        const int n = n0 + j;
        if (n >= npad) continue;
        const bool real = n < N && l < L;
        Cp[(size_t)(n / BN) * (Lp + 1) * BN + (size_t)(1 + l) * BN + n % BN] = real ? -2.0f * cen[j][l] : 0.f;
        CT[((size_t)(n / EX_SW) * Lp + l) * EX_SW + n % EX_SW] = real ? orig[j][l] : 0.f;
    }
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// Two rows at once on the packed FP32 pipe: (da, db) += ((xa, xb) - (c, c))^2,
// each lane rounded exactly as the scalar __fsub_rn / fmaf pair would be.
__device__ __forceinline__ void sqdiff2(float xa, float xb, uint64_t cc, float &da, float &db)
{
    asm("{\n\t.reg .b64 x, d, a;\n\t"
        "mov.b64 x, {%2, %3};\n\t"
        "sub.rn.f32x2 d, x, %4;\n\t"
        "mov.b64 a, {%0, %1};\n\t"
        "fma.rn.f32x2 a, d, d, a;\n\t"
        "mov.b64 {%0, %1}, a;\n\t}"
        : "+f"(da), "+f"(db)
        : "f"(xa), "f"(xb), "l"(cc));
}

// Shared state of an assignment CTA (static shared memory of the kernel).
template <int TBM>
struct AssignSmemT {
    uint64_t bar[2];
    int abort;
    float rec_v1[2][TBM], rec_v2[2][TBM];
    int rec_id[2][TBM];
};

using AssignSmem = AssignSmemT<BM>;

// Barrier of the 2 TBM threads running one tile: the whole CTA (id 0), or a
// named barrier of a thread group (id > 0) when a CTA runs several tiles.
__device__ __forceinline__ void tile_sync(int id, int threads)
{
    if (id == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Nearest codevector of the TBM rows starting at m0 (see the file header);
// 2 TBM threads: warps are 4x8 thread grids of 8x8 (row, codevector) tiles,
// TBM / 32 warp rows x 2 warp columns.
// The two chunk barriers persist across calls of one CTA: use0/use1 count
// their completed phases.  Returns false (after reporting) if a bulk copy
// timed out; every thread of the tile returns the same value.  `expire`
// (a test hook) makes the first chunk wait give up at once, as a wait that
// ran out of time would.  The tile's threads are threadIdx.x = tbase ..
// tbase + 2 TBM - 1, synchronised by tile_sync(sync_id) (0: the whole CTA).
template <int TBM>
__device__ __forceinline__ bool assign_f32_tile_t(
    const float *__restrict__ X, int64_t M, int L, int Lp, const float *__restrict__ Cp,
    const float *__restrict__ kn, int N, const float *__restrict__ mu, const float *__restrict__ C,
    DevState *st, int32_t *__restrict__ assign, float *__restrict__ e, int32_t *__restrict__ flags,
    int64_t m0, float *smem, AssignSmemT<TBM> &sh, uint32_t &use0, uint32_t &use1, int expire = 0,
    int tbase = 0, int sync_id = 0)
{
    uint64_t *bar = sh.bar;
    auto &rec_v1 = sh.rec_v1;
    auto &rec_v2 = sh.rec_v2;
    auto &rec_id = sh.rec_id;
    const int tid = (int)threadIdx.x - tbase;
    const int nchunk = (N + BN - 1) / BN;
    const int chunk_floats = (Lp + 1) * BN;
    const uint32_t chunk_bytes = (uint32_t)chunk_floats * 4u;
    float *xs = smem;                       // [Lp][TBM]
    float *cbuf0 = xs + Lp * TBM;            // [Lp + 1][BN]
    float *cbuf1 = cbuf0 + chunk_floats;
    const uint32_t base0 = use0, base1 = use1;
    auto parity = [&](int k) -> uint32_t { return ((k & 1 ? base1 : base0) + (uint32_t)(k >> 1)) & 1u; };

    if (tid == 0) {
        for (int k = 0; k < 2 && k < nchunk; ++k) {
            mbar_expect_tx(&bar[k], chunk_bytes);
            bulk_load(k ? cbuf1 : cbuf0, Cp + (size_t)k * chunk_floats, chunk_bytes, &bar[k]);
        }
    }

    // Stage the centred x tile, transposed: xs[l][r] (zero outside M x L).
    bool bad = false;
    for (int i = tid; i < TBM * Lp; i += (2 * TBM)) {
        const int r = i % TBM, l = i / TBM;
        const int64_t m = m0 + r;
        float v = 0.f;
        if (m < M && l < L) {
            const float xv = X[m * L + l];
            bad = bad || !isfinite(xv);
            v = xv - mu[l];
        }
        xs[l * TBM + r] = v;
    }
    if (bad) flag_error(st, ERR_NONFINITE);

    const int warp = tid >> 5, lane = tid & 31;
    const int wr = warp >> 1, wc = warp & 1;
    const int ly = lane >> 3, lx = lane & 7;
    const int rA = wr * 32 + ly * 4;   // rows rA..rA+3 and rA+16..rA+19
    const int cA = wc * 64 + lx * 4;   // codevectors cA..cA+3 and cA+32..cA+35

    float v1[8], v2[8];
    int mk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        v1[i] = INFINITY;
        v2[i] = INFINITY;
        mk[i] = 0;
    }
    tile_sync(sync_id, 2 * TBM);

    int k_stop = nchunk;
    for (int k = 0; k < nchunk; ++k) {
        const int b = k & 1;
        const float *cb = b ? cbuf1 : cbuf0;
        const bool ok = (expire && k == 0) ? false : mbar_wait_bounded(&bar[b], parity(k));
        if (!ok) sh.abort = 1;
        if (ok) {
            float acc[8][8];
            {
                const float4 s0a = lds4(&cb[cA]), s0b = lds4(&cb[cA + 32]);
                const float4 xa = lds4(&xs[rA]), xb = lds4(&xs[rA + 16]);
                const float4 ca = lds4(&cb[BN + cA]), cc = lds4(&cb[BN + cA + 32]);
                const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
                const float cv[8] = {ca.x, ca.y, ca.z, ca.w, cc.x, cc.y, cc.z, cc.w};
                const float s0[8] = {s0a.x, s0a.y, s0a.z, s0a.w, s0b.x, s0b.y, s0b.z, s0b.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(xv[i], cv[j], s0[j]);
            }
#pragma unroll 4
            for (int l = 1; l < Lp; ++l) {
                const float4 xa = lds4(&xs[l * TBM + rA]), xb = lds4(&xs[l * TBM + rA + 16]);
                const float4 ca = lds4(&cb[(1 + l) * BN + cA]), cc = lds4(&cb[(1 + l) * BN + cA + 32]);
                const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
                const float cv[8] = {ca.x, ca.y, ca.z, ca.w, cc.x, cc.y, cc.z, cc.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(xv[i], cv[j], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float old = v1[i];
#pragma unroll
                for (int j = 0; j < 8; j += 2) {   // codevectors j, j + 1: a split pair (2k, 2k + 1)
                    const float a = fminf(acc[i][j], acc[i][j + 1]);
                    v2[i] = fminf(v2[i], fmaxf(v1[i], a));
                    v1[i] = fminf(v1[i], a);
                }
                mk[i] = (v1[i] < old) ? k : mk[i];
            }
        }
        tile_sync(sync_id, 2 * TBM);
        if (sh.abort) {
            k_stop = k;
            break;
        }
        if (tid == 0 && k + 2 < nchunk) {
            mbar_expect_tx(&bar[b], chunk_bytes);
            bulk_load(cbuf0 + b * chunk_floats, Cp + (size_t)(k + 2) * chunk_floats, chunk_bytes,
                      &bar[b]);
        }
    }
    if (k_stop < nchunk) {
        // A bulk copy did not land in time: wait (bounded) for the copies
        // still in flight, report, and leave the rows unwritten.
        if (tid == 0) {
            for (int kk = k_stop; kk < nchunk && kk < k_stop + 2; ++kk)
                (void)mbar_wait_bounded(&bar[kk & 1], parity(kk));
            flag_error(st, ERR_TIMEOUT);
        }
        return false;
    }
    use0 = base0 + (uint32_t)((nchunk + 1) >> 1);
    use1 = base1 + (uint32_t)(nchunk >> 1);

    // Merge the 8 lanes that share rows (lx = 0..7), then the two warps (wc).
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int id = mk[i] * 16 + wc * 8 + lx;
        float a1 = v1[i], a2 = v2[i];
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const float b1 = __shfl_xor_sync(0xffffffffu, a1, o);
            const float b2 = __shfl_xor_sync(0xffffffffu, a2, o);
            const int bid = __shfl_xor_sync(0xffffffffu, id, o);
            a2 = fminf(fminf(a2, b2), fmaxf(a1, b1));
            const bool take = (b1 < a1) || (b1 == a1 && bid < id);
            a1 = take ? b1 : a1;
            id = take ? bid : id;
        }
        if (lx == 0) {
            const int r = (i < 4) ? rA + i : rA + 12 + i;
            rec_v1[wc][r] = a1;
            rec_v2[wc][r] = a2;
            rec_id[wc][r] = id;
        }
    }
    tile_sync(sync_id, 2 * TBM);
    const int r = tid;
    const int64_t m = m0 + r;
    if (tid >= TBM || m >= M) return true;
    float V1, V2;
    int ID;
    {
        const float a1 = rec_v1[0][r], a2 = rec_v2[0][r], b1 = rec_v1[1][r], b2 = rec_v2[1][r];
        const int ia = rec_id[0][r], ib = rec_id[1][r];
        V2 = fminf(fminf(a2, b2), fmaxf(a1, b1));
        const bool take = (b1 < a1) || (b1 == a1 && ib < ia);
        V1 = take ? b1 : a1;
        ID = take ? ib : ia;
    }

    // Recover the index: recompute the winning group's 8 chains exactly.
    const int kw = ID >> 4, nl = ((ID >> 3) & 1) * 64 + (ID & 7) * 4;
    const float *blk = Cp + (size_t)kw * chunk_floats;
    float s[8];
    {
        const float4 t0 = __ldg(reinterpret_cast<const float4 *>(blk + nl));
        const float4 t1 = __ldg(reinterpret_cast<const float4 *>(blk + nl + 32));
        const float4 c0 = __ldg(reinterpret_cast<const float4 *>(blk + BN + nl));
        const float4 c1 = __ldg(reinterpret_cast<const float4 *>(blk + BN + nl + 32));
        const float x0 = xs[r];
        s[0] = fmaf(x0, c0.x, t0.x);
        s[1] = fmaf(x0, c0.y, t0.y);
        s[2] = fmaf(x0, c0.z, t0.z);
        s[3] = fmaf(x0, c0.w, t0.w);
        s[4] = fmaf(x0, c1.x, t1.x);
        s[5] = fmaf(x0, c1.y, t1.y);
        s[6] = fmaf(x0, c1.z, t1.z);
        s[7] = fmaf(x0, c1.w, t1.w);
    }
#pragma unroll 4
    for (int l = 1; l < Lp; ++l) {
        const float4 c0 = __ldg(reinterpret_cast<const float4 *>(blk + (1 + l) * BN + nl));
        const float4 c1 = __ldg(reinterpret_cast<const float4 *>(blk + (1 + l) * BN + nl + 32));
        const float x = xs[l * TBM + r];
        s[0] = fmaf(x, c0.x, s[0]);
        s[1] = fmaf(x, c0.y, s[1]);
        s[2] = fmaf(x, c0.z, s[2]);
        s[3] = fmaf(x, c0.w, s[3]);
        s[4] = fmaf(x, c1.x, s[4]);
        s[5] = fmaf(x, c1.y, s[5]);
        s[6] = fmaf(x, c1.z, s[6]);
        s[7] = fmaf(x, c1.w, s[7]);
    }
    int i1 = -1;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (i1 < 0 && s[j] == V1) i1 = kw * BN + nl + (j < 4 ? j : 28 + j);

    bool certified = false;
    const int ip = i1 ^ 1;                       // the other member of i1's pair
    const bool pair = ip < N;
    if (i1 >= 0 && i1 < N && V1 < INFINITY) {
        float xn2 = 0.f;
        for (int l = 0; l < L; ++l) xn2 = fmaf(xs[l * TBM + r], xs[l * TBM + r], xn2);
        const float xn2u = xn2 * SLOP;
        const float R = (float)(L + 2) * U32 * xn2u * SLOP;
        const float kc = pair ? fmaxf(kn[i1], kn[ip]) : kn[i1];
        const float cmax = __uint_as_float(st->cmax_bits);
        const float eta = U32 * (sqrtf(xn2u) + cmax) * SLOP;
        const float g1sq = xn2u + V1 + 2.f * kc + R + 4.f * U32 * (xn2u + fabsf(V1));
        const float g1 = sqrtf(fmaxf(g1sq, 0.f)) * SLOP;
        const float margin = (2.f * R + 2.f * kc + 4.f * eta * (g1 + eta)) * SLOP;
        certified = (V2 - V1) > margin;
    }
    int win = i1;
    float dwin = 0.f;
    if (certified) {
        // the pair's exact FP32 direct-form distances decide between its members
        // (each sum in index order; both in one loop, float4 loads when the rows allow)
        const float *xr = X + m * L;
        const float *ca = C + (size_t)i1 * L;
        const float *cb = C + (size_t)(pair ? ip : i1) * L;
        float da = 0.f, db = 0.f;
        if ((L & 3) == 0 && ((reinterpret_cast<uintptr_t>(xr) | reinterpret_cast<uintptr_t>(ca) |
                              reinterpret_cast<uintptr_t>(cb)) & 15u) == 0) {
#pragma unroll 4
            for (int q = 0; q < (L >> 2); ++q) {
                const float4 x4 = __ldg(reinterpret_cast<const float4 *>(xr) + q);
                const float4 a4 = __ldg(reinterpret_cast<const float4 *>(ca) + q);
                const float4 b4 = __ldg(reinterpret_cast<const float4 *>(cb) + q);
                float d = __fsub_rn(x4.x, a4.x);
                da = fmaf(d, d, da);
                d = __fsub_rn(x4.y, a4.y);
                da = fmaf(d, d, da);
                d = __fsub_rn(x4.z, a4.z);
                da = fmaf(d, d, da);
                d = __fsub_rn(x4.w, a4.w);
                da = fmaf(d, d, da);
                d = __fsub_rn(x4.x, b4.x);
                db = fmaf(d, d, db);
                d = __fsub_rn(x4.y, b4.y);
                db = fmaf(d, d, db);
                d = __fsub_rn(x4.z, b4.z);
                db = fmaf(d, d, db);
                d = __fsub_rn(x4.w, b4.w);
                db = fmaf(d, d, db);
            }
        } else {
            for (int l = 0; l < L; ++l) {
                const float x = xr[l];
                float d = __fsub_rn(x, ca[l]);
                da = fmaf(d, d, da);
                d = __fsub_rn(x, cb[l]);
                db = fmaf(d, d, db);
            }
        }
        dwin = da;
        if (pair) {
            // |fl(d2) - d2| <= (L + 2) u d2 for either sum (kept as (L + 4) u)
            const float tol = (float)(L + 4) * U32 * (da + db) * SLOP;
            if (db < da - tol) {
                win = ip;
                dwin = db;
            } else if (!(da < db - tol)) {
                certified = false;
            }
        }
    }
    if (certified) {
        assign[m] = win;
        e[m] = dwin;
    } else {
        flags[atomicAdd(&st->nflag, 1)] = (int32_t)m;
    }
    return true;
}

// Exact FP32 direct-form re-scoring of the rows k_assign_f32 could not
// certify: d = sum_l (x_l - c_l)^2 in index order (the same expression as a
// certified row's e), minimum with the lowest index on ties.  A CTA takes a
// group of EX_R flagged rows (k-major in shared memory) and streams the
// original codebook through two shared buffers of EX_SW codevectors (one TMA
// bulk copy each, bounded mbarrier waits); thread t scores codevector
// t % EX_SW of each chunk against rows 4 * (t / EX_SW) .. + 3.  The
// (distance, index) minimum is reduced in a fixed order (shuffles, then the
// warps of a row half in order).
struct ExactSmem {
    float xs[LMAX][EX_R];
    uint64_t bar[2];
    int abort;
    float rb[EX_THREADS / 32][4];
    int ri[EX_THREADS / 32][4];
};

// Re-scores flagged group g (EX_R rows) of one problem; uses[] count the
// completed phases of the two chunk barriers across calls of one CTA.
// Returns false after a time-out (reported); uniform across the CTA.
__device__ __forceinline__ bool exact_group(const float *__restrict__ X, int L, int Lp,
                                            const float *__restrict__ CT, int N, DevState *st,
                                            const int32_t *__restrict__ flags, int nflag,
                                            int32_t *__restrict__ assign, float *__restrict__ e,
                                            int g, float *cbuf, ExactSmem &sh, uint32_t *uses)
{
    auto &xs = sh.xs;
    uint64_t *bar = sh.bar;
    auto &rb = sh.rb;
    auto &ri = sh.ri;
    const int nchunk = (N + EX_SW - 1) / EX_SW;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int j = tid % EX_SW, half = tid / EX_SW;
    const uint32_t chunk_floats = (uint32_t)Lp * EX_SW;
    const uint32_t chunk_bytes = chunk_floats * 4u;
    {
        const int nr = min(EX_R, nflag - g * EX_R);
        for (int i = tid; i < EX_R * L; i += EX_THREADS) {
            const int r = i % EX_R, l = i / EX_R;
            xs[l][r] = r < nr ? X[(int64_t)flags[g * EX_R + r] * L + l] : 0.f;
        }
        if (tid == 0)
            for (int k = 0; k < 2 && k < nchunk; ++k) {
                mbar_expect_tx(&bar[k], chunk_bytes);
                bulk_load(cbuf + k * chunk_floats, CT + (size_t)k * chunk_floats, chunk_bytes, &bar[k]);
            }
        __syncthreads();
        float best[4];
        int bi[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            best[q] = INFINITY;
            bi[q] = 0x7fffffff;
        }
        int k_stop = nchunk;
        for (int k = 0; k < nchunk; ++k) {
            const int b = k & 1;
            const bool ok = mbar_wait_bounded(&bar[b], uses[b] & 1u);
            uses[b] += 1u;
            if (!ok) sh.abort = 1;
            const float *cb = cbuf + b * chunk_floats;
            const int n = k * EX_SW + j;
            if (ok && n < N) {
                float d2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
                for (int l = 0; l < L; ++l) {
                    const float c = cb[l * EX_SW + j];
                    const float4 x4 = lds4(&xs[l][half * 4]);
                    float d = x4.x - c;
                    d2[0] = fmaf(d, d, d2[0]);
                    d = x4.y - c;
                    d2[1] = fmaf(d, d, d2[1]);
                    d = x4.z - c;
                    d2[2] = fmaf(d, d, d2[2]);
                    d = x4.w - c;
                    d2[3] = fmaf(d, d, d2[3]);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (d2[q] < best[q]) {
                        best[q] = d2[q];
                        bi[q] = n;
                    }
            }
            __syncthreads();
            if (sh.abort) {
                k_stop = k;
                break;
            }
            if (tid == 0 && k + 2 < nchunk) {
                mbar_expect_tx(&bar[b], chunk_bytes);
                bulk_load(cbuf + b * chunk_floats, CT + (size_t)(k + 2) * chunk_floats, chunk_bytes,
                          &bar[b]);
            }
        }
        if (k_stop < nchunk) {
            if (tid == 0) {
                for (int kk = k_stop + 1; kk < nchunk && kk < k_stop + 2; ++kk)
                    (void)mbar_wait_bounded(&bar[kk & 1], uses[kk & 1] & 1u);
                flag_error(st, ERR_TIMEOUT);
            }
            return false;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
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
                rb[warp][q] = best[q];
                ri[warp][q] = bi[q];
            }
        }
        __syncthreads();
        if (tid < nr) {
            const int hw = (tid / 4) * (EX_SW / 32), q = tid % 4;   // first warp of the row's half
            float bb = rb[hw][q];
            int ii = ri[hw][q];
            for (int w = hw + 1; w < hw + EX_SW / 32; ++w)
                if (rb[w][q] < bb || (rb[w][q] == bb && ri[w][q] < ii)) {
                    bb = rb[w][q];
                    ii = ri[w][q];
                }
            const int row = flags[g * EX_R + tid];
            const bool valid = ii >= 0 && ii < N;
            if (!valid) flag_error(st, ERR_NONFINITE);   // only NaN rows compare false everywhere
            assign[row] = valid ? ii : 0;
            e[row] = valid ? bb : 0.f;
        }
        __syncthreads();
    }
    return true;
}

__device__ __forceinline__ void exact_init(ExactSmem &sh)
{
    if (threadIdx.x == 0) {
        mbar_init(&sh.bar[0], 1);
        mbar_init(&sh.bar[1], 1);
        fence_mbar_init();
        sh.abort = 0;
    }
    __syncthreads();
}

}  // namespace
}  // namespace lbg
