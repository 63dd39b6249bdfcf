// k_assign_tc.cu -- cell allocation (nearest codevector) on the 5th-generation
// tensor cores: BF16 operands, FP32 accumulation in tensor memory.
//
// Paper: Algorithm 1 "Cell Allocation" / Sec. 2.2 step 1, as in k_assign.cu;
// this is the same search with the cross term on tcgen05.mma.
//
// Operands.  With an integer centring vector mu, centred 8-bit image vectors
// x~ = x - mu are integers in [-255, 255], exact in BF16.  The scaled
// codevector c' = -2 c~ (FP32) is split into two BF16 pieces p_hi + p_mid with
// an FP32-exact remainder r = c' - p_hi - p_mid (|r| <= 2^-16 |c'|); the chain
// start s0 = fl(||c~||^2 - k') and the row constant X2 = fl(||x~||^2) are split
// exactly into three pieces each.  One GEMM
//     A = [ x~ | 1 1 1 X2_hi X2_mid X2_lo 0 ... ]      (K = Lk + 16)
//     B = [ p_hi | p_mid | s0 pieces 1 1 1 0 ... ]     (x~ reused twice)
// therefore accumulates X2 + s0 + x~.c' - x~.r = X2 + f - k' - x~.r (~ d - k',
// the distance up to k'), with |x~.r_n| <= ||x~|| rho, rho = max_n ||r_n||
// (measured by the preparation kernel), besides the tensor core's FP32
// accumulation error.  X2 is the same in every column of a row, so it cancels
// in V2 - V1.  (A third piece would make x~.c' exact at 3/2 the MMAs and
// codebook bytes; on the image workloads the remainder term certifies all
// but a few tenths of a percent of the rows.)
// Real-valued data (Lk <= 32, the split form): x~ = fl(x - mu) is cut into
// x_hi = bf16(x~) and x_lo = bf16(x~ - x_hi) with an FP32 remainder rem
// (|rem| <= 2^-16 |x~|); A = [ x_hi | x_lo | norm block ], and a row tile with
// any x_lo != 0 adds the Lk/16 MMAs x_lo . p_hi per job.  The pieces miss
// x_hi . r_n, x_lo . (p_mid + r_n) and rem . c'_n, all within
// ||x~|| (rho + 2^-14 cmax)(1 + 2^-7); X2 of such a tile is sum (x_hi + x_lo)^2,
// within 2^-14 ||x~||^2 of ||x~||^2.  Both go into E and the X2 term of the
// certificates below; the centring error of fl(x - mu) is the eta term.  With
// Lk = 48 or 64 a tile whose x~ is not exact in BF16 sends its rows to the
// exact fallback.
// Accumulation model.  Measured on GB300 (BF16 products, K up to 256, mixed
// exponents) the error stayed below (K/16) * 2^-24 * (sum of |products|); the
// library assumes tau = (K/16 + 2) * 2^-22 * (1 + 2^-7) of (sum of |products| +
// |s0| + X2), a factor of about 4.8 above the worst case measured.  With
// sum |x~_l c'_l| <= ||x~||^2 + ||c~||^2 this gives
//     |v_n - (X2 + f_n - k'_n)| <= tau (2 ||x~||^2 + 2 ||c~_n||^2) + u ||c~_n||^2 + E,
// E = ||x~|| rho, and with k'_n = (2 tau + 2^-23) ||c~_n||^2, R' = 2 tau ||x~||^2
// the certificate of k_assign.cu applies, over groups: the columns are taken
// in groups of G = 2, 4 or 8 consecutive codevectors, V1 is the smallest value
// and V2 the smallest value outside V1's group.  The group's member with the
// smallest FP32 direct-form distance is the candidate ii (it must beat every
// other member by more than the direct form's rounding bound, else the row is
// not certified).  The member j that produced V1 has ||x~ - c~_j||^2 <= V1 +
// 2k'_j + R' + E (+ epilogue and X2 terms) and ii is not farther than j, while
// every codevector outside the group has ||x~ - c~_n||^2 >= V2 - R' - E, so
// V2 - V1 > 2R' + 2k'_grp + 2E + 4 eta (g1 + eta) + 2^(JBITS-23) (|V1| + |V2|),
// with k'_grp the group's largest k' and the last term for the epilogue's index
// packing, proves ii the exact argmin.  A second certificate needs no bound
// on V1's member.  With X2 + f_n = ||x~ - c~_n||^2 + (X2 - ||x~||^2) and
// k'_n >= 2 tau ||c~_n||^2 + u ||c~_n||^2, the bound gives
//     ||x~ - c~_n||^2 >= v_n - R' - E - |X2 - ||x~||^2|,
// and every codevector outside the best group has v_n >= V2, so
// ||x - c_n||^2 >= (sqrt(V2 - R' - E - P - (L+2) u ||x~||^2) - eta)^2, P the
// packing term.  The winner's FP32 direct-form distance d gives ||x - c_ii||^2
// <= d (1 + (L+4) u); when the lower bound exceeds that, ii is the exact
// argmin.  A row is certified when either certificate holds.  The two
// children of a split (2i, 2i + 1) share a group, so right after a split a
// row's nearest pair of twins is resolved by their exact distances and V2
// comes from the next parent, not from the twin.
//
// Epilogue.  Each thread owns one row and one half (72 columns) of every
// tile, taken as 72/G groups of G columns.  The group minimum (three-input
// mins) gets the in-half group index (JBITS = 6, 5, 4 bits for G = 2, 4, 8)
// in its low mantissa bits (one LOP3; the value moves by less than
// 2^(JBITS-23) of it); two groups at a time then enter the running top-2 of
// group minima (five ALU operations for the two): 2.25, 1.375 and 0.94 ALU
// operations per value; a per-tile compare records the tile, and the two
// halves of a row are merged through shared memory at the end.  The tail
// scores the best group's G members exactly (G/2 per half) and a certified
// row keeps the winner's FP32 direct-form distance as e(m).  G is chosen per
// launch by Lk and N (lbg_opts.tc_group forces it).
// Codebooks whose pieces do not add up exactly send their rows to the exact
// FP32 fallback.
// Kernel layout (256 rows per CTA; k_assign_tc takes one row tile per CTA,
// k_assign_tc_p walks the row tiles with one CTA per SM):
//   prologue      the epilogue warps stage the x tile (coalesced) as centred
//                 BF16 rows in shared memory, then each thread writes its half
//                 of its row's A operand (x~ and the norm block) into tensor
//                 memory with tcgen05.st: the MMAs read A from TMEM and only B
//                 from shared memory, which leaves shared-memory bandwidth for
//                 the codebook stream;
//   warp 0        producer: TMA bulk copies of prepared codebook tiles (144
//                 codevectors x KB BF16, already in the MMA's shared-memory
//                 layout) into a ring of 3 stages (2 in k_assign_tc_p);
//   warp 1        allocates 512 TMEM columns, one thread issues the MMAs: job
//                 j = 2 t + a (tile t, accumulator a of 128 rows) accumulates
//                 into slot j % 3 of a ring of three 144-column accumulators;
//   warps 2..17   epilogue, one (row, column half) per thread: tcgen05.ld of
//                 its 72 values per job, running top-2 of group minima with the
//                 group index (two interleaved chains); after the last tile the
//                 two halves of each row merge, compute the exact distances of
//                 the best group's G codevectors, and the half-0 thread
//                 runs the certificate, writes the index and e(m) or flags the
//                 row.
// Every mbarrier wait is bounded (2 s); on a time-out the CTA stops issuing,
// reports LBG_ERR_TIMEOUT, waits for its own copies and frees its TMEM.
#include "lbg_internal.cuh"

#include <cuda_bf16.h>
#include <math.h>

namespace lbg {
namespace {

constexpr int TC_NACC = 2;                     // 128-row accumulators per CTA
constexpr int TC_ROWS = 128 * TC_NACC;         // 256 rows per CTA
constexpr int TC_NT = 144;                     // codevectors per tile (MMA N): 3 accumulator
                                               // slots of 144 columns and A fill the 512 TMEM
                                               // columns; wider MMAs need fewer issues per flop,
                                               // which keeps the single issuing thread ahead of
                                               // the tensor pipe while its SM sub-partition also
                                               // runs epilogue warps (N = 128 issued about one
                                               // MMA per 86 cycles for 64 cycles of work)
constexpr int TC_HALF = TC_NT / 2;             // columns per epilogue thread per tile
// Columns per group (GRP = 2, 4 or 8): the running top-2 is over group minima,
// and a group holds whole split pairs (children 2i, 2i + 1).  Eight columns take
// 0.94 ALU operations per value in the epilogue but eight exact distances per
// row in the tail; four take 1.375 and four, two 2.25 and two.  GrpCfg<GRP>: groups per epilogue
// thread per tile, bits of the in-half group index, and the packing bound
// 2^(JBITS - 23) (packing changes a value by less than this fraction of it).
template <int GRP>
struct GrpCfg;
template <>
struct GrpCfg<2> {
    static constexpr int GROUPS = 36, JBITS = 6;
    static constexpr float PACK = 7.62939453125e-6f;
};
template <>
struct GrpCfg<4> {
    static constexpr int GROUPS = 18, JBITS = 5;
    static constexpr float PACK = 3.814697265625e-6f;
};
template <>
struct GrpCfg<8> {
    static constexpr int GROUPS = 9, JBITS = 4;
    static constexpr float PACK = 1.9073486328125e-6f;
};
constexpr int TC_GRP_MAX = 8;
                                               // by less than this fraction of it
constexpr float TC_EVAL = 9.5367431640625e-7f;   // 2^-20: FP32 evaluation of the second certificate
constexpr int TC_STAGES = 3;
constexpr int TC_EPI_WARPS = 8 * TC_NACC;      // 16: (accumulator, lane quarter, half)
constexpr int TC_THREADS = 32 * (2 + TC_EPI_WARPS);
constexpr int TC_SLOTS = 3;                    // accumulator ring: (tile, accumulator) jobs
constexpr int TC_A_COL = TC_SLOTS * TC_NT;     // TMEM column of the A operand (x~ rows)
constexpr int TC_TMEM_COLS = 512;              // 3 x 144 accumulator columns + 2 x (L + 16)/2
constexpr int TC_LMAX = 64;
constexpr int TC_PIECES = 2;                   // BF16 pieces of c' in B (K blocks of x~ . c')
constexpr int TC_NCH = 2;                      // independent min-chains of the epilogue (the other
                                               // epilogue warps of the sub-partition hide the
                                               // chains' latency; fewer chains, less bookkeeping)
static_assert(TC_A_COL + 2 * ((TC_LMAX + 16) / 2) <= TC_TMEM_COLS, "accumulators + A exceed TMEM");

// The A operand of a row (K BF16 elements, two per TMEM column): x~ and the
// norm block.  For LK <= 32 the row also holds a second piece of x~:
// x~ = x_hi + x_lo + rem with x_hi = bf16(x~), x_lo = bf16(x~ - x_hi) and
// |rem| <= 2^-16 |x~|, so that rows whose centred values are not exact in BF16
// (real-valued data) stay on the tensor cores: a tile with any x_lo != 0 gets
// LK/16 more MMAs per job (x_lo . p_hi) and the certificate counts the terms
// the pieces miss.  Layout [x_hi (LK) | x_lo (LK) | norm (16)], else
// [x~ (LK) | norm (16)].
template <int LK>
struct TcA {
    static constexpr bool SPLIT = LK <= 32;
    static constexpr int KA = SPLIT ? 2 * LK + 16 : LK + 16;
    static constexpr int COLS = KA / 2;                  // TMEM columns per accumulator
    static constexpr int NORM = SPLIT ? 2 * LK : LK;    // element offset of the norm block
};
static_assert(TC_A_COL + 2 * TcA<32>::COLS <= TC_TMEM_COLS && TC_A_COL + 2 * TcA<64>::COLS <= TC_TMEM_COLS,
              "accumulators + A exceed TMEM");
static_assert(TC_HALF == 72 && GrpCfg<2>::GROUPS * 2 == TC_HALF && GrpCfg<8>::GROUPS * 8 == TC_HALF &&
                  GrpCfg<2>::GROUPS <= (1 << GrpCfg<2>::JBITS) && GrpCfg<8>::GROUPS <= (1 << GrpCfg<8>::JBITS),
              "epilogue loads 64 + 8 columns in whole groups");

constexpr float U32 = 5.9604644775390625e-8f;   // 2^-24
constexpr float SLOP = 1.0000305175781250f;     // 1 + 2^-15


// Byte offset of element (row, k) in the canonical K-major, no-swizzle
// layout: 8-row x 16-byte core matrices; core matrices along K are 128 bytes
// apart (LBO), 8-row groups are sbo bytes apart (SBO).
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k, uint32_t sbo)
{
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// tcgen05 shared-memory matrix descriptor: start address, LBO, SBO (all >> 4),
// version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_NT >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// The epilogue steps of one job: group j holds columns GRP j .. GRP j + GRP - 1
// of the thread's half; its minimum (three-input mins) carries the group index
// in its JBITS low mantissa bits (one LOP3; `keymask` = ~(2^JBITS - 1) comes in
// as a kernel argument so that the mask stays in a register and the immediate
// is the index).  Groups enter the running top-2 of their chain two at a time:
// with m = min(k1, k2), h = max(k1, k2), the top-2 of {c1, c2, k1, k2} is
// c1' = min(c1, m), c2' = min(c2, max(c1, m), h) (five operations for two
// groups instead of six; the same values as one group at a time).  Pair p of
// groups goes to chain p % NCH; an odd last group enters chain (GROUPS / 2) % NCH
// alone.
template <int GRP, int J>
__device__ __forceinline__ float group_key(const float *v, int keymask)
{
    const float *g = v + GRP * J;
    float lo;
    if constexpr (GRP == 8)
        lo = fmin3(fmin3(g[0], g[1], g[2]), fmin3(g[3], g[4], g[5]), fminf(g[6], g[7]));
    else if constexpr (GRP == 4)
        lo = fminf(fmin3(g[0], g[1], g[2]), g[3]);
    else
        lo = fminf(g[0], g[1]);
    int kb;
    asm("lop3.b32 %0, %1, %2, %3, 0xEA;" : "=r"(kb) : "r"(__float_as_int(lo)), "r"(keymask), "n"(J));
    return __int_as_float(kb);
}
template <int GRP, int P>
struct GroupSteps {
    __device__ __forceinline__ static void run(const float *v, float *c1, float *c2, int keymask)
    {
        if constexpr (P % 2 == 1) {   // an odd last group enters alone
            GroupSteps<GRP, P - 1>::run(v, c1, c2, keymask);
            constexpr int q = ((P - 1) / 2) % TC_NCH;
            const float k = group_key<GRP, P - 1>(v, keymask);
            c2[q] = fminf(c2[q], fmaxf(c1[q], k));
            c1[q] = fminf(c1[q], k);
        } else if constexpr (P >= 2) {
            GroupSteps<GRP, P - 2>::run(v, c1, c2, keymask);
            constexpr int q = ((P - 2) / 2) % TC_NCH;
            const float k1 = group_key<GRP, P - 2>(v, keymask), k2 = group_key<GRP, P - 1>(v, keymask);
            const float m = fminf(k1, k2), h = fmaxf(k1, k2);
            c2[q] = fmin3(c2[q], fmaxf(c1[q], m), h);
            c1[q] = fminf(c1[q], m);
        }
    }
};

__device__ __forceinline__ void named_sync(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Store n consecutive 32-bit columns of the warp's 32 lanes (n = 4, 8, 16).
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t *r)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
                 "r"(r[2]), "r"(r[3])
                 : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *r)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *r)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
                     taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
                 "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
}
template <int NW>
__device__ __forceinline__ void tmem_st_words(uint32_t taddr, const uint32_t *r)
{
    int c = 0;
    if (NW - c >= 16) { tmem_st16(taddr + c, r + c); c += 16; }
    if (NW - c >= 8) { tmem_st8(taddr + c, r + c); c += 8; }
    if (NW - c >= 4) { tmem_st4(taddr + c, r + c); c += 4; }
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// tcgen05.mma, kind::f16, with the A operand in tensor memory (row = lane,
// two BF16 of K per 32-bit column) and B in shared memory, and tcgen05.commit,
// each issued by one elected lane of a converged warp (the whole warp runs the
// issue loop, so its addresses stay warp-uniform).
__device__ __forceinline__ void mma_bf16_ta_elect(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p, e;\n\telect.sync _|e, 0xffffffff;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(TC_IDESC), "r"(acc)
        : "memory");
}
// One whole job of the L = 64 form (K = 2 x 64 + 16: nine MMAs, the x~ K-blocks
// kk = 0..3 against both pieces of c', then the norm block) and its commit in one
// instruction sequence (addresses formed by adds inside it, one election): the
// issuing warp shares its SM sub-partition with ALU-bound epilogue warps and gets
// few issue slots, so the fewer instructions per MMA the better.
__device__ __forceinline__ void job9_elect(uint32_t d, uint32_t a0, uint64_t b0, uint32_t bar)
{
    asm volatile(
        "{\n\t.reg .pred e, pf, pt;\n\t.reg .b32 a1, a2, a3, a4;\n\t"
        ".reg .b64 b1, b2, b3, b4, b5, b6, b7, b8;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 pf, %4, %4;\n\t"
        "setp.eq.b32 pt, %4, %4;\n\t"
        "add.u32 a1, %1, 8;\n\tadd.u32 a2, %1, 16;\n\tadd.u32 a3, %1, 24;\n\tadd.u32 a4, %1, 32;\n\t"
        "add.s64 b1, %2, 16;\n\tadd.s64 b2, %2, 32;\n\tadd.s64 b3, %2, 48;\n\tadd.s64 b4, %2, 64;\n\t"
        "add.s64 b5, %2, 80;\n\tadd.s64 b6, %2, 96;\n\tadd.s64 b7, %2, 112;\n\tadd.s64 b8, %2, 128;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, pf;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], b1, %3, pt;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], b2, %3, pt;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], b3, %3, pt;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], b4, %3, pt;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], b5, %3, pt;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], b6, %3, pt;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], b7, %3, pt;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a4], b8, %3, pt;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%5];\n\t}" ::"r"(d),
        "r"(a0), "l"(b0), "r"(TC_IDESC), "r"(0), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mma_commit_elect(uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}

// Staged BF16 x~ rows in shared memory.  Rows of LK < 64 elements are padded
// by 8 (16 bytes) so that a thread per row reads 16-byte chunks without bank
// conflicts; 64-element rows (128 bytes) are not padded but have their eight
// 16-byte chunks permuted by the row (chunk c at c ^ (row & 7)), which does
// the same in less space.
template <int LK>
struct XsRow {
    static constexpr int STR = LK == 64 ? 64 : LK + 8;   // BF16 per staged row
};
template <int LK>
__device__ __forceinline__ int xs_at(int r, int l)
{
    if (LK == 64) return r * 64 + ((((l >> 3) ^ (r & 7)) << 3) | (l & 7));
    return r * XsRow<LK>::STR + l;
}

// The A words of one half of a row (half H of the K = LK + 16 elements, two
// BF16 per word): centred x~ from the staged row (zero past L and for rows
// past M), and the running sum of squares of those x~ in order.  Half 1 also
// holds the norm block, filled in later.  FULL: L == LK, nothing to mask.
template <int LK, int H, bool FULL>
__device__ __forceinline__ void a_words(const __nv_bfloat16 *XS, const __nv_bfloat16 *XL, int crow, int L,
                                        bool live, uint32_t *wv, float &part)
{
    constexpr int KA = TcA<LK>::KA, HK = KA / 2, E0 = H * HK;
    constexpr int XEND = TcA<LK>::NORM;                // x~ elements (both pieces) end here
    constexpr int XE = E0 + HK <= XEND ? HK : XEND - E0;   // x~ elements in this half
#pragma unroll
    for (int w = 0; w < HK / 2; ++w) wv[w] = 0u;
#pragma unroll
    for (int g = 0; g < XE / 8; ++g) {
        // element E0 + 8 g: x_hi at l = e, or (split) x_lo at l = e - LK
        const int e = E0 + 8 * g;
        const bool lo_piece = TcA<LK>::SPLIT && e >= LK;
        const int l8 = lo_piece ? e - LK : e;
        const __nv_bfloat16 *src = lo_piece ? XL : XS;
        const uint4 q = live ? *reinterpret_cast<const uint4 *>(src + xs_at<LK>(crow, l8))
                             : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t qs[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e0 = l8 + 2 * j;
            const uint32_t lo = (FULL || e0 < L) ? (qs[j] & 0xFFFFu) : 0u;
            const uint32_t hi = (FULL || e0 + 1 < L) ? (qs[j] >> 16) : 0u;
            wv[4 * g + j] = lo | (hi << 16);
            if (!TcA<LK>::SPLIT) {   // ||x~||^2 of the exact form; the split form sums it apart
                const float a = __uint_as_float(lo << 16), b = __uint_as_float(hi << 16);
                part = fmaf(a, a, part);
                part = fmaf(b, b, part);
            }
        }
    }
}

// Accumulation-error coefficient tau of the file header for KB accumulated
// BF16 elements.
__host__ __device__ inline double tc_tau(int KB)
{
    return (double)(KB / 16 + 2) * 2.384185791015625e-7 * 1.0078125;   // 2^-22, (1 + 2^-7)
}

// K of one B row: the pieces of c' (LK each) and the 16-element norm block.
__host__ __device__ constexpr int tc_kb(int LK) { return TC_PIECES * LK + 16; }

// Accumulated K of a job: x_hi . (p_hi + p_mid), x_lo . p_hi on a split tile,
// the norm block.  tau of the split form also covers sum |x_lo p_hi| (below
// 2^-7 of the rest): the factor 1 + 2^-6.
__host__ __device__ constexpr int tc_keff(int LK) { return LK <= 32 ? 3 * LK + 16 : 2 * LK + 16; }
__host__ __device__ inline double tc_tau_eff(int LK)
{
    return tc_tau(tc_keff(LK)) * (LK <= 32 ? 1.015625 : 1.0);
}

// Split an FP32 value into two BF16 pieces h + m; returns the remainder
// v - h - m, which is exact in FP32 (each subtraction is; |v - h - m| <= 2^-16 |v|
// for normal numbers), NaN or Inf for non-finite v.
__device__ __forceinline__ float split2(float v, __nv_bfloat16 &h, __nv_bfloat16 &m)
{
    h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    return r1 - __bfloat162float(m);
}

// Split an FP32 value into three BF16 pieces that add up to it exactly (for
// normal numbers); returns false if the remainder is not zero.
__device__ __forceinline__ bool split3(float v, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l)
{
    h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    l = __float2bfloat16_rn(r2);
    return isfinite(v) ? (r2 - __bfloat162float(l)) == 0.f : isinf(v);
}

// Prepared BF16 codebook: codevector rows x KB BF16 in the core-matrix layout
// (8-row groups SBO = KB/8 * 128 bytes apart), so that tile t (TC_NT rows) is
// the contiguous block at t * TC_NT * KB * 2 bytes; K columns [0,Lk) p_hi,
// [Lk,2Lk) p_mid of c' = -2 (c - mu), [2Lk, 2Lk+3) the pieces of s0, three
// ones, zeros elsewhere; padding codevectors (up to whole tiles) have
// s0 = 2^100.  Also k'_n, the chunk-major original codebook for the exact
// fallback (both BN-padded), max ||c~|| and max ||c' - p_hi - p_mid||.
constexpr int PT_N = 32;   // codevectors per preparation CTA

// Rows of the prepared codebook for N codevectors: whole tiles and whole BN
// chunks, in whole preparation CTAs.
__host__ __device__ inline int tc_prep_rows(int N)
{
    const int t = round_up(N, TC_NT), b = round_up(N, BN);
    return round_up(t > b ? t : b, PT_N);
}

template <int LK>
__global__ void __launch_bounds__(256)
    k_prep_tc(const float *__restrict__ C, const int32_t *n_dev, int n_host, int L, int Lp,
              const float *__restrict__ mu, __nv_bfloat16 *__restrict__ Bp, float *__restrict__ kn,
              float *__restrict__ CT, DevState *st)
{
    if (st->finished) return;
    const int N = cur_n(n_dev, n_host);
    if (N <= st->direct_max) return;   // k_assign_direct's stages need no prepared codebook
    const int n0 = blockIdx.x * PT_N;
    if (n0 >= tc_prep_rows(N)) return;
    const int NPk = round_up(N, BN);      // k'_n and CT entries (BN-padded)
    constexpr int KB = tc_kb(LK);
    constexpr uint32_t sbo = (uint32_t)(KB / 8) * 128u;
    __shared__ float cs[PT_N][LK + 1];   // codevectors as given (0 past L / N)
    __shared__ float ct[PT_N][LK + 1];   // centred c~ = c - mu
    __shared__ float s0s[PT_N];
    __shared__ double sqs[PT_N];
    __shared__ int s_bad, s_inexact;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        s_bad = 0;
        s_inexact = 0;
    }
    __syncthreads();
    // this CTA's block of C is contiguous: read it coalesced
    for (int i = tid; i < PT_N * L; i += blockDim.x) {
        const int r = i / L, l = i - r * L, n = n0 + r;
        const float c = n < N ? C[(size_t)n0 * L + i] : 0.f;
        if (!isfinite(c)) s_bad = 1;
        cs[r][l] = c;
        ct[r][l] = n < N ? c - mu[l] : 0.f;
    }
    for (int i = tid; i < PT_N * (LK - L); i += blockDim.x) {
        const int r = i / (LK - L), l = L + i % (LK - L);
        cs[r][l] = 0.f;
        ct[r][l] = 0.f;
    }
    __syncthreads();
    // ||c~||^2 in FP64: warp w sums codevectors w, w + 8, ... over its lanes
    // (fixed shuffle tree), then k'_n and the chain start s0
    for (int r = warp; r < PT_N; r += blockDim.x / 32) {
        double sq = 0.0;
        for (int l = lane; l < L; l += 32) sq = fma((double)ct[r][l], (double)ct[r][l], sq);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) sqs[r] = sq;
    }
    __syncthreads();
    if (tid < PT_N) {   // warp 0: one codevector per lane
        const int n = n0 + tid;
        uint32_t cbits = 0u;
        if (n < N) {
            const double sq = sqs[tid];
            const double k = (2.0 * tc_tau_eff(LK) + 1.1920928955078125e-7) * sq;   // 2 tau + 2^-23
            const float kf = __double2float_ru(k);
            s0s[tid] = __double2float_rn(sq - (double)kf);
            kn[n] = kf;
            cbits = __float_as_uint(__fsqrt_ru(__double2float_ru(sq)));   // >= ||c~_n||
        } else {
            s0s[tid] = 1.2676506002282294e30f;   // padding: 2^100, finite so index packing cannot make a NaN
            if (n < NPk) kn[n] = 0.f;
        }
        // max ||c~_n|| of the block (bits of non-negative floats order as integers): one atomic per CTA
        cbits = __reduce_max_sync(0xffffffffu, cbits);
        if (tid == 0 && cbits) atomicMax(&st->cmax_bits, cbits);
    }
    __syncthreads();
    // B rows: K in [0, LK) p_hi of c' = -2 c~, [LK, 2LK) p_mid, then the s0
    // pieces, three ones (x the row's X2 pieces), zeros.  A unit is (codevector,
    // 8 dims): each value is split once and its two pieces go out as two
    // 16-byte core-matrix rows; the squared remainders c' - p_hi - p_mid of the
    // unit (exact in FP32, summed in FP64 in a fixed order) go to rsq.
    uint8_t *tile = reinterpret_cast<uint8_t *>(Bp);
    const int rt = n0;
    constexpr int G8 = LK / 8;
    __shared__ double rsq[PT_N][G8];
    bool inexact = false;
    for (int u = tid; u < PT_N * G8; u += blockDim.x) {
        const int r = u / G8, g = u - r * G8, l0 = 8 * g;
        uint32_t w[TC_PIECES][4];
        double q = 0.0;
#pragma unroll
        for (int e2 = 0; e2 < 4; ++e2) {
            __nv_bfloat16 h0, m0, h1, m1;
            const float r0 = split2(-2.0f * ct[r][l0 + 2 * e2], h0, m0);
            const float r1 = split2(-2.0f * ct[r][l0 + 2 * e2 + 1], h1, m1);
            inexact |= !isfinite(r0) || !isfinite(r1);
            q = fma((double)r0, (double)r0, q);
            q = fma((double)r1, (double)r1, q);
            w[0][e2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            w[1][e2] = (uint32_t)__bfloat16_as_ushort(m0) | ((uint32_t)__bfloat16_as_ushort(m1) << 16);
        }
        rsq[r][g] = q;
#pragma unroll
        for (int pc = 0; pc < TC_PIECES; ++pc)
            *reinterpret_cast<uint4 *>(tile + core_off(rt + r, pc * LK + l0, sbo)) =
                make_uint4(w[pc][0], w[pc][1], w[pc][2], w[pc][3]);
    }
    if (tid < PT_N) {   // the norm block of each codevector: two 16-byte rows
        const int r = tid;
        const bool real = n0 + r < N;
        __nv_bfloat16 h, m, o;
        const bool ex = split3(s0s[r], h, m, o);
        if (real) inexact |= !ex;
        const uint32_t one = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
        uint4 nb;
        if (real) {
            nb.x = (uint32_t)__bfloat16_as_ushort(h) | ((uint32_t)__bfloat16_as_ushort(m) << 16);
            nb.y = (uint32_t)__bfloat16_as_ushort(o) | (one << 16);
            nb.z = one | (one << 16);
            nb.w = 0u;
        } else {
            nb = make_uint4((uint32_t)__bfloat16_as_ushort(h), 0u, 0u, 0u);
        }
        *reinterpret_cast<uint4 *>(tile + core_off(rt + r, TC_PIECES * LK, sbo)) = nb;
        *reinterpret_cast<uint4 *>(tile + core_off(rt + r, TC_PIECES * LK + 8, sbo)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (inexact) s_inexact = 1;
    // FP32 codebook for the exact fallback, chunk-major (coalesced along n)
    if (n0 < NPk)
        for (int i = tid; i < PT_N * Lp; i += blockDim.x) {
            const int l = i / PT_N, r = i - l * PT_N, n = n0 + r;
            CT[((size_t)(n / EXACT_SW) * Lp + l) * EXACT_SW + n % EXACT_SW] = l < L ? cs[r][l] : 0.f;
        }
    __syncthreads();
    if (tid < PT_N) {   // warp 0: ||c'_n - p_hi - p_mid|| rounded up, max of the block, one atomic
        double q = 0.0;
#pragma unroll
        for (int g = 0; g < G8; ++g) q += rsq[tid][g];
        uint32_t rbits = __float_as_uint(__double2float_ru(sqrt(q)));
        rbits = __reduce_max_sync(0xffffffffu, rbits);
        if (tid == 0 && rbits) atomicMax(&st->rho_bits, rbits);
    }
    if (tid == 0) {
        if (s_bad) flag_error(st, ERR_NONFINITE);
        if (s_inexact) atomicOr(&st->tc_inexact, 1);
    }
}

// ---------------------------------------------------------------- shared parts
// Static shared state of the assignment kernels.
struct TcSmem {
    uint64_t full[3], empty[3], tfull[TC_SLOTS], tempty[TC_SLOTS], xfull, xempty, aready;
    uint32_t tmem_base;
    int abort, inexact, prod_last, mma_tile, mma_job, x_issued, x_done;
    int xsplit;        // the (per-tile kernel's) tile has x_lo pieces
    int xsplit2[2];    // the same per row tile of the persistent kernel, by parity
    union {   // the tail's two uses are separated by a named barrier
        struct {
            float v1[2][TC_ROWS], v2[2][TC_ROWS];   // the halves' top-2 (tail merge)
            int i1[2][TC_ROWS];
        } m;
        struct {
            float d[TC_GRP_MAX][TC_ROWS];           // exact distances of the best group (tail);
                                                    // d[0..1]: ||x~||^2 halves (A write)
            float k[2][TC_ROWS];                    // the halves' largest k' of the group (tail)
        } r;
    };
};

__device__ __forceinline__ bool named_sync_or(int id, int threads, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(threads)
        : "memory");
    return r != 0;
}

// One centred x value into the staged BF16 rows; flags non-finite input and
// values for which x~ = x - mu is not exact in FP32 (TwoSum error) or BF16.
// In the split form (LK <= 32) x~ = fl(x - mu) need not be exact (the
// certificate's centring term covers it) and its second BF16 piece goes to XL;
// `split` records a nonzero second piece.
template <int LK>
__device__ __forceinline__ void tc_put_x(__nv_bfloat16 *XS, __nv_bfloat16 *XL, int i, int L, float xv,
                                         const float *__restrict__ mu, bool &bad, bool &inexact, bool &split)
{
    const int r = i / L, l = i - r * L;
    bad = bad || !isfinite(xv);
    const float ml = __ldg(mu + l);
    const float v = __fsub_rn(xv, ml);
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    if constexpr (TcA<LK>::SPLIT) {
        const __nv_bfloat16 lo = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(b)));   // v - b exact
        split = split || __bfloat162float(lo) != 0.f;
        XL[xs_at<LK>(r, l)] = lo;
    } else {
        const float bb = __fsub_rn(v, xv);
        const float err = __fadd_rn(__fsub_rn(xv, __fsub_rn(v, bb)), __fsub_rn(-ml, bb));
        inexact = inexact || err != 0.f || (__bfloat162float(b) != v);
    }
    XS[xs_at<LK>(r, l)] = b;
}

// The A operand in tensor memory: each epilogue thread writes its half of its
// row's K = TcA<LK>::KA BF16 (two per column): x~ (both pieces in the split
// form; zero past L and for rows past M), then in half 1 the norm block 1 1 1
// (x s0 pieces), X2 = ||x~||^2 in three BF16 pieces, zeros.  ||x~||^2 is half
// 0's sum of squares plus half 1's in that order.  Returns ||x~||^2 of the
// thread's row; the caller fences and synchronises before the MMAs read A.
template <int LK, bool FULL>
__device__ __forceinline__ float tc_write_a(const __nv_bfloat16 *XS, const __nv_bfloat16 *XL, int L, bool live,
                                            int crow, int half, int acc, int warp, uint32_t tmem, TcSmem &sh)
{
    constexpr int KA = TcA<LK>::KA, NW = KA / 4;
    uint32_t wv[NW];
    float part = 0.f;
    if (half == 0) a_words<LK, 0, FULL>(XS, XL, crow, L, live, wv, part);
    else a_words<LK, 1, FULL>(XS, XL, crow, L, live, wv, part);
    if (TcA<LK>::SPLIT && live) {
        // ||x~||^2 as sum (x_hi + x_lo)^2 in index order, half 0 over l < LK / 2 (the rest in
        // half 1); it differs from ||x~||^2 by less than 2^-14 ||x~||^2 besides rounding
#pragma unroll
        for (int l = half * (LK / 2); l < (half + 1) * (LK / 2); ++l) {
            if (!FULL && l >= L) break;
            const float v = __bfloat162float(XS[xs_at<LK>(crow, l)]) + __bfloat162float(XL[xs_at<LK>(crow, l)]);
            part = fmaf(v, v, part);
        }
    }
    sh.r.d[half][crow] = part;
    named_sync(1, 32 * TC_EPI_WARPS);
    const float xn2 = __fadd_rn(sh.r.d[0][crow], sh.r.d[1][crow]);
    if (half == 1) {
        __nv_bfloat16 h, mi, lo;
        split3(xn2, h, mi, lo);
        const uint32_t one = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
        constexpr int w0 = (TcA<LK>::NORM - KA / 2) / 2;   // first norm-block word of half 1
        wv[w0] = one | (one << 16);
        wv[w0 + 1] = one | ((uint32_t)__bfloat16_as_ushort(h) << 16);
        wv[w0 + 2] = (uint32_t)__bfloat16_as_ushort(mi) | ((uint32_t)__bfloat16_as_ushort(lo) << 16);
    }
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    tmem_st_words<NW>(tmem + lane_base + (uint32_t)(TC_A_COL + acc * (KA / 2) + half * NW), wv);
    tmem_st_wait();
    return xn2;
}

// The epilogue of one row tile: for each codebook tile t, job j0 + 2t + acc
// (accumulator slot (j0 + 2t + acc) % 3); the thread's 72 values per job go
// through the group top-2; returns the merged (V1, V2, group's first column)
// of the thread's half: V1 the smallest group minimum, V2 the second smallest
// (the smallest value outside V1's group).
template <int GRP>
__device__ __forceinline__ void tc_jobs(TcSmem &sh, uint32_t tmem, int warp, int lane, int acc, int half,
                                        int ntiles, int j0, int keymask, float &V1, float &V2, int &i1)
{
    constexpr int NCH = TC_NCH;
    constexpr int JMASK = (1 << GrpCfg<GRP>::JBITS) - 1;
    float c1[NCH], c2[NCH];
    int cg[NCH];
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
        c1[q] = INFINITY;
        c2[q] = INFINITY;
        cg[q] = 0;
    }
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    // job j = j0 + 2 t + acc: slot j % 3 and the parity of j / 3, stepped by j += 2
    int slot = (j0 + acc) % TC_SLOTS;
    uint32_t par = (uint32_t)((j0 + acc) / TC_SLOTS) & 1u;
    for (int t = 0; t < ntiles; ++t) {
        if (t > 0) {
            slot += 2;
            if (slot >= TC_SLOTS) {
                slot -= TC_SLOTS;
                par ^= 1u;
            }
        }
        if (sh.abort || !mbar_wait_bounded_sleep(&sh.tfull[slot], par)) {
            sh.abort = 1;
            continue;
        }
        tc_fence_after();
        float v[TC_HALF];
        const uint32_t col = (uint32_t)(slot * TC_NT + half * TC_HALF);
        tmem_ld32(tmem + lane_base + col, v);
        tmem_ld32(tmem + lane_base + col + 32u, v + 32);
        tmem_ld8(tmem + lane_base + col + 64u, v + 64);
        tmem_ld_wait();
        // the values are in registers: hand the accumulator back to the MMA
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.tempty[slot]);
        float s1[NCH];
#pragma unroll
        for (int q = 0; q < NCH; ++q) s1[q] = c1[q];
        GroupSteps<GRP, GrpCfg<GRP>::GROUPS>::run(v, c1, c2, keymask);
#pragma unroll
        for (int q = 0; q < NCH; ++q) cg[q] = c1[q] < s1[q] ? t : cg[q];
    }
    // merge the chains; i1 is the first column of the minimum's group:
    // tile * TC_NT + half * TC_HALF + GRP * (the low bits)
    V1 = c1[0];
    V2 = c2[0];
    i1 = cg[0] * TC_NT + half * TC_HALF + GRP * (__float_as_int(c1[0]) & JMASK);
#pragma unroll
    for (int q = 1; q < NCH; ++q) {
        const int iq = cg[q] * TC_NT + half * TC_HALF + GRP * (__float_as_int(c1[q]) & JMASK);
        V2 = fminf(fminf(V2, c2[q]), fmaxf(V1, c1[q]));
        const bool take = c1[q] < V1 || (c1[q] == V1 && iq < i1);
        V1 = take ? c1[q] : V1;
        i1 = take ? iq : i1;
    }
}

// The end of a row tile (all 16 epilogue warps; uses named barriers 1 and 2):
// the two halves of a row merge their top-2 in a fixed order; the candidate
// is a member of the group i1 .. i1 + 7, and each half computes the exact
// FP32 distances of four members.  With L a multiple of 4 the warp does it
// cooperatively: a half-warp per row, a float4 of x and of the codevector per
// lane (coalesced reads of X and C), each lane sums its four terms
// (x_l - c_l)^2 in order, and a butterfly over the 16 lanes of each half-warp
// reduces the 16 rows' partial sums at once (a fixed tree: 15 shuffles per
// lane); the owner lane of each row takes its sum.  The half-0 thread then
// takes the member with the smallest distance when it beats the other seven
// by more than the rounding bound of the FP32 sums, runs the certificates,
// and writes a(m), e(m) or flags the row.  `usable` = the tile's x~ and the
// codebook split are exact.
// `xsplit`: the tile's x~ has second BF16 pieces (split form).
template <int LK, int GRP>
__device__ __forceinline__ void tc_tail(TcSmem &sh, int warp, int lane, int acc, int half, int rr,
                                        int64_t m0, const float *__restrict__ X, int64_t M, int L, int N,
                                        const float *__restrict__ C, const float *__restrict__ kn, float xn2,
                                        bool usable_tile, bool xsplit, float cmax, float rho, float V1, float V2,
                                        int i1, DevState *st,
                                        int32_t *__restrict__ assign, float *__restrict__ e,
                                        int32_t *__restrict__ flags, int64_t flag_base)
{
    const int crow = 128 * acc + rr;
    const int64_t m = m0 + crow;
    sh.m.v1[half][crow] = V1;
    sh.m.v2[half][crow] = V2;
    sh.m.i1[half][crow] = i1;
    named_sync(1, 32 * TC_EPI_WARPS);
    {
        const float A1 = sh.m.v1[0][crow], A2 = sh.m.v2[0][crow], B1 = sh.m.v1[1][crow], B2 = sh.m.v2[1][crow];
        const int ai = sh.m.i1[0][crow], bi = sh.m.i1[1][crow];
        V2 = fminf(fminf(A2, B2), fmaxf(A1, B1));
        const bool take = B1 < A1 || (B1 == A1 && bi < ai);
        V1 = take ? B1 : A1;
        i1 = take ? bi : ai;
    }
    named_sync(2, 32 * TC_EPI_WARPS);   // merge inputs read: sh.r may now overwrite sh.m
    const bool usable = m < M && !sh.abort && usable_tile && i1 >= 0 && i1 < N && V1 < INFINITY;
    // the best group is codevectors i1 .. i1 + GRP - 1; this half scores members
    // i1 + (GRP / 2) half + g
    float kmax = 0.f;
    const bool coop = (L & 3) == 0 && ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(X)) & 15u) == 0;
    // members in passes of CPB: the x rows are loaded once per pass for all its members
    constexpr int CPB = GRP / 2 < 2 ? GRP / 2 : 2;
#pragma unroll 1
    for (int g0 = 0; g0 < GRP / 2; g0 += CPB) {
        int ccand[CPB];
#pragma unroll
        for (int c = 0; c < CPB; ++c) {
            const int cand = i1 + (GRP / 2) * half + g0 + c;
            ccand[c] = (usable && cand < N) ? cand : -1;
            if (ccand[c] >= 0) kmax = fmaxf(kmax, __ldg(kn + ccand[c]));
        }
        float dc[CPB];
#pragma unroll
        for (int c = 0; c < CPB; ++c) dc[c] = INFINITY;
        if (coop) {
            const int rq = lane & 15, sub = lane >> 4;
            const int64_t mrow0 = m0 + 128 * acc + 32 * (warp & 3);   // row of lane 0
            float p[CPB][16];
#pragma unroll
            for (int bt = 0; bt < 4; ++bt) {   // four batches of 4 rows
                int crs[CPB][4];
#pragma unroll
                for (int c = 0; c < CPB; ++c)
#pragma unroll
                    for (int k = 0; k < 4; ++k) crs[c][k] = __shfl_sync(0xffffffffu, ccand[c], 2 * (4 * bt + k) + sub);
                float4 c4[CPB][4], x4[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int64_t mr = mrow0 + 2 * (4 * bt + k) + sub;
                    bool any = false;
#pragma unroll
                    for (int c = 0; c < CPB; ++c) {
                        const bool on = crs[c][k] >= 0 && 4 * rq < L;
                        any = any || on;
                        c4[c][k] = on ? __ldg(reinterpret_cast<const float4 *>(C + (size_t)crs[c][k] * L) + rq)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    x4[k] = any ? __ldg(reinterpret_cast<const float4 *>(X + mr * L) + rq)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int c = 0; c < CPB; ++c)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float d = __fsub_rn(x4[k].x, c4[c][k].x);
                        float q = d * d;
                        d = __fsub_rn(x4[k].y, c4[c][k].y);
                        q = fmaf(d, d, q);
                        d = __fsub_rn(x4[k].z, c4[c][k].z);
                        q = fmaf(d, d, q);
                        d = __fsub_rn(x4[k].w, c4[c][k].w);
                        p[c][4 * bt + k] = fmaf(d, d, q);
                    }
            }
#pragma unroll
            for (int c = 0; c < CPB; ++c) {
#pragma unroll
                for (int lvl = 8; lvl >= 1; lvl >>= 1) {
                    const bool up = (rq & lvl) != 0;
#pragma unroll
                    for (int i = 0; i < lvl; ++i) {
                        const float send = up ? p[c][i] : p[c][i + lvl];
                        const float keep = up ? p[c][i + lvl] : p[c][i];
                        p[c][i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, lvl));
                    }
                }
                // lane (sub, rq) now holds the sum of row 2 rq + sub
                const float got = __shfl_sync(0xffffffffu, p[c][0], (lane & 1) * 16 + (lane >> 1));
                if (ccand[c] >= 0) dc[c] = got;
            }
        } else {
#pragma unroll
            for (int c = 0; c < CPB; ++c)
                if (ccand[c] >= 0) {
                    const float *xr = X + m * L;
                    const float *cr = C + (size_t)ccand[c] * L;
                    float d2 = 0.f;
                    for (int l = 0; l < L; ++l) {
                        const float d = __fsub_rn(__ldg(xr + l), __ldg(cr + l));
                        d2 = fmaf(d, d, d2);
                    }
                    dc[c] = d2;
                }
        }
#pragma unroll
        for (int c = 0; c < CPB; ++c) sh.r.d[(GRP / 2) * half + g0 + c][crow] = dc[c];
    }
    sh.r.k[half][crow] = kmax;
    named_sync(2, 32 * TC_EPI_WARPS);
    if (half == 0 && m < M && !sh.abort) {
        // the group member with the smallest FP32 direct-form distance wins when every other
        // member's distance exceeds it by more than the rounding bound of the FP32 sums,
        // |fl(d2) - d2| <= (L + 2) u d2 for any order of the L terms (kept as (L + 4) u); else
        // the row is not certified
        bool certified = false;
        if (usable) {
            float dd[GRP];
#pragma unroll
            for (int g = 0; g < GRP; ++g) dd[g] = sh.r.d[g][crow];
            int w = 0;
#pragma unroll
            for (int g = 1; g < GRP; ++g) w = dd[g] < dd[w] ? g : w;
            const float da = dd[w];
            bool sure = true;
#pragma unroll
            for (int g = 0; g < GRP; ++g) {   // members past N have no distance (infinity)
                const float tol = (float)(L + 4) * U32 * (da + dd[g]) * SLOP;
                if (g != w && dd[g] < INFINITY && !(da < dd[g] - tol)) sure = false;
            }
            const int ii = i1 + w;
            // k' of the member that produced V1 is unknown: the group's largest bounds it
            const float ka = fmaxf(sh.r.k[0][crow], sh.r.k[1][crow]);
            if (sure) {
                const double tau = tc_tau_eff(LK);
                const float xn2u = xn2 * SLOP;
                const float R = 2.f * (float)tau * xn2u * SLOP;
                const float eta = U32 * (sqrtf(xn2u) + cmax) * SLOP;
                // index packing of the group minima
                const float pack = GrpCfg<GRP>::PACK * (fabsf(V1) + fabsf(V2));
                // the MMA sums x~ . (p_hi + p_mid) and misses x~ . r_n, r_n = c'_n - p_hi - p_mid:
                // |x~ . r_n| <= ||x~|| rho for every n (Cauchy-Schwarz).  A split tile sums
                // x_hi . (p_hi + p_mid) + x_lo . p_hi instead: it misses x_hi . r_n (<= ||x~|| rho
                // (1 + 2^-8)), x_lo . (p_mid + r_n) and rem . c'_n, with ||x_lo|| <= 2^-8 ||x~||,
                // ||p_mid|| <= 2^-8 (1 + 2^-8) ||c'||, ||rem|| <= 2^-16 ||x~|| and ||c'|| <= 2 cmax:
                // all within ||x~|| (rho (1 + 2^-7) + 2^-14 (1 + 2^-7) cmax)
                const float E = xsplit ? sqrtf(xn2u) * (rho + 6.103515625e-05f * cmax) * 1.0078125f * SLOP
                                         : sqrtf(xn2u) * rho * SLOP;
                // |fl(||x~||^2) - ||x~||^2|: X2 as the MMA saw it (a split tile's X2 is
                // sum (x_hi + x_lo)^2: another 2^-14 ||x~||^2)
                const float xerr = (float)(L + 2) * U32 * xn2u + (xsplit ? 6.103515625e-05f * xn2u : 0.f);
                // the member j that produced V1 has ||x~ - c~_j||^2 - k'_j ~ V1 (X2 included), and
                // the winner ii is not farther than j: bound its g1^2 from above
                const float g1sq = V1 + 2.f * ka + R + pack + E + xerr;
                const float g1 = sqrtf(fmaxf(g1sq, 0.f)) * SLOP;
                const float margin = (2.f * R + 2.f * ka + pack + 2.f * E + 4.f * eta * (g1 + eta)) * SLOP;
                certified = (V2 - V1) > margin;
                if (!certified) {
                    // second certificate: every codevector outside the group has
                    // ||x - c_n||^2 >= (sqrt(V2 - R - E - pack - xerr) - eta)^2, which must
                    // exceed the winner's direct-form distance rounded up
                    const float lb = V2 - (R + E + pack + xerr) * SLOP;
                    const float ub = da * (1.f + (float)(L + 4) * U32) * SLOP;
                    certified = lb > 0.f && (lb - 2.f * eta * sqrtf(lb) * SLOP) * (1.f - TC_EVAL) > ub * (1.f + TC_EVAL);
                }
            }
            if (certified) {
                assign[m] = ii;
                e[m] = da;
            }
        }
        if (!certified) flags[atomicAdd(&st->nflag, 1)] = (int32_t)(flag_base + m);
    }
}


// One job's MMAs (not the JOB9 form): x_hi . p_hi, x_hi . p_mid, x_lo . p_hi on
// a split tile, and the norm block; d the accumulator, at the A operand.
template <int LK>
__device__ __forceinline__ void mma_job_elect(uint32_t d, uint32_t at, uint64_t bst, bool xsplit)
{
#pragma unroll
    for (int seg = 0; seg < TC_PIECES; ++seg)
#pragma unroll
        for (int kk = 0; kk < LK / 16; ++kk)
            mma_bf16_ta_elect(d, at + (uint32_t)(8 * kk), bst + (uint64_t)(seg * LK + kk * 16), (seg | kk) ? 1u : 0u);
    if (TcA<LK>::SPLIT && xsplit)
#pragma unroll
        for (int kk = 0; kk < LK / 16; ++kk)
            mma_bf16_ta_elect(d, at + (uint32_t)(LK / 2 + 8 * kk), bst + (uint64_t)(kk * 16), 1u);
    mma_bf16_ta_elect(d, at + (uint32_t)(TcA<LK>::NORM / 2), bst + (uint64_t)(TC_PIECES * LK), 1u);
}

// ---------------------------------------------------------------- one CTA per row tile
template <int LK, int GRP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_assign_tc(const float *__restrict__ X, int64_t M, int L,
                const __nv_bfloat16 *__restrict__ Bp, const float *__restrict__ kn,
                const int32_t *n_dev, int n_host, const float *__restrict__ mu,
                const float *__restrict__ C, DevState *st, int32_t *__restrict__ assign,
                float *__restrict__ e, int32_t *__restrict__ flags, int keymask,
                int64_t flag_base, int n_lo, int n_hi)
{
    if (st->finished) return;
    const int N = cur_n(n_dev, n_host);
    if (N < n_lo || N >= n_hi || N <= st->direct_max) return;   // another kernel serves this size
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ TcSmem sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (N + TC_NT - 1) / TC_NT;
    constexpr int KB = tc_kb(LK);
    constexpr int XSTR = XsRow<LK>::STR;                       // staged row stride (BF16)
    constexpr uint32_t sbo_b = (uint32_t)(KB / 8) * 128u;
    constexpr uint32_t xs_bytes = (uint32_t)TC_ROWS * XSTR * 2u;
    constexpr uint32_t xl_bytes = TcA<LK>::SPLIT ? xs_bytes : 0u;   // x_lo rows (split form)
    constexpr uint32_t stage_bytes = (uint32_t)TC_NT * KB * 2u;
    __nv_bfloat16 *XS = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *XL = reinterpret_cast<__nv_bfloat16 *>(smem + xs_bytes);
    uint8_t *Bs = smem + xs_bytes + xl_bytes;
    const int64_t m0 = (int64_t)blockIdx.x * TC_ROWS;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], 1);
        }
        for (int b = 0; b < TC_SLOTS; ++b) {
            mbar_init(&sh.tfull[b], 1);
            mbar_init(&sh.tempty[b], TC_EPI_WARPS / TC_NACC);
        }
        fence_mbar_init();
        sh.abort = 0;
        sh.inexact = 0;
        sh.xsplit = 0;
        sh.prod_last = -1;
        sh.mma_tile = -1;
        sh.mma_job = -1;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&sh.tmem_base)),
                     "n"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }

    // Epilogue thread <-> (row, column half): TMEM lane quarter = warp % 4
    // (the quarter a warp may access), accumulator acc, half of the columns.
    const int acc = ((warp - 2) >> 2) & 1;
    const int half = (warp - 2) >> 3;
    const int rr = 32 * (warp & 3) + lane;
    const int64_t m = m0 + 128 * acc + rr;
    const int crow = 128 * acc + rr;
    const bool epi = warp >= 2 && warp < 2 + TC_EPI_WARPS;
    if (epi) {
        // Stage the centred x tile as BF16 rows in shared memory: the TC_ROWS x
        // L tile is contiguous in X, so the epilogue threads read it as a flat
        // array (coalesced, eight 16-byte loads in flight per thread).
        constexpr int ST = 32 * TC_EPI_WARPS;                 // 512 staging threads
        const int et = tid - 64;
        const int64_t rows = M - m0 < TC_ROWS ? M - m0 : TC_ROWS;
        bool inexact = false, bad = false, split = false;
        const float *Xt = X + m0 * L;
        const int total = (int)rows * L;
        if ((L & 3) == 0 && (reinterpret_cast<uintptr_t>(Xt) & 15u) == 0) {
            const float4 *X4 = reinterpret_cast<const float4 *>(Xt);
            const int total4 = total >> 2;
            int i = et;
            for (; i + 7 * ST < total4; i += 8 * ST) {
                float4 q[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) q[u] = __ldg(X4 + i + u * ST);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int f = 4 * (i + u * ST);
                    tc_put_x<LK>(XS, XL, f, L, q[u].x, mu, bad, inexact, split);
                    tc_put_x<LK>(XS, XL, f + 1, L, q[u].y, mu, bad, inexact, split);
                    tc_put_x<LK>(XS, XL, f + 2, L, q[u].z, mu, bad, inexact, split);
                    tc_put_x<LK>(XS, XL, f + 3, L, q[u].w, mu, bad, inexact, split);
                }
            }
            for (; i < total4; i += ST) {
                const float4 q = __ldg(X4 + i);
                tc_put_x<LK>(XS, XL, 4 * i, L, q.x, mu, bad, inexact, split);
                tc_put_x<LK>(XS, XL, 4 * i + 1, L, q.y, mu, bad, inexact, split);
                tc_put_x<LK>(XS, XL, 4 * i + 2, L, q.z, mu, bad, inexact, split);
                tc_put_x<LK>(XS, XL, 4 * i + 3, L, q.w, mu, bad, inexact, split);
            }
        } else {
            for (int i = et; i < total; i += ST)
                tc_put_x<LK>(XS, XL, i, L, __ldg(Xt + i), mu, bad, inexact, split);
        }
        if (bad) flag_error(st, ERR_NONFINITE);
        if (inexact) sh.inexact = 1;
        if (split) sh.xsplit = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem_base;
    // codebook state written by the preparation kernel (constant here)
    const bool tc_exact_cb = st->tc_inexact == 0;
    const float cmax = __uint_as_float(st->cmax_bits);
    const float rho = __uint_as_float(st->rho_bits);

    float xn2 = 0.f;
    const bool xsplit = sh.xsplit != 0;
    if (epi)
        xn2 = L == LK ? tc_write_a<LK, true>(XS, XL, L, m < M, crow, half, acc, warp, tmem, sh)
                      : tc_write_a<LK, false>(XS, XL, L, m < M, crow, half, acc, warp, tmem, sh);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0) {
        // ---------------- producer
        if (lane == 0) {
            for (int t = 0; t < ntiles; ++t) {
                const int s = t % TC_STAGES;
                if (t >= TC_STAGES && !mbar_wait_bounded_sleep(&sh.empty[s], (uint32_t)((t / TC_STAGES) - 1) & 1u)) {
                    sh.abort = 1;
                    break;
                }
                if (sh.abort) break;
                mbar_expect_tx(&sh.full[s], stage_bytes);
                bulk_load(Bs + s * stage_bytes,
                          reinterpret_cast<const uint8_t *>(Bp) + (size_t)t * stage_bytes, stage_bytes,
                          &sh.full[s]);
                sh.prod_last = t;
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: job j = 2 t + a (tile t, accumulator a)
        // goes to slot j % 3 of the ring.  The issue of an MMA returns about
        // when the tensor pipe takes it, so the issuer's own instructions sit
        // on the tensor pipe's critical path: the whole warp runs the loop
        // (warp-uniform addresses; waits suspend instead of spinning) and one
        // elected lane issues each MMA and commit.
        const uint64_t bdesc0 = smem_desc(smem_addr(Bs), 128u, sbo_b);
        bool ok = true;
        for (int t = 0; t < ntiles && ok; ++t) {
            const int s = t % TC_STAGES;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded_sleep(&sh.full[s], (uint32_t)(t / TC_STAGES) & 1u))) {
                ok = false;
                break;
            }
            // Descriptors differ only in their start-address field: add the
            // byte offset / 16 to the base descriptor (addresses < 256 KB, no carry).
            const uint64_t bst = bdesc0 + ((uint64_t)(s * stage_bytes) >> 4);
#pragma unroll
            for (int a = 0; a < TC_NACC; ++a) {
                const int j = 2 * t + a, slot = j % TC_SLOTS;
                if ((j >= TC_SLOTS &&
                     !__all_sync(0xffffffffu, mbar_wait_bounded_sleep(&sh.tempty[slot], (uint32_t)((j / TC_SLOTS) - 1) & 1u))) ||
                    sh.abort) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(slot * TC_NT);
                const uint32_t at = tmem + (uint32_t)(TC_A_COL + a * TcA<LK>::COLS);
                mma_job_elect<LK>(d, at, bst, xsplit);
                mma_commit_elect(&sh.tfull[slot]);
                if (lane == 0) sh.mma_job = j;
            }
            if (!ok) break;
            mma_commit_elect(&sh.empty[s]);
            if (lane == 0) sh.mma_tile = t;
        }
        if (!ok && lane == 0) sh.abort = 1;
        __syncwarp();
    } else if (epi) {
        // ---------------- epilogue: one (row, column half) per thread
        float V1, V2;
        int i1;
        tc_jobs<GRP>(sh, tmem, warp, lane, acc, half, ntiles, 0, keymask, V1, V2, i1);
        tc_tail<LK, GRP>(sh, warp, lane, acc, half, rr, m0, X, M, L, N, C, kn, xn2, !sh.inexact && tc_exact_cb,
                         xsplit, cmax, rho, V1, V2, i1, st, assign, e, flags, flag_base);
    }

    tc_fence_before();
    __syncthreads();
    if (sh.abort) {
        // Stop: wait (bounded) for the bulk copies nobody consumed and for the
        // last committed MMAs, then free TMEM below.
        if (tid == 0) {
            for (int t = sh.mma_tile + 1; t <= sh.prod_last; ++t)
                (void)mbar_wait_bounded(&sh.full[t % TC_STAGES], (uint32_t)(t / TC_STAGES) & 1u);
            if (sh.mma_job >= 0)
                (void)mbar_wait_bounded(&sh.tfull[sh.mma_job % TC_SLOTS], (uint32_t)(sh.mma_job / TC_SLOTS) & 1u);
            flag_error(st, ERR_TIMEOUT);
        }
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TC_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------- persistent
// One CTA per SM loops over the row tiles blockIdx.x, + gridDim.x, ...  The
// producer also streams each next x tile (one TMA bulk copy of its TC_ROWS x L
// floats) into a shared FP32 buffer while the current tile's MMAs run; at a
// tile boundary the epilogue warps convert it (centring, exactness checks) and
// write the next A operand into tensor memory as soon as the previous tile's
// MMAs are done (they have consumed its last jobs), and only then finish the
// previous tile (merge, exact group distances, certificate), so the tensor pipe
// starts the next tile while that tail runs.  Codebook tiles stream through
// a 2-stage ring (a third stage fits but measured no faster: the copies are
// limited by the SM's bandwidth from L2, not by their latency); job and tile
// counters run across row tiles, so the barriers' phases continue.
// Needs L % 4 == 0 and a 16-byte aligned X (the launcher checks).
constexpr int TC_PSTAGES = 2;

template <int LK, int GRP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_assign_tc_p(const float *__restrict__ X, int64_t M, int L,
                  const __nv_bfloat16 *__restrict__ Bp, const float *__restrict__ kn,
                  const int32_t *n_dev, int n_host, const float *__restrict__ mu,
                  const float *__restrict__ C, DevState *st, int32_t *__restrict__ assign,
                  float *__restrict__ e, int32_t *__restrict__ flags, int keymask,
                  int64_t flag_base, int n_lo, int n_hi)
{
    if (st->finished) return;
    const int N = cur_n(n_dev, n_host);
    if (N < n_lo || N >= n_hi || N <= st->direct_max) return;   // another kernel serves this size
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ TcSmem sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (N + TC_NT - 1) / TC_NT;
    const int64_t nrt = (M + TC_ROWS - 1) / TC_ROWS;   // row tiles
    const int K = (int)((nrt - (int64_t)blockIdx.x + gridDim.x - 1) / gridDim.x);   // this CTA's
    constexpr int KB = tc_kb(LK);
    constexpr int XSTR = XsRow<LK>::STR;
    constexpr uint32_t sbo_b = (uint32_t)(KB / 8) * 128u;
    constexpr uint32_t stage_bytes = (uint32_t)TC_NT * KB * 2u;
    constexpr uint32_t xs_bytes = (uint32_t)TC_ROWS * XSTR * 2u;
    constexpr uint32_t xl_bytes = TcA<LK>::SPLIT ? xs_bytes : 0u;   // x_lo rows (split form)
    uint8_t *Bs = smem;
    __nv_bfloat16 *XS = reinterpret_cast<__nv_bfloat16 *>(smem + TC_PSTAGES * stage_bytes);
    __nv_bfloat16 *XL = reinterpret_cast<__nv_bfloat16 *>(smem + TC_PSTAGES * stage_bytes + xs_bytes);
    float *XF = reinterpret_cast<float *>(smem + TC_PSTAGES * stage_bytes + xs_bytes + xl_bytes);
    auto tile_m0 = [&](int k) -> int64_t {
        return ((int64_t)blockIdx.x + (int64_t)k * gridDim.x) * TC_ROWS;
    };
    auto tile_rows = [&](int k) -> int64_t {
        const int64_t r = M - tile_m0(k);
        return r < TC_ROWS ? r : TC_ROWS;
    };

    if (tid == 0) {
        for (int s = 0; s < TC_PSTAGES; ++s) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], 1);
        }
        for (int b = 0; b < TC_SLOTS; ++b) {
            mbar_init(&sh.tfull[b], 1);
            mbar_init(&sh.tempty[b], TC_EPI_WARPS / TC_NACC);
        }
        mbar_init(&sh.xfull, 1);
        mbar_init(&sh.xempty, 1);
        mbar_init(&sh.aready, 1);
        fence_mbar_init();
        sh.abort = 0;
        sh.prod_last = -1;
        sh.mma_tile = -1;
        sh.mma_job = -1;
        sh.x_issued = -1;
        sh.x_done = -1;
        sh.xsplit2[0] = sh.xsplit2[1] = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&sh.tmem_base)),
                     "n"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem_base;
    const bool tc_exact_cb = st->tc_inexact == 0;
    const float cmax = __uint_as_float(st->cmax_bits);
    const float rho = __uint_as_float(st->rho_bits);
    const int acc = ((warp - 2) >> 2) & 1;
    const int half = (warp - 2) >> 3;
    const int rr = 32 * (warp & 3) + lane;
    const int crow = 128 * acc + rr;
    const bool epi = warp >= 2 && warp < 2 + TC_EPI_WARPS;

    if (warp == 0) {
        // ---------------- producer: x tiles and codebook tiles
        if (lane == 0 && K > 0) {
            // x tile kx into XF once x tile kx - 1 has been converted; never after
            // a time-out (sh.x_issued counts the copies for the drain below)
            auto load_x = [&](int kx) -> bool {
                if (kx < 1 || kx >= K || kx <= sh.x_issued) return true;
                if (!mbar_wait_bounded_sleep(&sh.xempty, (uint32_t)(kx - 1) & 1u) || sh.abort) {
                    sh.abort = 1;
                    return false;
                }
                const uint32_t bytes = (uint32_t)(tile_rows(kx) * L * 4);
                mbar_expect_tx(&sh.xfull, bytes);
                bulk_load(XF, X + tile_m0(kx) * L, bytes, &sh.xfull);
                sh.x_issued = kx;
                return true;
            };
            {   // x tile 0
                const uint32_t bytes = (uint32_t)(tile_rows(0) * L * 4);
                mbar_expect_tx(&sh.xfull, bytes);
                bulk_load(XF, X + tile_m0(0) * L, bytes, &sh.xfull);
                sh.x_issued = 0;
            }
            for (int k = 0; k < K && !sh.abort; ++k) {
                for (int t = 0; t < ntiles; ++t) {
                    const int G = k * ntiles + t, s = G % TC_PSTAGES;
                    if (G >= TC_PSTAGES &&
                        !mbar_wait_bounded_sleep(&sh.empty[s], (uint32_t)((G / TC_PSTAGES) - 1) & 1u)) {
                        sh.abort = 1;
                        break;
                    }
                    if (sh.abort) break;
                    mbar_expect_tx(&sh.full[s], stage_bytes);
                    bulk_load(Bs + s * stage_bytes,
                              reinterpret_cast<const uint8_t *>(Bp) + (size_t)t * stage_bytes, stage_bytes,
                              &sh.full[s]);
                    sh.prod_last = G;
                    // x tile k + 1 as soon as x tile k has been converted (at tile k's
                    // boundary); it lands during tile k's MMAs
                    if (t == 0 && !load_x(k + 1)) break;
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (as in k_assign_tc), per row tile after
        // its A operand is in tensor memory
        const uint64_t bdesc0 = smem_desc(smem_addr(Bs), 128u, sbo_b);
        // L = 64 with two pieces: a job is one instruction sequence (job9_elect)
        constexpr bool JOB9 = LK == 64 && TC_PIECES == 2;
        bool ok = true;
        // job j: accumulator slot j % 3 and the parity of j / 3; codebook tile G: stage
        // G % TC_PSTAGES and the parity of G / TC_PSTAGES, all stepped (no divisions);
        // the last committed job and tile are published once, at the end
        int j = 0, slot = 0, G = 0, s = 0, last_job = -1, last_tile = -1;
        uint32_t jpar = 0u, gpar = 0u;
        for (int k = 0; k < K && ok; ++k) {
            if (!__all_sync(0xffffffffu, mbar_wait_bounded_sleep(&sh.aready, (uint32_t)k & 1u)) || sh.abort) {
                ok = false;
                break;
            }
            const bool xsp = sh.xsplit2[k & 1] != 0;   // published before aready
            for (int t = 0; t < ntiles && ok; ++t) {
                if (!__all_sync(0xffffffffu, mbar_wait_bounded_sleep(&sh.full[s], gpar))) {
                    ok = false;
                    break;
                }
                const uint64_t bst = bdesc0 + ((uint64_t)(s * stage_bytes) >> 4);
#pragma unroll
                for (int a = 0; a < TC_NACC; ++a) {
                    if ((j >= TC_SLOTS && !__all_sync(0xffffffffu, mbar_wait_bounded_sleep(&sh.tempty[slot], jpar ^ 1u))) ||
                        sh.abort) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(slot * TC_NT);
                    if (JOB9) {
                        job9_elect(d, tmem + (uint32_t)(TC_A_COL + a * TcA<LK>::COLS), bst,
                                   smem_addr(&sh.tfull[slot]));
                    } else {
                        mma_job_elect<LK>(d, tmem + (uint32_t)(TC_A_COL + a * TcA<LK>::COLS), bst, xsp);
                        mma_commit_elect(&sh.tfull[slot]);
                    }
                    last_job = j++;
                    if (++slot == TC_SLOTS) {
                        slot = 0;
                        jpar ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit_elect(&sh.empty[s]);
                last_tile = G++;
                if (++s == TC_PSTAGES) {
                    s = 0;
                    gpar ^= 1u;
                }
            }
        }
        if (lane == 0) {
            sh.mma_job = last_job;
            sh.mma_tile = last_tile;
        }
        if (!ok && lane == 0) sh.abort = 1;
        __syncwarp();
    } else if (epi) {
        // ---------------- epilogue warps.  Every warp passes the same named
        // barriers in the same order for every k, also after a time-out (work
        // is skipped, barriers are not).
        constexpr int ST = 32 * TC_EPI_WARPS;
        constexpr int NCHUNK = 1;   // the x tile is converted in one piece at the boundary
        const int et = tid - 64;
        float pV1 = INFINITY, pV2 = INFINITY, pxn2 = 0.f;
        int pi1 = -1;
        bool pusable = false, next_exact = false, next_split = false, psplit = false;
        bool cv_bad = false, cv_inexact = false, cv_split = false;
        // Convert piece c (of NCHUNK) of x tile kk from XF into centred BF16
        // rows in XS; the last piece publishes the tile's exactness and frees XF.
        auto convert = [&](int kk, int c) {
            if (c == 0) {
                cv_bad = false;
                cv_inexact = false;
                cv_split = false;
                if (!sh.abort) {
                    if (!mbar_wait_bounded_sleep(&sh.xfull, (uint32_t)kk & 1u)) sh.abort = 1;
                    else if (tid == 64) sh.x_done = kk;   // xfull phases observed: 0 .. kk
                }
            }
            if (!sh.abort) {
                const int total4 = (int)(tile_rows(kk) * L) >> 2;
                const int per = (total4 + NCHUNK - 1) / NCHUNK;
                const int lo = c * per, hi = min(total4, lo + per);
                const float4 *X4 = reinterpret_cast<const float4 *>(XF);
                if ((4 * ST) % L == 0) {
                    // L divides 4 ST: a thread's four columns are the same in every
                    // round, so mu is read once and rows advance by 4 ST / L
                    const int i0 = lo + et;
                    const int l0 = (4 * i0) % L, dr = 4 * ST / L;
                    const float4 m4 = make_float4(__ldg(mu + l0), __ldg(mu + l0 + 1), __ldg(mu + l0 + 2),
                                                  __ldg(mu + l0 + 3));
                    int r = (4 * i0) / L;
                    for (int i = i0; i < hi; i += ST, r += dr) {
                        const float4 q = X4[i];
                        const float xv[4] = {q.x, q.y, q.z, q.w};
                        const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
                        uint32_t bits[4], lbits[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            cv_bad = cv_bad || !isfinite(xv[u]);
                            const float v = __fsub_rn(xv[u], mv[u]);
                            const __nv_bfloat16 b = __float2bfloat16_rn(v);
                            if constexpr (TcA<LK>::SPLIT) {
                                const __nv_bfloat16 lo = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(b)));
                                cv_split = cv_split || __bfloat162float(lo) != 0.f;
                                lbits[u] = __bfloat16_as_ushort(lo);
                            } else {
                                const float bb = __fsub_rn(v, xv[u]);
                                const float err =
                                    __fadd_rn(__fsub_rn(xv[u], __fsub_rn(v, bb)), __fsub_rn(-mv[u], bb));
                                cv_inexact = cv_inexact || err != 0.f || (__bfloat162float(b) != v);
                                lbits[u] = 0u;
                            }
                            bits[u] = __bfloat16_as_ushort(b);
                        }
                        *reinterpret_cast<uint2 *>(XS + xs_at<LK>(r, l0)) =
                            make_uint2(bits[0] | (bits[1] << 16), bits[2] | (bits[3] << 16));
                        if (TcA<LK>::SPLIT)
                            *reinterpret_cast<uint2 *>(XL + xs_at<LK>(r, l0)) =
                                make_uint2(lbits[0] | (lbits[1] << 16), lbits[2] | (lbits[3] << 16));
                    }
                } else {
                    for (int i = lo + et; i < hi; i += ST) {
                        const float4 q = X4[i];
                        tc_put_x<LK>(XS, XL, 4 * i, L, q.x, mu, cv_bad, cv_inexact, cv_split);
                        tc_put_x<LK>(XS, XL, 4 * i + 1, L, q.y, mu, cv_bad, cv_inexact, cv_split);
                        tc_put_x<LK>(XS, XL, 4 * i + 2, L, q.z, mu, cv_bad, cv_inexact, cv_split);
                        tc_put_x<LK>(XS, XL, 4 * i + 3, L, q.w, mu, cv_bad, cv_inexact, cv_split);
                    }
                }
            }
            if (c == NCHUNK - 1) {
                if (cv_bad) flag_error(st, ERR_NONFINITE);
                next_exact = !named_sync_or(1, 32 * TC_EPI_WARPS, cv_inexact);
                next_split = TcA<LK>::SPLIT && named_sync_or(1, 32 * TC_EPI_WARPS, cv_split);
                if (tid == 64 && !sh.abort) mbar_arrive(&sh.xempty);   // XF may take the next x tile
            }
        };
        for (int k = 0; k <= K; ++k) {
            float xn2 = 0.f;
            bool tile_exact = false, tile_split = false;
            if (k < K) {
                // convert x tile k (it is in XF) into centred BF16 rows; then, all 16
                // warps having consumed the previous tile's last jobs (before the
                // conversion's named barrier), its MMAs are done and A may be rewritten
                for (int c = 0; c < NCHUNK; ++c) convert(k, c);
                tile_exact = next_exact;
                tile_split = next_split;
                xn2 = L == LK ? tc_write_a<LK, true>(XS, XL, L, tile_m0(k) + crow < M, crow, half, acc, warp, tmem, sh)
                              : tc_write_a<LK, false>(XS, XL, L, tile_m0(k) + crow < M, crow, half, acc, warp, tmem, sh);
                tc_fence_before();
                named_sync(1, 32 * TC_EPI_WARPS);
                if (tid == 64) {
                    sh.xsplit2[k & 1] = tile_split ? 1 : 0;   // read by the MMA issuer after aready
                    mbar_arrive(&sh.aready);
                }
            }
            // the previous tile's tail runs while the tensor pipe starts on this one
            if (k >= 1)
                tc_tail<LK, GRP>(sh, warp, lane, acc, half, rr, tile_m0(k - 1), X, M, L, N, C, kn, pxn2, pusable,
                                 psplit, cmax, rho, pV1, pV2, pi1, st, assign, e, flags, flag_base);
            if (k < K) {
                tc_jobs<GRP>(sh, tmem, warp, lane, acc, half, ntiles, 2 * k * ntiles, keymask, pV1, pV2, pi1);
                pxn2 = xn2;
                pusable = tile_exact && tc_exact_cb;
                psplit = tile_split;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (sh.abort) {
        // Stop: wait (bounded) for the copies nobody consumed and for the last
        // committed MMAs, then free TMEM below.
        if (tid == 0) {
            for (int G = sh.mma_tile + 1; G <= sh.prod_last; ++G)
                (void)mbar_wait_bounded(&sh.full[G % TC_PSTAGES], (uint32_t)(G / TC_PSTAGES) & 1u);
            // x copies are issued in tile order and complete xfull's phases in
            // that order: wait for every issued copy past the last phase observed
            for (int k = sh.x_done + 1; k <= sh.x_issued; ++k)
                (void)mbar_wait_bounded(&sh.xfull, (uint32_t)k & 1u);
            if (sh.mma_job >= 0)
                (void)mbar_wait_bounded(&sh.tfull[sh.mma_job % TC_SLOTS], (uint32_t)(sh.mma_job / TC_SLOTS) & 1u);
            flag_error(st, ERR_TIMEOUT);
        }
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TC_TMEM_COLS)
                     : "memory");
    }
}

__global__ void k_round_mu(float *mu, int L)
{
    const int l = threadIdx.x;
    if (l < L) mu[l] = rintf(mu[l]);
}

}  // namespace

size_t tc_codebook_bytes(int NP, int L) { return (size_t)tc_prep_rows(NP) * tc_kb(round_up(L, 16)) * 2; }

bool tc_supported(int L) { return L >= 1 && L <= TC_LMAX; }

void launch_round_mu(float *mu, int L, cudaStream_t s) { LBG_COUNTED k_round_mu<<<1, 128, 0, s>>>(mu, L); }

void launch_prep_tc(const float *C, int N_alloc, const int32_t *n_dev, int n_host, int L,
                    const float *mu, void *Bp, float *kn, float *CT, DevState *st, cudaStream_t s)
{
    const int blocks = tc_prep_rows(N_alloc) / PT_N;
    __nv_bfloat16 *B = static_cast<__nv_bfloat16 *>(Bp);
    const int Lp = round_up(L, 4);
    switch (round_up(L, 16)) {
    case 16: LBG_COUNTED k_prep_tc<16><<<blocks, 256, 0, s>>>(C, n_dev, n_host, L, Lp, mu, B, kn, CT, st); break;
    case 32: LBG_COUNTED k_prep_tc<32><<<blocks, 256, 0, s>>>(C, n_dev, n_host, L, Lp, mu, B, kn, CT, st); break;
    case 48: LBG_COUNTED k_prep_tc<48><<<blocks, 256, 0, s>>>(C, n_dev, n_host, L, Lp, mu, B, kn, CT, st); break;
    default: LBG_COUNTED k_prep_tc<64><<<blocks, 256, 0, s>>>(C, n_dev, n_host, L, Lp, mu, B, kn, CT, st); break;
    }
}

// Group size of the epilogue by codebook size: larger groups cut the per-value
// epilogue work and the flagged rows, smaller ones the tail's exact distances
// per row.  Measured on GB300 (search + exact re-scoring, ms): image blocks
// L = 64, N = 4096: G = 2 0.491, 4 0.474, 8 0.519; N = 2048: 0.312, 0.308,
// 0.368; N = 1024: 0.206, 0.216, 0.276; L = 16, N = 4096: 3.36, 2.83, 2.99;
// N = 1024: 1.206, 1.165, 1.564; mixture L = 32, N = 4096: 0.324, 0.257, 0.257;
// N = 512: 0.077, 0.077, 0.105.
template <int LK>
struct TcGroups {
    static constexpr int SMALL = 2, LARGE = 4, AT = LK <= 32 ? 1024 : 2048;
};

template <int LK, int GRP>
static void launch_tc_g(const float *X, int64_t M, int L, const __nv_bfloat16 *B, const float *kn,
                        const int32_t *n_dev, int n_host, const float *mu, const float *C, DevState *st,
                        int32_t *assign, float *e, int32_t *flags, cudaStream_t s, int64_t m_lo, int64_t grid,
                        int n_lo, int n_hi)
{
    const int keymask = ~((1 << GrpCfg<GRP>::JBITS) - 1);
    if ((L & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0) {
        // persistent: 2 codebook stages + staged BF16 rows + the FP32 x tile
        const size_t need = (size_t)TC_PSTAGES * TC_NT * tc_kb(LK) * 2 +
                            (size_t)(TcA<LK>::SPLIT ? 2 : 1) * TC_ROWS * XsRow<LK>::STR * 2 + (size_t)TC_ROWS * LK * 4;
        // at least 120 KB so that a single CTA (and its 512 TMEM columns) owns the SM
        const size_t smem = need > 120 * 1024 ? need : 120 * 1024;
        cudaFuncSetAttribute(k_assign_tc_p<LK, GRP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int64_t g = grid < num_sms() ? grid : num_sms();
        LBG_COUNTED k_assign_tc_p<LK, GRP><<<(unsigned)g, TC_THREADS, smem, s>>>(
            X, M, L, B, kn, n_dev, n_host, mu, C, st, assign, e, flags, keymask, m_lo, n_lo, n_hi);
        return;
    }
    const size_t need = (size_t)(TcA<LK>::SPLIT ? 2 : 1) * TC_ROWS * XsRow<LK>::STR * 2 +
                        (size_t)TC_STAGES * TC_NT * tc_kb(LK) * 2;
    // at least 120 KB so that a single CTA (and its 512 TMEM columns) owns the SM
    const size_t smem = need > 120 * 1024 ? need : 120 * 1024;
    cudaFuncSetAttribute(k_assign_tc<LK, GRP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LBG_COUNTED k_assign_tc<LK, GRP><<<(unsigned)grid, TC_THREADS, smem, s>>>(
        X, M, L, B, kn, n_dev, n_host, mu, C, st, assign, e, flags, keymask, m_lo, n_lo, n_hi);
}

template <int LK>
static void launch_tc(const float *X, int64_t M, int L, const void *Bp, const float *kn,
                      const int32_t *n_dev, int n_host, const float *mu, const float *C, DevState *st,
                      int32_t *assign, float *e, int32_t *flags, cudaStream_t s, int64_t m_lo, int grp)
{
    // rows [m_lo, M): the kernels see them as rows [0, M - m_lo) of offset arrays and add
    // m_lo back only to the flag list entries (global row numbers)
    X += m_lo * L;
    assign += m_lo;
    e += m_lo;
    M -= m_lo;
    const int64_t grid = (M + TC_ROWS - 1) / TC_ROWS;
    if (grid <= 0) return;
    const __nv_bfloat16 *B = static_cast<const __nv_bfloat16 *>(Bp);
    auto go = [&](int G, int n_lo, int n_hi) {
        if (G == 8)
            launch_tc_g<LK, 8>(X, M, L, B, kn, n_dev, n_host, mu, C, st, assign, e, flags, s, m_lo, grid, n_lo, n_hi);
        else if (G == 4)
            launch_tc_g<LK, 4>(X, M, L, B, kn, n_dev, n_host, mu, C, st, assign, e, flags, s, m_lo, grid, n_lo, n_hi);
        else
            launch_tc_g<LK, 2>(X, M, L, B, kn, n_dev, n_host, mu, C, st, assign, e, flags, s, m_lo, grid, n_lo, n_hi);
    };
    if (grp) {   // forced
        go(grp, 0, 1 << 30);
        return;
    }
    // by size: TcGroups<LK>::SMALL below AT codevectors, LARGE from there on
    constexpr int small = TcGroups<LK>::SMALL, large = TcGroups<LK>::LARGE, at = TcGroups<LK>::AT;
    if (small == large || !n_dev) {   // one kernel; the size is known here, or both agree
        go(n_host >= at ? large : small, 0, 1 << 30);
    } else {   // training: the stage size is on the device, each kernel takes its range
        go(small, 0, at);
        if (n_host >= at) go(large, at, 1 << 30);
    }
}

void launch_assign_tc(const float *X, int64_t M, int L, const void *Bp, const float *kn,
                      const int32_t *n_dev, int n_host, const float *mu, const float *C,
                      DevState *st, int32_t *assign, float *e, int32_t *flags, cudaStream_t s,
                      int64_t m_lo, int grp)
{
    switch (round_up(L, 16)) {
    case 16: launch_tc<16>(X, M, L, Bp, kn, n_dev, n_host, mu, C, st, assign, e, flags, s, m_lo, grp); break;
    case 32: launch_tc<32>(X, M, L, Bp, kn, n_dev, n_host, mu, C, st, assign, e, flags, s, m_lo, grp); break;
    case 48: launch_tc<48>(X, M, L, Bp, kn, n_dev, n_host, mu, C, st, assign, e, flags, s, m_lo, grp); break;
    default: launch_tc<64>(X, M, L, Bp, kn, n_dev, n_host, mu, C, st, assign, e, flags, s, m_lo, grp); break;
    }
}

}  // namespace lbg
