// lbg_internal.cuh -- device state, tile constants and PTX helpers shared by
// the kernels of the LBG library (internal; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbg {

// Nearest-codevector tile: a CTA owns BM training rows and streams the
// codebook through shared memory in chunks of BN codevectors.
constexpr int BM = 128;
constexpr int BN = 128;
constexpr int ASSIGN_THREADS = 256;
constexpr int LMAX = 128;     // = LBG_MAX_DIM
constexpr int NMAX = 8192;    // = LBG_MAX_CODEBOOK

// Cell-table build: rows are cut into at most HIST_CHUNKS_MAX contiguous
// chunks (one CTA each); the segmented centroid sums cut the cell-sorted
// row order into pieces of SEG rows (one warp each).
constexpr int HIST_CHUNKS_MAX = 304;   // cap; plans use min(this, 2 x SMs)
// The exact re-scoring kernel stages the original codebook in chunks of
// EXACT_SW codevectors, stored k-major inside a chunk.
constexpr int EXACT_SW = 128;
constexpr int HIST_THREADS = 256;

// Error bits in DevState::err.
constexpr uint32_t ERR_NONFINITE = 1u;
constexpr uint32_t ERR_TIMEOUT = 2u;
constexpr uint32_t ERR_INTERNAL = 4u;

// Pass modes of the control kernel.
constexpr int MODE_STEP = 0;    // lbg_lloyd_step / vq_encode: no stop test
constexpr int MODE_TRAIN = 1;   // lbg_train: stop test, split, finish

constexpr int ACT_UPDATE = 0, ACT_SPLIT = 1, ACT_FINISH = 2, ACT_NONE = 3;

// Device-resident state of one call.  lbg_train keeps the whole stage/pass
// control here so that passes can be issued without host round trips.
struct DevState {
    int32_t n_cur;        // codebook size of the current stage
    int32_t pass;         // pass index within the stage
    int32_t total;        // passes run so far
    int32_t action;       // decision of the last stop test (ACT_*)
    int32_t finished;     // 1 once training has ended (all kernels then no-op)
    int32_t warn;         // 1 if some stage was cut at max_passes
    int32_t nflag;        // rows flagged for exact re-scoring in this pass
    int32_t n_exact_last; // nflag of the last pass (for step / encode reports)
    int32_t tc_inexact;   // 1 if a BF16 codebook did not split exactly (tensor-core path)
    uint32_t err;         // ERR_* bits
    uint32_t cmax_bits;   // bits of max_n ||c_n - mu|| (non-negative float)
    uint32_t rho_bits;    // bits of max_n ||c'_n - (its BF16 pieces)|| (tensor-core path)
    uint32_t done_ctr;    // CTAs done in a fused kernel (its last CTA finishes and resets it)
    double D;             // total distortion of the last pass
    double D_prev;        // distortion of the previous pass of the stage
    uint64_t t_pass0;     // %globaltimer at the start of the traced pass (lbg_train trace)
    int32_t trace_on;     // 1 while a traced pass of lbg_train is in progress
    int32_t direct_max;   // stages of at most this many cells take k_assign_direct (lbg_train; 0: none)
};

// Device pass record (mirrors lbg_pass_record).
struct PassRecord {
    int32_t stage_n, pass, action, n_exact;
    double D;
    int32_t n_empty;      // cells with no row in the pass's allocation
    float ms;             // device time of the pass (%globaltimer)
};

// One problem of a batched call (device-resident descriptor; every pointer
// is that problem's own region of the batched workspace).
struct BatchSet {
    const float *X;        // [M x L] rows of this problem
    int64_t M;
    int N;                 // final codebook size (allocated cells)
    int NP;                // N rounded up to BN
    int CH;                // histogram / scatter chunks
    int G;                 // blocks of the initial mean
    int64_t R;             // rows per chunk
    int64_t S;             // rows per segmented-sum piece
    float *C, *Calt;       // [N x L] current codebook, split scratch
    float *Cp, *kn, *CT;   // prepared codebook
    float *mu;             // [Lp] centring vector
    DevState *st;
    int32_t *assign, *flags, *table, *counts, *off, *perm;
    int32_t *qcell, *cell_done;   // piece cells and per-cell piece counters (persistent pass)
    int64_t nq;                   // warp pieces of the cell sums
    float *e, *pieces;
    double *dpart, *mpart;
};

// Prefix arrays (device, S + 1 entries each) mapping the blocks of a batched
// launch to problems: block b belongs to problem s with pre[s] <= b < pre[s+1].
struct BatchMaps {
    const int32_t *hist, *scan, *prep, *cellsum, *combine, *split, *copy, *mean, *exact_unused;
    const int64_t *tiles;  // assign work items: row tiles of BM rows
};

__host__ __device__ inline int find_set(const int32_t *pre, int S, int64_t b)
{
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)pre[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__host__ __device__ inline int find_set64(const int64_t *pre, int S, int64_t b)
{
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Codebook size of a launch: the stage size on the device (training) or the host's.
__device__ __forceinline__ int cur_n(const int32_t *n_dev, int n_host) { return n_dev ? *n_dev : n_host; }

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ inline int64_t round_up64(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared through the TMA unit, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Same test with a suspend-time hint: a waiting thread sleeps (instead of
// spinning and taking issue slots) until the phase completes or ~hint_ns pass.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`, giving up after ~2 s of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 0u && global_ns() - t0 > 2000000000ull) return false;
    }
}

// Bounded wait that sleeps between tests (for waits expected to be long).
__device__ __forceinline__ bool mbar_wait_bounded_sleep(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait_sleep(bar, parity, 100000u)) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
}

__device__ __forceinline__ void flag_error(DevState *st, uint32_t bits) { atomicOr(&st->err, bits); }

// ------------------------------------------------------------ host helpers
// Kernel launches issued by the library, a diagnostic count read through
// lbg_launch_count(); a replayed CUDA graph adds the kernels it holds.  Every
// launch site is written `LBG_COUNTED kernel<<<...>>>(...)`.
void note_launch();
#define LBG_COUNTED ::lbg::note_launch(),
// Multiprocessor count of the current device (queried once per device).
int num_sms();

// ------------------------------------------------------------ launchers
// Codebook preparation (k_assign.cu).
void launch_codebook_mean(const float *C, int N, int L, float *mu, cudaStream_t s);
// mean (rounded to integers if round_mu) and, if st, the initial DevState of a
// step / encode with N codevectors, in one launch.
void launch_begin(const float *C, int N, int L, float *mu, bool round_mu, DevState *st, cudaStream_t s);
void launch_prep(const float *C, int N_alloc, const int32_t *n_dev, int n_host, int L, int Lp,
                 const float *mu, float *Cp, float *kn, float *CT, int NP, DevState *st,
                 cudaStream_t s);
// Nearest codevector of rows [m_lo, M) of X (row indices, assign, e and flags
// stay global).  expire != 0 (test hook): every CTA's first bounded wait gives
// up at once (the time-out path: drain, report LBG_ERR_TIMEOUT, no row written).
void launch_assign(const float *X, int64_t M, int L, int Lp, const float *Cp, const float *kn,
                   const int32_t *n_dev, int n_host, const float *mu, const float *C, DevState *st,
                   int32_t *assign, float *e, int32_t *flags, cudaStream_t s, int64_t m_lo = 0,
                   int expire = 0);
void launch_exact(const float *X, int L, int Lp, const float *CT, const int32_t *n_dev, int n_host,
                  DevState *st, const int32_t *flags, int32_t *assign, float *e, int64_t M,
                  cudaStream_t s);
// Exact re-scoring with the flagged rows' work spread over at most
// exact_split_ctas() CTAs: scratch of 2 x exact_split_ctas() x exact_split_rows()
// partial minima and exact_split_ctas() group counters, the counters zero on entry.
int exact_split_ctas();
int exact_split_rows();
void launch_exact_split(const float *X, int L, int Lp, const float *CT, const int32_t *n_dev, int n_host,
                        DevState *st, const int32_t *flags, int32_t *assign, float *e, float *part_d,
                        int32_t *part_i, int32_t *cnt, int64_t M, cudaStream_t s);
void launch_decode(const int32_t *assign, int64_t M, int L, const float *C, float *Xhat,
                   cudaStream_t s);

// Tensor-core (BF16 / tcgen05) nearest codevector (k_assign_tc.cu).
size_t tc_codebook_bytes(int NP, int L);
bool tc_supported(int L);
void launch_round_mu(float *mu, int L, cudaStream_t s);
void launch_prep_tc(const float *C, int N_alloc, const int32_t *n_dev, int n_host, int L,
                    const float *mu, void *Bp, float *kn, float *CT, DevState *st, cudaStream_t s);
// Every row against all N codevectors in the FP32 direct form (k_assign_direct,
// k_assign.cu): the kernel runs only when N <= st->direct_max, the search and
// preparation kernels only when N > st->direct_max.
bool direct_supported(int L, const void *X, const void *C);
void launch_assign_direct(const float *X, int64_t M, int L, const float *C, const int32_t *n_dev, int n_host,
                          DevState *st, int32_t *assign, float *e, cudaStream_t s);
void launch_assign_tc(const float *X, int64_t M, int L, const void *Bp, const float *kn,
                      const int32_t *n_dev, int n_host, const float *mu, const float *C,
                      DevState *st, int32_t *assign, float *e, int32_t *flags, cudaStream_t s, int64_t m_lo = 0,
                      int grp = 0);

// Cell table, distortion and centroid update (k_update.cu).
void launch_mean(const float *X, int64_t M, int L, double *part, int G, float *mu, float *C0,
                 DevState *st, cudaStream_t s);
void launch_hist(const int32_t *assign, const float *e, int64_t M, int64_t R, int CH,
                 const int32_t *n_dev, int n_host, bool do_hist, int32_t *table, double *dpart,
                 DevState *st, bool train, cudaStream_t s);
// Step / encode / backward forms (MODE_STEP, N on the host): k_hist + k_ctl and
// k_scan + k_offsets, each pair in one launch whose last CTA does the second part.
void launch_hist_ctl(const int32_t *assign, const float *e, int64_t M, int64_t R, int CH, int N,
                     bool do_hist, int32_t *table, double *dpart, DevState *st, cudaStream_t s);
void launch_scan_offsets(int32_t *table, int CH, int N, int32_t *counts, int32_t *off, DevState *st,
                         cudaStream_t s);
void launch_ctl(const double *dpart, int CH, DevState *st, int mode, double theta, int max_passes,
                int N_target, PassRecord *records, int max_records, cudaStream_t s);
void launch_scatter(const int32_t *assign, int64_t M, int64_t R, int CH, const int32_t *table,
                    const int32_t *off, const int32_t *n_dev, int n_host, int32_t *perm,
                    DevState *st, bool train, cudaStream_t s);
void launch_cellsum(const float *X, int64_t M, int L, const int32_t *perm, const int32_t *off,
                    const int32_t *n_dev, int n_host, int64_t S, float *pieces, DevState *st,
                    bool train, cudaStream_t s);
// Fused update of the step and training forms: k_scan + k_offsets in one
// launch that also builds qcell[q] (the cell of the first row of warp piece q),
// zeroes cell_done[N] and copies empty cells to C_out; then the cell sums with
// the centroid division folded in (the last piece of a cell combines it).
void launch_scan_offsets_q(int32_t *table, int CH, const int32_t *n_dev, int n_host, int32_t *counts,
                           int32_t *off, int32_t *qcell, int32_t *cell_done, int64_t S, int L,
                           const float *C_in, float *C_out, DevState *st, bool train, cudaStream_t s);
void launch_cellsum_c(const float *X, int64_t M, int L, const int32_t *perm, const int32_t *off,
                      const int32_t *qcell, const int32_t *n_dev, int n_host, int64_t S, float *pieces,
                      int32_t *cell_done, float *C_out, DevState *st, bool train, cudaStream_t s);
void launch_split(const float *C_cur, float *C_alt, int N_alloc, int L, double delta, bool mult,
                  DevState *st, cudaStream_t s);
void launch_reseed(const int32_t *off, const int32_t *n_dev, int n_host, int L, double delta,
                   float *C, DevState *st, bool train, cudaStream_t s);
// Batched problems (k_update.cu / k_assign.cu): one launch per step for all problems.
void launch_b_mean(const BatchSet *sets, int S, const int32_t *pre_mean, int total_blocks, int L,
                   cudaStream_t s);
void launch_b_hist(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int NMAXB,
                   cudaStream_t s);
void launch_b_ctl(const BatchSet *sets, int S, double theta, int max_passes, cudaStream_t s);
void launch_b_scan(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, cudaStream_t s);
void launch_b_offsets(const BatchSet *sets, int S, cudaStream_t s);
void launch_b_scatter(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int NMAXB,
                      cudaStream_t s);
void launch_b_cellsum(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int L,
                      bool vec, cudaStream_t s);
void launch_b_combine(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int L,
                      cudaStream_t s);
void launch_b_split(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int L,
                    double delta, bool mult, cudaStream_t s);
void launch_b_advance(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int L,
                      cudaStream_t s);
void launch_b_prep(const BatchSet *sets, int S, const int32_t *pre, int total_blocks, int L, int Lp,
                   cudaStream_t s);
// Persistent batched nearest-codevector launch over (problem, row tile) work
// items; tile_rows 64 or 128 (pre_tiles counts tiles of that height), grid =
// SMs x ctas_per_sm CTAs.
void launch_b_assign(const BatchSet *sets, int S, const int64_t *pre_tiles, int64_t total_tiles,
                     int L, int Lp, int *counter, int tile_rows, int ctas_per_sm, cudaStream_t s);
void launch_b_exact(const BatchSet *sets, int S, int L, int Lp, int max_ngroups, cudaStream_t s);
void launch_b_reset(const BatchSet *sets, int S, int *counter, cudaStream_t s);
// One Lloyd pass of every problem in one cooperative launch (k_batched.cu):
// the phases of the launches above, separated by bounded grid-wide barriers.
struct BatchPass {
    const BatchSet *sets;
    int S, L, Lp, NMAXB;
    const int32_t *pre_prep, *pre_hist, *pre_scan, *pre_cellsum, *pre_combine, *pre_split, *pre_copy;
    int32_t tot_prep, tot_hist, tot_scan, tot_cellsum, tot_combine, tot_split, tot_copy;
    const int64_t *pre_tiles;   // row tiles of 64 rows (each CTA runs two at a time)
    int64_t ntiles;
    int *counter;               // assignment work items taken
    unsigned *bar;              // [0] arrivals, [1] generation, [2] abort (zero before the first pass)
    double theta, delta;
    int max_passes, mult, vec;
    int direct_max;             // problems at stages of at most this many cells: every row against
                                // every codevector (direct_tile); 0: none
    size_t phase_smem;          // dynamic shared memory of the phases; the state tables follow
};
// Resident CTAs per SM the persistent pass can have (0: it does not fit) and its
// dynamic shared memory.
int batch_pass_fit(int S, int L, int NMAXB, size_t *phase_smem, size_t *smem);
// false if the cooperative launch was refused (then the per-phase launches run)
bool launch_b_pass(const BatchPass &a, int ctas_per_sm, size_t smem, cudaStream_t s);

// Backward at a fixed cell table; the upstream gradient is gD, or *gD_dev
// (device) when gD_dev is not null.
void launch_grad_x(const float *X, int64_t M, int L, const float *C, int N, const int32_t *assign,
                   float gD, const float *gD_dev, float *e, float *dX, DevState *st, cudaStream_t s);
void launch_combine_grad(const float *pieces, const int32_t *off, int N, int L, int64_t S,
                         const float *C, float gD, const float *gD_dev, float *dC, cudaStream_t s);
void launch_advance(const float *C_alt, float *C_cur, int N_alloc, int L, DevState *st,
                    cudaStream_t s);
// Pass trace of lbg_train: start (stamp, codebook of the pass) and end (cell
// table, empty cells and device time into the pass record).
void launch_trace_begin(DevState *st, const float *C, int N, int L, float *trace_C, int cap,
                        cudaStream_t s);
void launch_trace_end(DevState *st, const int32_t *assign, int64_t M, const int32_t *counts,
                      PassRecord *rec, int max_rec, int32_t *trace_A, int cap, cudaStream_t s);

}  // namespace lbg
