/*
 * lbgvq.h -- C ABI of the GB300 (sm_103a) LBG vector-quantizer library.
 *
 * The library designs a vector-quantization codebook with the LBG algorithm
 * as described by Annaji & Rao, "Parallelization of the LBG Vector
 * Quantization Algorithm for Shared Memory Systems":
 *   - Sec. 2.2 "LBG Algorithm": minimum-distortion partition, distortion,
 *     relative stop test, replacement of each codevector by its cell centroid;
 *   - Sec. 3.2 / Algorithm 1: initial codebook = centroid of the training set
 *     (Table 1), codebook splitting [c + delta], [c - delta], cell allocation
 *     (nearest codevector per training vector = the cell table), integration
 *     of distortions, updation (cell centroids);
 *   - Abstract / Sec. 1: replacement of arbitrary data by the nearest
 *     codevector (encoding).
 * Every step runs in CUDA kernels of this library on the calling device.
 *
 * Conventions for every entry point
 *   - Matrices are row-major and contiguous: X is [M x L] (M vectors of
 *     dimension L, the paper's M x k training matrix), a codebook is
 *     [N x L] float32.
 *   - Array arguments may be DEVICE pointers (cudaMalloc / managed memory)
 *     or HOST pointers (pageable or pinned).  Host arrays are copied to and
 *     from device scratch inside the call; device arrays are used in place.
 *     Scalars returned through `double *D` are always host memory.
 *   - The caller owns every array it passes.  The library owns only its
 *     internal device scratch, cached per device and released by
 *     lbg_release_workspace().  Calls on one device are serialised by an
 *     internal lock; each call synchronises its stream before it returns.
 *   - Work is issued on opts->stream (a cudaStream_t; NULL = the legacy
 *     default stream) of the current CUDA device.
 *   - Distance is the squared Euclidean distance; ties go to the lowest
 *     codevector index.  D is the SUM over vectors of the minimum distance
 *     (the paper's total distortion TD; the mean is D / M).
 *   - Arguments are validated before any device work: invalid arguments
 *     return an error and leave outputs untouched.  Device-side failures
 *     (non-finite input, a wait that timed out) are reported by status.
 *
 * Limits: 1 <= L <= LBG_MAX_DIM, 1 <= N <= LBG_MAX_CODEBOOK, N a power of 2
 * for lbg_train (Sec. 2.2: codebook sizes are powers of 2), M < 2^31.
 */
#ifndef LBGVQ_H
#define LBGVQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBG_MAX_DIM 128
#define LBG_MAX_CODEBOOK 8192

typedef enum lbg_status {
    LBG_OK = 0,
    LBG_WARN_MAXPASS = 1,     /* a stage hit max_passes before the stop test held */
    LBG_ERR_ARG = -1,         /* invalid size, pointer or parameter */
    LBG_ERR_NOT_POW2 = -2,    /* N (or n_init) is not a power of 2 */
    LBG_ERR_NONFINITE = -3,   /* NaN or Inf in X or in a codebook */
    LBG_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    LBG_ERR_NOMEM = -5,       /* device scratch could not be allocated */
    LBG_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
    LBG_ERR_UNSUPPORTED = -7  /* option not available on this device/build */
} lbg_status;

typedef enum lbg_precision {
    LBG_PREC_FP32 = 0,        /* FP32 FFMA distances, certified; exact FP32 fallback */
    LBG_PREC_BF16 = 1         /* tensor cores (BF16 operands, FP32 accumulation), certified
                                 against an accumulation-error model; exact FP32 fallback.
                                 L <= 64.  Meant for data whose centred values are exact in
                                 BF16 (integer samples such as 8-bit pixels); other data stay
                                 correct but every row goes to the exact fallback. */
} lbg_precision;

/* Actions a pass of lbg_train can end with (lbg_pass_record.action). */
enum { LBG_ACT_UPDATE = 0, LBG_ACT_SPLIT = 1, LBG_ACT_FINISH = 2 };

/* Indices into lbg_opts.phase_ms. */
enum {
    LBG_PHASE_PREP = 0,    /* codebook preparation (centring, layout) */
    LBG_PHASE_ASSIGN = 1,  /* nearest-codevector kernel */
    LBG_PHASE_EXACT = 2,   /* exact re-scoring of uncertified rows */
    LBG_PHASE_UPDATE = 3,  /* cell table + centroid update (incl. distortion) */
    LBG_PHASE_TOTAL = 4,   /* whole call on the device (excl. host copies) */
    LBG_NUM_PHASES = 5
};

/* One pass of lbg_train (one cell allocation of Algorithm 1). */
typedef struct lbg_pass_record {
    int32_t stage_n;   /* codebook size of the stage */
    int32_t pass;      /* pass index within the stage, from 0 */
    int32_t action;    /* LBG_ACT_* taken after the stop test */
    int32_t n_exact;   /* rows re-scored exactly by the fallback kernel */
    double D;          /* total distortion of the pass */
    int32_t n_empty;   /* cells (of stage_n) that no row chose in this pass */
    float ms;          /* device time of the pass, from the start of its first
                          kernel to the end of its last (%globaltimer, about
                          1 us resolution) */
} lbg_pass_record;

/* Tile choice of lbg_train_batched's persistent nearest-codevector launch and
 * the calibration behind it (see lbg_opts.autotune). */
typedef struct lbg_tune_report {
    int32_t tile_rows;            /* training rows per work item: 64 or 128 */
    int32_t ctas_per_sm;          /* resident CTAs per SM of the persistent grid */
    int32_t from_cache;           /* 1: chosen by an earlier calibration of the same bucket */
    int32_t n_candidates;         /* candidates timed by this call (0 if none ran) */
    int32_t cand_tile_rows[8];
    int32_t cand_ctas_per_sm[8];
    float cand_ms[8];             /* device time of one batched assignment of all problems at
                                     their final codebook sizes, per candidate (best of 2) */
    int32_t persistent;           /* 1: each pass ran as one persistent cooperative launch */
} lbg_tune_report;

/* Device-side report of an enqueued lbg_lloyd_step / vq_encode (see
 * lbg_opts.result_dev).  Written by the last launch of the call. */
typedef struct lbg_step_result {
    double D;                     /* sum of the minimum squared distances */
    int32_t n_exact;              /* rows re-scored exactly */
    int32_t status;               /* lbg_status of the device work: LBG_OK,
                                     LBG_ERR_NONFINITE, LBG_ERR_TIMEOUT or LBG_ERR_CUDA */
} lbg_step_result;

typedef struct lbg_opts {
    int32_t precision;          /* lbg_precision; default LBG_PREC_FP32 */
    int32_t max_passes;         /* per stage (lbg_train); <= 0 means 1000 */
    void *stream;               /* cudaStream_t; NULL = legacy default stream */
    lbg_pass_record *records;   /* host array for lbg_train's pass trace, or NULL */
    int32_t max_records;        /* capacity of records */
    int32_t *n_records;         /* host: number of passes run (may exceed capacity), or NULL */
    float *phase_ms;            /* host float[LBG_NUM_PHASES]: device time per phase, or NULL */
    int32_t *n_exact;           /* host: rows re-scored exactly (step / encode), or NULL */
    int32_t split_multiplicative; /* 0 (default, the paper): c + delta, c - delta;
                                     1: c (1 + delta), c (1 - delta) (lbg_train) */
    int32_t reseed_empty;       /* 0 (default): an empty cell keeps its codevector;
                                   1: after each update, every empty cell (in index order)
                                   takes c_b + delta from the largest cell b, which moves to
                                   c_b - delta (lbg_train, lbg_lloyd_step; uses delta_reseed
                                   in lbg_lloyd_step) */
    double delta_reseed;        /* offset for reseed_empty in lbg_lloyd_step (lbg_train uses
                                   its delta) */
    int32_t autotune;           /* lbg_train_batched: 1 (default) picks the tile of the batched
                                   nearest-codevector launch by timing the candidates (64 or 128
                                   rows per work item x resident CTAs per SM) once per bucket
                                   (L, largest N, total M) and device, then reuses the choice;
                                   0: 128 rows, 2 CTAs per SM.  Results do not depend on it. */
    int32_t tile_rows;          /* lbg_train_batched: force 64 or 128 rows (0: autotune) */
    int32_t ctas_per_sm;        /* lbg_train_batched: force 1, 2 or 4 (0: autotune; 4 needs
                                   64-row tiles) */
    lbg_tune_report *tune_report; /* host out for lbg_train_batched, or NULL */
    lbg_step_result *result_dev;  /* lbg_lloyd_step / vq_encode: DEVICE out, or NULL.  Non-NULL
                                     makes the call asynchronous: it validates, enqueues the
                                     pass on `stream` and returns without waiting; *result_dev
                                     receives D, n_exact and the device status when the stream
                                     reaches the end of the pass.  Every array must then be
                                     device memory of the current device, and the host outs
                                     (D, n_exact, phase_ms) must be NULL (else LBG_ERR_ARG).
                                     Later calls of this library on any stream of the device
                                     wait for the enqueued pass before touching its scratch. */
    float *trace_C;             /* lbg_train: DEVICE [trace_cap x N x L] or NULL.  Pass p (counted
                                   over the whole run from 0, as the records) writes the codebook
                                   its allocation used (the stage's stage_n rows; the rest of the
                                   N x L slot is left as it was) to trace_C + p N L.  Passes
                                   beyond trace_cap are not written. */
    int32_t *trace_assign;      /* lbg_train: DEVICE [trace_cap x M] or NULL.  Pass p writes its
                                   cell table (nearest codevector of every row under that
                                   codebook) to trace_assign + p M. */
    int32_t trace_cap;          /* passes trace_C / trace_assign hold */
    int32_t test_expire_wait;   /* test hook, 0 in normal use.  Non-zero: in an FP32
                                   lbg_lloyd_step / vq_encode, the first bounded wait of every CTA
                                   of the nearest-codevector kernel gives up at once, as if its
                                   codebook copy had not landed within the time limit.  Each CTA
                                   then waits (bounded) for the copies it issued, writes no row and
                                   reports; the call returns LBG_ERR_TIMEOUT.  Such calls are
                                   launched directly, never recorded into a graph.  Ignored by the
                                   other entry points and by LBG_PREC_BF16. */
    int32_t batched_per_phase;  /* lbg_train_batched: 0 (default) runs each Lloyd pass of all
                                   problems as one persistent cooperative launch (phases
                                   separated by bounded grid-wide barriers); 1 issues one
                                   launch per phase (the tile options and the autotuner apply
                                   only there).  Results do not depend on it. */
    const float *grad_scale_dev; /* lbg_distortion_backward: DEVICE float or NULL.  When set, the
                                    upstream gradient is read from it on the device and the gD
                                    argument is ignored (an autograd caller then needs no host
                                    read of it); every array must be device memory. */
    int32_t tc_group;           /* LBG_PREC_BF16: codevectors per group of the tensor-core
                                   search's running top-2 (the best group is re-scored exactly
                                   per row): 0 (default) chooses by L and N; 2, 4 or 8 forces
                                   it (other values: LBG_ERR_ARG).  Assignments do not depend on
                                   it; e(m) of a row may differ in its last bits (the exact
                                   fallback sums in another order). */
} lbg_opts;

/* Fill *opts with the defaults (FP32, 1000 passes, default stream, no trace,
 * autotuned batched tiles, synchronous calls). */
void lbg_opts_init(lbg_opts *opts);

/*
 * lbg_train -- design an N-level codebook (Sec. 2.2 + Algorithm 1).
 *
 *   X        [M x L] training vectors (read only).
 *   N        final codebook size, a power of 2.
 *   delta    split offset >= 0: every centroid c becomes c + delta (child 2i)
 *            and c - delta (child 2i + 1), added to every component
 *            (Sec. 3.2 "Codebook Splitting").
 *   theta    stop threshold >= 0: a stage ends when D == 0 or
 *            (D_prev - D) / D <= theta, D_prev = +inf at the start of each
 *            stage (Sec. 2.2 step 2).
 *   C        [N x L] out: final codebook.  If n_init > 0 its first n_init
 *            rows are read first as the starting codebook (resume).
 *   n_init   0: start from the centroid of X (Table 1); else a power of 2
 *            <= N: resume from the n_init-entry codebook held in C.
 *   assign   [M] out, nullable: the cell table of the final codebook.
 *   D        host out, nullable: total distortion of (C, assign).
 * A finished stage keeps the codebook that produced its D (before any
 * update), so (C, assign, D) are mutually consistent.  An empty cell keeps
 * its codevector.  Returns LBG_OK, LBG_WARN_MAXPASS (some stage was cut at
 * max_passes and training went on), or an error.
 */
lbg_status lbg_train(const float *X, int64_t M, int32_t L, int32_t N, double delta,
                     double theta, float *C, int32_t n_init, int32_t *assign, double *D,
                     const lbg_opts *opts);

/*
 * lbg_lloyd_step -- one Lloyd pass from a given codebook: cell allocation,
 * integration of distortions and updation (Algorithm 1), without stop test
 * or split.
 *
 *   X      [M x L] vectors; M may be 0 (every cell is then empty).
 *   C_in   [N x L] codebook used for the allocation (N >= 1, any value).
 *   C_out  [N x L] out: centroid of every cell; empty cells copy C_in.
 *          May alias C_in.
 *   assign [M] out, nullable: nearest codevector of every row under C_in.
 *   D      host out, nullable: sum of the minimum distances under C_in.
 * The device work of a call depends only on its device pointers, sizes and
 * options; it is recorded once into a CUDA graph under that key and replayed
 * by later calls with the same key (phase_ms calls launch directly, so that
 * the phases can be timed).  With opts->result_dev the call only enqueues.
 */
lbg_status lbg_lloyd_step(const float *X, int64_t M, int32_t L, int32_t N,
                          const float *C_in, float *C_out, int32_t *assign, double *D,
                          const lbg_opts *opts);

/*
 * vq_encode -- replace arbitrary vectors by their nearest codevector
 * (Abstract; Sec. 1).
 *
 *   X     [M x L] vectors to encode; M may be 0.
 *   C     [N x L] codebook (N >= 1).
 *   idx   [M] out: index of the nearest codevector.
 *   Xhat  [M x L] out, nullable: the decoded vectors C[idx[m]].
 *   D     host out, nullable: sum of the squared distances.
 * Replayed from a recorded CUDA graph and optionally asynchronous, as
 * lbg_lloyd_step (with opts->result_dev, D is always computed).
 */
lbg_status vq_encode(const float *X, int64_t M, int32_t L, const float *C, int32_t N,
                     int32_t *idx, float *Xhat, double *D, const lbg_opts *opts);

/*
 * lbg_train_batched -- S independent LBG designs (Sec. 2.2 + Algorithm 1, as
 * lbg_train) of uneven sizes, advanced together: every Lloyd pass of all
 * problems is one persistent cooperative launch (its phases separated by
 * bounded grid-wide barriers, the nearest-codevector search over (problem,
 * row tile) work items), recorded into a CUDA graph and replayed.  When the
 * device cannot hold that launch (shared memory for large L and N), or with
 * opts->batched_per_phase, a pass is a recorded sequence of one launch per
 * phase instead.
 *
 *   S        number of problems, >= 1.
 *   X        rows of all problems concatenated in problem order, [sum M_s x L]
 *            (device or host).
 *   row_off  HOST int64 [S + 1]: problem s owns rows [row_off[s], row_off[s+1]),
 *            M_s = row_off[s+1] - row_off[s] >= 1.
 *   N        HOST int32 [S]: codebook sizes, powers of 2 <= LBG_MAX_CODEBOOK.
 *   C        [sum N_s x L] out: codebooks concatenated in problem order.
 *   assign   [sum M_s] out, nullable: each problem's cell table (indices local
 *            to its codebook).
 *   D        HOST [S] out, nullable: each problem's final distortion.
 * opts: stream, max_passes, split_multiplicative, batched_per_phase, the tile
 * options are honoured; precision must be LBG_PREC_FP32; n_records receives the
 * largest pass count of a problem; tune_report gives the tile used (128 rows,
 * resident CTAs per SM of the persistent launch, when that form ran).
 * Per problem the results are those lbg_train would give.
 */
lbg_status lbg_train_batched(int32_t S, const float *X, const int64_t *row_off, int32_t L,
                             const int32_t *N, double delta, double theta, float *C,
                             int32_t *assign, double *D, const lbg_opts *opts);

/*
 * lbg_distortion_backward -- the distortion of Sec. 2.2, D = sum_m
 * ||x_m - c_a(m)||^2, at a FIXED cell table a, and its gradients scaled by
 * the upstream gradient gD (the differentiable form of the paper's
 * distortion; the paper itself has no gradient):
 *   dC[n] = 2 gD (count_n c_n - sum_{a(m)=n} x_m)      [N x L], nullable
 *   dX[m] = 2 gD (x_m - c_a(m))                         [M x L], nullable
 *   D     = the distortion at the fixed cell table      host out, nullable
 *   X [M x L], C [N x L], assign [M] (values in [0, N)) as for the other calls.
 * dC is deterministic (fixed-order cell sums, no float atomics).  gD must be
 * finite (LBG_ERR_ARG) unless opts->grad_scale_dev supplies it on the device.
 * With opts->result_dev the call only enqueues, as lbg_lloyd_step: D and the
 * device status land in *result_dev (D must then be NULL and every array
 * device memory).
 */
lbg_status lbg_distortion_backward(const float *X, int64_t M, int32_t L, const float *C, int32_t N,
                                   const int32_t *assign, float gD, float *dC, float *dX, double *D,
                                   const lbg_opts *opts);

/*
 * vq_encode_noalloc -- vq_encode for callers that cannot allocate device
 * memory.  (The paper has no counterpart: it concerns how this library gets
 * its scratch, not the method.)
 *
 * Who needs it: a serving loop that reserved its device memory up front and
 * must not pay for, or be stalled by, a cudaMalloc in steady state
 * (cudaMalloc can synchronise the device); a process whose framework
 * allocator already holds nearly all device memory, so a raw cudaMalloc
 * would fail; code that may allocate only during initialisation.  vq_encode
 * and the other entry points grow a cached workspace with cudaMalloc; this
 * one calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Its scratch is one fixed 16 MiB __device__ array inside the library, held
 * on every GPU that loads the library's device code until the process exits
 * (that load, by the first call of the library on a device that uses these
 * kernels, is when the array comes into being).  The first call on a device
 * also looks up the array's device address (cudaGetSymbolAddress with the
 * device current).  All calls share the array and each re-initialises what it
 * needs, so calls whose work overlaps on the GPU (other streams, other host
 * threads) race.  Every call reads its result back and synchronises its
 * stream before it returns, so it cannot be called on a stream that is being
 * captured into a CUDA graph.
 *
 *   X     [M x L] DEVICE array; 0 <= M <= INT32_MAX (LBG_ERR_ARG beyond;
 *         rows are processed in chunks of 2^20).
 *   C     [N x L] DEVICE codebook.
 *   idx   [M] DEVICE out: nearest codevector (same rule as vq_encode).
 *   D     host out, nullable: sum of the squared distances.
 *   stream  cudaStream_t (NULL = legacy default stream); synchronised before return.
 * Limits of the fixed scratch: N <= 4096 and L <= 128; larger sizes return
 * LBG_ERR_UNSUPPORTED.  Host pointers return LBG_ERR_ARG.
 */
lbg_status vq_encode_noalloc(const float *X, int64_t M, int32_t L, const float *C, int32_t N,
                             int32_t *idx, double *D, void *stream);

/* Human-readable text of a status code (static storage). */
const char *lbg_status_string(lbg_status s);

/* Free the cached device scratch of the current device. */
lbg_status lbg_release_workspace(void);

/*
 * lbg_set_workspace_limit -- cap, in bytes, on the cached device scratch of
 * every device (0 = no cap, the default).  The cap is enforced where the
 * scratch is allocated: a call that needs more than the cap behaves as if
 * cudaMalloc had refused -- the cached scratch of the device is released (as
 * for any growth) and the call returns LBG_ERR_NOMEM with its outputs
 * untouched.  Lifting or raising the cap makes later calls succeed again.
 * (A memory budget for the library's scratch; no counterpart in the paper.)
 */
lbg_status lbg_set_workspace_limit(size_t bytes);

/*
 * lbg_launch_count -- number of CUDA kernels this library has launched in
 * this process (all devices): direct launches, plus the kernels of a
 * recorded graph each time it is replayed.  Recording a graph launches
 * nothing and is not counted.  A diagnostic for reports; no counterpart in
 * the paper.
 */
int64_t lbg_launch_count(void);

/*
 * lbg_measure_fp32_peak -- the FP32 FMA throughput of the current device,
 * measured: a kernel of independent FFMA chains on every SM (32 warps per SM,
 * 8 chains per thread) is timed with CUDA events on `stream` after a warm-up
 * launch.  *tflops = 2 flop per lane FMA / time (TFLOP/s, at whatever SM clock
 * the device ran), *sms = the device's multiprocessor count (either out may be
 * NULL).  The denominator of the FP32 nearest-codevector kernel's roofline;
 * no counterpart in the paper.  Synchronises the stream.
 */
lbg_status lbg_measure_fp32_peak(void *stream, double *tflops, int32_t *sms);

/* Library ABI version (this header: 2). */
int32_t lbg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBGVQ_H */
