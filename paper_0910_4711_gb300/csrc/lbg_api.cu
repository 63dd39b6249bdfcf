// lbg_api.cu -- host side of the C ABI declared in include/lbgvq.h:
// argument validation, per-device workspace, host<->device staging and the
// launch sequences of lbg_train / lbg_lloyd_step / vq_encode.
#include "lbgvq.h"
#include "lbg_internal.cuh"

#include <math.h>
#include <string.h>

#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <algorithm>
#include <vector>

using namespace lbg;

namespace {
constexpr int MAX_DEVICES = 64;
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_sms[MAX_DEVICES];
std::atomic<size_t> g_ws_limit{0};
}  // namespace

namespace lbg {
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int num_sms()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        (void)cudaGetLastError();
        return 1;
    }
    int n = g_sms[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        return 1;
    }
    g_sms[dev].store(n, std::memory_order_relaxed);
    return n;
}
}  // namespace lbg

namespace {

struct Workspace {
    void *base = nullptr;
    size_t bytes = 0;
};

std::mutex g_mu;
Workspace g_ws[MAX_DEVICES];
// Recorded at the end of every asynchronous call's device work; every call
// makes its stream wait for it before touching the workspace.
cudaEvent_t g_ws_done[MAX_DEVICES];

void seq_clear(int dev);

// Byte offsets of the scratch arrays of one call inside the workspace.
struct Plan {
    int64_t M = 0, R = 0, S = 0, nq = 0;
    int L = 0, Lp = 0, N = 0, NP = 0, CH = 0, G = 0, max_rec = 0;
    int grp = 0;       // tensor-core search: codevectors per top-2 group (0: by L and N)
    bool tc = false;   // tensor-core (BF16) allocation
    size_t state, rec, Cp, kn, CT, mu, Ccur, Calt, assign, e, flags, table, dpart, counts, off, perm,
        pieces, mpart, Xs, Cin, Cout, Xhat, Bp, xpart_d, xpart_i, xcnt, qcell, cell_done;
    size_t total = 0;
    size_t take(size_t bytes)
    {
        const size_t at = total;
        total += (bytes + 255) / 256 * 256;
        return at;
    }
};

Plan make_plan(int64_t M, int L, int N, int max_rec, bool host_X, bool need_assign, bool host_C,
               bool host_Xhat, bool tc)
{
    Plan p;
    p.tc = tc;
    p.M = M;
    p.L = L;
    p.Lp = round_up(L, 4);
    p.N = N;
    p.NP = round_up(N, BN);
    p.max_rec = max_rec;
    // histogram / scatter chunks: <= HIST_CHUNKS_MAX CTAs of R rows (R a multiple of 256)
    int64_t ch = (M + 1023) / 1024;
    const int64_t ch_cap = std::min<int64_t>(HIST_CHUNKS_MAX, 2 * (int64_t)num_sms());
    if (ch > ch_cap) ch = ch_cap;
    if (ch < 1) ch = 1;
    p.R = round_up64((M + ch - 1) / ch, 256);
    if (p.R < 256) p.R = 256;
    p.CH = (int)((M + p.R - 1) / p.R);
    if (p.CH < 1) p.CH = 1;
    // centroid pieces: one warp per S cell-sorted rows, aiming at >= 64 warps per SM
    const int64_t warps = (int64_t)num_sms() * 64;
    int64_t S = round_up64((M + warps - 1) / warps, 32);
    if (S < 128) S = 128;
    if (S > 4096) S = 4096;
    p.S = S;
    p.nq = (M + S - 1) / S;
    int64_t g = (M + 4095) / 4096;
    if (g > 2 * num_sms()) g = 2 * num_sms();
    if (g < 1) g = 1;
    p.G = (int)g;

    p.state = p.take(sizeof(DevState));
    p.rec = p.take(sizeof(PassRecord) * (size_t)(max_rec > 0 ? max_rec : 1));
    p.Cp = p.take(sizeof(float) * (size_t)(p.NP / BN) * (p.Lp + 1) * BN);
    p.kn = p.take(sizeof(float) * (size_t)p.NP);
    p.CT = p.take(sizeof(float) * (size_t)p.Lp * p.NP);
    p.mu = p.take(sizeof(float) * (size_t)p.Lp);
    p.Ccur = p.take(sizeof(float) * (size_t)N * L);
    p.Calt = p.take(sizeof(float) * (size_t)N * L);
    p.assign = need_assign ? p.take(sizeof(int32_t) * (size_t)(M > 0 ? M : 1)) : 0;
    p.e = p.take(sizeof(float) * (size_t)(M > 0 ? M : 1));
    p.flags = p.take(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    p.table = p.take(sizeof(int32_t) * (size_t)p.CH * N);
    p.dpart = p.take(sizeof(double) * (size_t)p.CH);
    p.counts = p.take(sizeof(int32_t) * (size_t)N);
    p.off = p.take(sizeof(int32_t) * (size_t)(N + 1));
    p.perm = p.take(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    p.pieces = p.take(sizeof(float) * (size_t)(N + p.nq) * L);
    p.qcell = p.take(sizeof(int32_t) * (size_t)(p.nq > 0 ? p.nq : 1));
    p.cell_done = p.take(sizeof(int32_t) * (size_t)(2 * N + p.nq));   // per cell, then per piece group
    p.mpart = p.take(sizeof(double) * (size_t)p.G * L);
    p.Xs = host_X ? p.take(sizeof(float) * (size_t)M * L) : 0;
    p.Cin = host_C ? p.take(sizeof(float) * (size_t)N * L) : 0;
    p.Cout = host_C ? p.take(sizeof(float) * (size_t)N * L) : 0;
    p.Xhat = host_Xhat ? p.take(sizeof(float) * (size_t)M * L) : 0;
    p.Bp = tc ? p.take(tc_codebook_bytes(p.NP, L)) : 0;
    p.xpart_d = p.take(sizeof(float) * 2 * (size_t)exact_split_ctas() * exact_split_rows());
    p.xpart_i = p.take(sizeof(int32_t) * 2 * (size_t)exact_split_ctas() * exact_split_rows());
    p.xcnt = p.take(sizeof(int32_t) * (size_t)exact_split_ctas());
    return p;
}

struct Call {
    int dev = 0;
    cudaStream_t s = nullptr;
    char *ws = nullptr;
    template <class T>
    T *at(size_t off) const
    {
        return reinterpret_cast<T *>(ws + off);
    }
};

#define CK(expr)                                    \
    do {                                            \
        if ((expr) != cudaSuccess) {                \
            (void)cudaGetLastError();               \
            return LBG_ERR_CUDA;                    \
        }                                           \
    } while (0)

lbg_status ensure_workspace(Call &c, size_t bytes)
{
    Workspace &w = g_ws[c.dev];
    const size_t cap = g_ws_limit.load();
    if (w.bytes < bytes || (cap != 0 && bytes > cap)) {
        if (w.base) {
            CK(cudaDeviceSynchronize());
            seq_clear(c.dev);
            cudaFree(w.base);
            w.base = nullptr;
            w.bytes = 0;
        }
        void *p = nullptr;
        if (cap != 0 && bytes > cap) return LBG_ERR_NOMEM;   // as if cudaMalloc had refused
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            return LBG_ERR_NOMEM;
        }
        w.base = p;
        w.bytes = bytes;
    }
    c.ws = static_cast<char *>(w.base);
    return LBG_OK;
}

// 1 = device-accessible, 0 = host memory, -1 = device memory of another GPU.
int where(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? 1 : -1;
    return 0;
}

bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

lbg_opts resolve(const lbg_opts *o)
{
    lbg_opts r;
    lbg_opts_init(&r);
    if (o) r = *o;
    if (r.max_passes <= 0) r.max_passes = 1000;
    if (!r.records) r.max_records = 0;
    return r;
}

lbg_status begin(Call &c, const lbg_opts &o)
{
    CK(cudaGetDevice(&c.dev));
    if (c.dev < 0 || c.dev >= MAX_DEVICES) return LBG_ERR_UNSUPPORTED;
    c.s = static_cast<cudaStream_t>(o.stream);
    if (g_ws_done[c.dev]) CK(cudaStreamWaitEvent(c.s, g_ws_done[c.dev], 0));
    return LBG_OK;
}

// Marks the workspace busy until the work enqueued so far on c.s is done.
lbg_status end_async(const Call &c)
{
    if (!g_ws_done[c.dev]) CK(cudaEventCreateWithFlags(&g_ws_done[c.dev], cudaEventDisableTiming));
    CK(cudaEventRecord(g_ws_done[c.dev], c.s));
    return LBG_OK;
}

lbg_status finish_status(const DevState &st)
{
    if (st.err & ERR_NONFINITE) return LBG_ERR_NONFINITE;
    if (st.err & ERR_TIMEOUT) return LBG_ERR_TIMEOUT;
    if (st.err & ERR_INTERNAL) return LBG_ERR_CUDA;
    return st.warn ? LBG_WARN_MAXPASS : LBG_OK;
}

struct Timer {
    bool on = false;
    cudaEvent_t ev[5] = {};
    lbg_status init(bool want)
    {
        on = want;
        if (!on) return LBG_OK;
        for (auto &e : ev) CK(cudaEventCreate(&e));
        return LBG_OK;
    }
    void mark(int i, cudaStream_t s)
    {
        if (on) cudaEventRecord(ev[i], s);
    }
    void report(float *out, bool per_phase)
    {
        if (!on) return;
        for (int i = 0; i < LBG_NUM_PHASES; ++i) out[i] = 0.f;
        if (per_phase) {
            for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&out[i], ev[i], ev[i + 1]);
        }
        cudaEventElapsedTime(&out[LBG_PHASE_TOTAL], ev[0], ev[4]);
    }
    ~Timer()
    {
        if (on)
            for (auto &e : ev) cudaEventDestroy(e);
    }
};

void init_state(DevState &h, int n_cur)
{
    memset(&h, 0, sizeof(h));
    h.n_cur = n_cur;
    h.D_prev = INFINITY;
}

// Device-side report of an asynchronous step / encode (finish_status without
// the max_passes warning, which only lbg_train raises).
__global__ void k_step_report(const DevState *st, lbg_step_result *r, int use_last)
{
    const uint32_t err = st->err;
    lbg_step_result o;
    o.D = st->D;
    o.n_exact = use_last ? st->n_exact_last : st->nflag;
    o.status = (err & ERR_NONFINITE)  ? LBG_ERR_NONFINITE
               : (err & ERR_TIMEOUT)  ? LBG_ERR_TIMEOUT
               : (err & ERR_INTERNAL) ? LBG_ERR_CUDA
                                      : LBG_OK;
    *r = o;
}

// Prepared codebook + one allocation (cell table of C under X) -> assign, e.
void run_prepare(const Call &c, const Plan &p, const float *C, const int32_t *n_dev, int n_host,
                 const float *mu, DevState *st, bool zero_bounds = true)
{
    if (zero_bounds) cudaMemsetAsync(&st->cmax_bits, 0, 2 * sizeof(uint32_t), c.s);   // cmax_bits, rho_bits
    if (p.tc)
        launch_prep_tc(C, p.N, n_dev, n_host, p.L, mu, c.at<void>(p.Bp), c.at<float>(p.kn),
                       c.at<float>(p.CT), st, c.s);
    else
        launch_prep(C, p.N, n_dev, n_host, p.L, p.Lp, mu, c.at<float>(p.Cp), c.at<float>(p.kn),
                    c.at<float>(p.CT), p.NP, st, c.s);
}

// Nearest codevector of rows [m_lo, m_hi) (default: all rows).
void run_assign(const Call &c, const Plan &p, const float *X, const float *C, const int32_t *n_dev,
                int n_host, const float *mu, DevState *st, int32_t *assign, int64_t m_lo = 0,
                int64_t m_hi = -1, int expire = 0)
{
    const int64_t M = m_hi < 0 ? p.M : m_hi;
    if (p.tc)
        launch_assign_tc(X, M, p.L, c.at<void>(p.Bp), c.at<float>(p.kn), n_dev, n_host, mu, C, st,
                         assign, c.at<float>(p.e), c.at<int32_t>(p.flags), c.s, m_lo, p.grp);
    else
        launch_assign(X, M, p.L, p.Lp, c.at<float>(p.Cp), c.at<float>(p.kn), n_dev, n_host, mu, C,
                      st, assign, c.at<float>(p.e), c.at<int32_t>(p.flags), c.s, m_lo, expire);
}

// Host-resident X: its rows go to the device staging buffer Xs in pieces on a
// copy stream, and the nearest-codevector search of each piece starts as soon
// as it has landed, so that the host-to-device copy (the larger cost of a step
// from host memory) overlaps the search.  A piece is one wave of the search
// (SMs x 256 rows; the FP32 kernel's wave, 2 x SMs x 128 rows, is the
// same), so that each piece's search keeps pace with the next piece's copy
// (measured ~210 GB/s host-to-device); at most HOST_CHUNKS pieces.  Every
// piece's copy is issued at the start of the call, right after the codebook's,
// before any kernel, so that the link is busy from the start.
constexpr int HOST_CHUNKS = 32;
constexpr int EV_BEGIN = HOST_CHUNKS, EV_RESULT = HOST_CHUNKS + 1, EV_D2H = HOST_CHUNKS + 2;
int64_t host_piece_rows() { return (int64_t)num_sms() * 256; }
cudaStream_t g_copy[MAX_DEVICES];
cudaEvent_t g_copy_ev[MAX_DEVICES][HOST_CHUNKS + 3];

bool ensure_copy_stream(int d)
{
    if (g_copy[d]) return true;
    if (cudaStreamCreateWithFlags(&g_copy[d], cudaStreamNonBlocking) != cudaSuccess) return false;
    for (auto &e : g_copy_ev[d])
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
}

// Piece k of np: rows [r0, r1), in whole 256-row tiles.
int host_pieces(const Plan &p)
{
    const int64_t piece = host_piece_rows();
    const int64_t np = (p.M + piece - 1) / piece;
    return (int)(np > HOST_CHUNKS ? HOST_CHUNKS : np);
}
void host_piece(const Plan &p, int k, int np, int64_t &r0, int64_t &r1)
{
    const int64_t tiles = (p.M + 255) / 256;
    r0 = std::min<int64_t>(p.M, tiles * k / np * 256);
    r1 = std::min<int64_t>(p.M, tiles * (k + 1) / np * 256);
}

// The copies may start once everything issued so far on c.s (earlier users of
// Xs) is done: host_copy_begin records that point.  The call then issues its
// codebook's copy (small) and host_copy_pieces every piece's copy, each
// recording its event: copies are served in the order they are issued, so the
// codebook's copy goes first rather than behind the whole of X.
bool host_copy_begin(const Call &c)
{
    const int d = c.dev;
    return ensure_copy_stream(d) && cudaEventRecord(g_copy_ev[d][EV_BEGIN], c.s) == cudaSuccess &&
           cudaStreamWaitEvent(g_copy[d], g_copy_ev[d][EV_BEGIN], 0) == cudaSuccess;
}
bool host_copy_pieces(const Call &c, const Plan &p, const float *hostX, float *Xs)
{
    const int d = c.dev;
    const int np = host_pieces(p);
    for (int k = 0; k < np; ++k) {
        int64_t r0, r1;
        host_piece(p, k, np, r0, r1);
        if (r1 <= r0) continue;
        const size_t off = (size_t)r0 * p.L, bytes = sizeof(float) * (size_t)(r1 - r0) * p.L;
        if (cudaMemcpyAsync(Xs + off, hostX + off, bytes, cudaMemcpyHostToDevice, g_copy[d]) != cudaSuccess ||
            cudaEventRecord(g_copy_ev[d][k], g_copy[d]) != cudaSuccess)
            return false;
    }
    return true;
}

// The search of each piece once its copy (host_copy_pieces) has landed.
bool run_assign_host(const Call &c, const Plan &p, float *Xs, const float *C, const int32_t *n_dev, int n_host,
                     const float *mu, DevState *st, int32_t *assign, int expire = 0)
{
    const int d = c.dev;
    const int np = host_pieces(p);
    for (int k = 0; k < np; ++k) {
        int64_t r0, r1;
        host_piece(p, k, np, r0, r1);
        if (r1 <= r0) continue;
        if (cudaStreamWaitEvent(c.s, g_copy_ev[d][k], 0) != cudaSuccess) return false;
        run_assign(c, p, Xs, C, n_dev, n_host, mu, st, assign, r0, r1, expire);
    }
    return true;
}

// A result that is final at this point of c.s goes to the host on the copy
// stream while c.s carries on; host_d2h_join makes c.s wait for it.
bool host_d2h_after(const Call &c, void *dst, const void *src, size_t bytes)
{
    const int d = c.dev;
    return ensure_copy_stream(d) && cudaEventRecord(g_copy_ev[d][EV_RESULT], c.s) == cudaSuccess &&
           cudaStreamWaitEvent(g_copy[d], g_copy_ev[d][EV_RESULT], 0) == cudaSuccess &&
           cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, g_copy[d]) == cudaSuccess &&
           cudaEventRecord(g_copy_ev[d][EV_D2H], g_copy[d]) == cudaSuccess;
}
bool host_d2h_join(const Call &c)
{
    return cudaStreamWaitEvent(c.s, g_copy_ev[c.dev][EV_D2H], 0) == cudaSuccess;
}

void run_exact(const Call &c, const Plan &p, const float *X, const int32_t *n_dev, int n_host,
               DevState *st, int32_t *assign)
{
    cudaMemsetAsync(c.at<int32_t>(p.xcnt), 0, sizeof(int32_t) * (size_t)exact_split_ctas(), c.s);
    launch_exact_split(X, p.L, p.Lp, c.at<float>(p.CT), n_dev, n_host, st, c.at<int32_t>(p.flags), assign,
                       c.at<float>(p.e), c.at<float>(p.xpart_d), c.at<int32_t>(p.xpart_i),
                       c.at<int32_t>(p.xcnt), p.M, c.s);
}

// Cell table and centroids after the histogram: cell sizes, offsets and piece
// cells in one launch, the stable placement, then the cell sums with the
// centroid division folded in (three launches).
void run_update(const Call &c, const Plan &p, const float *X, const int32_t *n_dev, int n_host,
                DevState *st, const int32_t *assign, const float *C_in, float *C_out, bool train)
{
    int32_t *table = c.at<int32_t>(p.table), *off = c.at<int32_t>(p.off);
    int32_t *qcell = c.at<int32_t>(p.qcell), *done = c.at<int32_t>(p.cell_done);
    launch_scan_offsets_q(table, p.CH, n_dev, n_host, c.at<int32_t>(p.counts), off, qcell, done, p.S, p.L,
                          C_in, C_out, st, train, c.s);
    launch_scatter(assign, p.M, p.R, p.CH, table, off, n_dev, n_host, c.at<int32_t>(p.perm), st,
                   train, c.s);
    launch_cellsum_c(X, p.M, p.L, c.at<int32_t>(p.perm), off, qcell, n_dev, n_host, p.S,
                     c.at<float>(p.pieces), done, C_out, st, train, c.s);
}

// Training stages of at most this many codevectors take k_assign_direct (every
// row against every codevector, FP32 direct form): measured per pass on the
// 8 x 8 image blocks, the tiled search with its certificate and re-scoring
// costs more below these sizes.
constexpr int DIRECT_MAX_TC = 8, DIRECT_MAX_F32 = 64;

// 0 = FP32, 1 = tensor cores, <0 = error status
int precision_mode(const lbg_opts &o, int L)
{
    if (o.tc_group != 0 && o.tc_group != 2 && o.tc_group != 4 && o.tc_group != 8) return LBG_ERR_ARG;
    if (o.precision == LBG_PREC_FP32) return 0;
    if (o.precision == LBG_PREC_BF16) return tc_supported(L) ? 1 : LBG_ERR_UNSUPPORTED;
    return LBG_ERR_ARG;
}

// One training pass recorded into a CUDA graph and replayed: many small
// kernels per pass are then issued with one launch.  Capture uses a private
// stream (the caller's may be the legacy default stream, which cannot be
// captured); if capture is not possible the pass is launched directly.
struct GraphPass {
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev = nullptr;
    int64_t kernels = 0;   // kernels recorded into the graph (counted per replay)
    template <class F>
    void build(cudaStream_t user, F &&issue)
    {
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            return;
        }
        // warm the kernels' attributes outside capture, in stream order
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            (void)cudaGetLastError();
            return;
        }
        const int64_t before = g_launches.load();
        issue(cap);
        kernels = g_launches.load() - before;
        g_launches.fetch_sub(kernels);   // recording launches nothing
        if (cudaStreamEndCapture(cap, &graph) != cudaSuccess || !graph ||
            cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            if (graph) cudaGraphDestroy(graph);
            graph = nullptr;
            exec = nullptr;
        }
        (void)user;
    }
    template <class F>
    void run(cudaStream_t user, F &&issue)
    {
        if (!exec) {
            issue(user);
            return;
        }
        cudaEventRecord(ev, user);
        cudaStreamWaitEvent(cap, ev, 0);
        cudaGraphLaunch(exec, cap);
        g_launches.fetch_add(kernels);
        cudaEventRecord(ev, cap);
        cudaStreamWaitEvent(user, ev, 0);
    }
    // Forget the recorded pass (its recording was incomplete): passes launch directly.
    void drop()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~GraphPass()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ev) cudaEventDestroy(ev);
        if (cap) cudaStreamDestroy(cap);
    }
};

// Replayed device sequences of lbg_lloyd_step / vq_encode.  Everything such
// a call launches follows from the device pointers it touches, its sizes and
// its options, so the sequence is recorded once into a graph under that key
// and later calls with the same key launch the graph on their own stream.
struct SeqKey {
    int dev, op, mode, flags;   // op: 0 step, 1 encode; flags: bit 0 reseed, 1 D, 2 decode,
                                // bits 8..: the tensor-core group option
    int64_t M;
    int L, N;
    size_t total;               // workspace plan size (fixes every scratch offset)
    double dres;
    const void *X, *C, *Co, *A, *H, *res, *ws;
    bool operator==(const SeqKey &k) const
    {
        return dev == k.dev && op == k.op && mode == k.mode && flags == k.flags && M == k.M &&
               L == k.L && N == k.N && total == k.total && dres == k.dres && X == k.X && C == k.C &&
               Co == k.Co && A == k.A && H == k.H && res == k.res && ws == k.ws;
    }
};

struct SeqGraph {
    SeqKey key;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
    int64_t kernels = 0;   // kernels recorded into the graph (counted per replay)
};

constexpr size_t SEQ_CACHE_MAX = 32;
std::vector<SeqGraph> g_seq;
uint64_t g_seq_clock = 0;
cudaStream_t g_cap[MAX_DEVICES];

// Destroys the cached graphs of device `dev` (all devices if dev < 0); the
// caller has made sure none of them is still running.
void seq_clear(int dev)
{
    for (size_t i = 0; i < g_seq.size();) {
        if (dev < 0 || g_seq[i].key.dev == dev) {
            cudaGraphExecDestroy(g_seq[i].exec);
            g_seq[i] = g_seq.back();
            g_seq.pop_back();
        } else {
            ++i;
        }
    }
}

// Launches the sequence of `key` on c.s: from the cache, else recorded now
// (on a private capturing stream: c.s may be the legacy stream), else issued
// directly when recording is not possible.
template <class F>
lbg_status seq_run(const Call &c, const SeqKey &key, F &&issue)
{
    SeqGraph *hit = nullptr;
    for (auto &g : g_seq)
        if (g.key == key) hit = &g;
    if (!hit) {
        if (!g_cap[c.dev] && cudaStreamCreateWithFlags(&g_cap[c.dev], cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            issue(c.s);
            CK(cudaGetLastError());
            return LBG_OK;
        }
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int64_t kernels = 0;
        if (cudaStreamBeginCapture(g_cap[c.dev], cudaStreamCaptureModeRelaxed) == cudaSuccess) {
            const int64_t before = g_launches.load();
            issue(g_cap[c.dev]);
            kernels = g_launches.load() - before;
            g_launches.fetch_sub(kernels);   // recording launches nothing
            if (cudaStreamEndCapture(g_cap[c.dev], &graph) != cudaSuccess || !graph ||
                cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
                exec = nullptr;
        }
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        if (!exec) {
            issue(c.s);
            CK(cudaGetLastError());
            return LBG_OK;
        }
        if (g_seq.size() >= SEQ_CACHE_MAX) {
            // evict the least recently used graph once every launch of it is done
            size_t old = 0;
            for (size_t i = 1; i < g_seq.size(); ++i)
                if (g_seq[i].used < g_seq[old].used) old = i;
            CK(cudaSetDevice(g_seq[old].key.dev));
            const lbg_status rc = cudaDeviceSynchronize() == cudaSuccess ? LBG_OK : LBG_ERR_CUDA;
            CK(cudaSetDevice(c.dev));
            if (rc != LBG_OK) {
                cudaGraphExecDestroy(exec);
                return rc;
            }
            cudaGraphExecDestroy(g_seq[old].exec);
            g_seq[old] = g_seq.back();
            g_seq.pop_back();
        }
        g_seq.push_back(SeqGraph{key, exec, 0, kernels});
        hit = &g_seq.back();
    }
    hit->used = ++g_seq_clock;
    CK(cudaGraphLaunch(hit->exec, c.s));
    g_launches.fetch_add(hit->kernels);
    return LBG_OK;
}

lbg_status check_dims(int64_t M, int32_t L, int32_t N)
{
    if (M < 0 || M > INT32_MAX) return LBG_ERR_ARG;
    if (L < 1 || L > LBG_MAX_DIM) return LBG_ERR_ARG;
    if (N < 1 || N > LBG_MAX_CODEBOOK) return LBG_ERR_ARG;
    return LBG_OK;
}

}  // namespace

extern "C" {

void lbg_opts_init(lbg_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = LBG_PREC_FP32;
    o->max_passes = 1000;
    o->autotune = 1;
}

int32_t lbg_version(void) { return 2; }

lbg_status lbg_set_workspace_limit(size_t bytes)
{
    g_ws_limit.store(bytes);
    return LBG_OK;
}

int64_t lbg_launch_count(void) { return g_launches.load(); }

const char *lbg_status_string(lbg_status s)
{
    switch (s) {
    case LBG_OK: return "ok";
    case LBG_WARN_MAXPASS: return "a stage reached max_passes before the stop test held";
    case LBG_ERR_ARG: return "invalid argument";
    case LBG_ERR_NOT_POW2: return "codebook size is not a power of 2";
    case LBG_ERR_NONFINITE: return "non-finite value in the input vectors or codebook";
    case LBG_ERR_CUDA: return "CUDA runtime error";
    case LBG_ERR_NOMEM: return "device scratch allocation failed";
    case LBG_ERR_TIMEOUT: return "a bounded device wait timed out";
    case LBG_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

lbg_status lbg_release_workspace(void)
{
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return LBG_ERR_UNSUPPORTED;
    if (g_ws[dev].base) {
        CK(cudaDeviceSynchronize());
        seq_clear(dev);
        cudaFree(g_ws[dev].base);
        g_ws[dev].base = nullptr;
        g_ws[dev].bytes = 0;
    }
    return LBG_OK;
}

lbg_status vq_encode(const float *X, int64_t M, int32_t L, const float *C, int32_t N, int32_t *idx,
                     float *Xhat, double *D, const lbg_opts *opts)
{
    lbg_status rc = check_dims(M, L, N);
    if (rc != LBG_OK) return rc;
    if (!C || (M > 0 && (!X || !idx))) return LBG_ERR_ARG;
    const lbg_opts o = resolve(opts);
    const int mode = precision_mode(o, L);
    if (mode < 0) return (lbg_status)mode;
    lbg_step_result *res = o.result_dev;
    if (res && (D || o.n_exact || o.phase_ms)) return LBG_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    Call c;
    if ((rc = begin(c, o)) != LBG_OK) return rc;
    if (res && where(res, c.dev) != 1) return LBG_ERR_ARG;
    if (M == 0) {
        if (D) *D = 0.0;
        if (o.n_exact) *o.n_exact = 0;
        if (res) CK(cudaMemsetAsync(res, 0, sizeof(*res), c.s));   // D = 0, n_exact = 0, LBG_OK
        return LBG_OK;
    }
    const int wX = where(X, c.dev), wC = where(C, c.dev), wI = where(idx, c.dev);
    const int wH = Xhat ? where(Xhat, c.dev) : 1;
    if (wX < 0 || wC < 0 || wI < 0 || wH < 0) return LBG_ERR_ARG;
    if (res && (wX != 1 || wC != 1 || wI != 1 || wH != 1)) return LBG_ERR_ARG;
    Plan p = make_plan(M, L, N, 0, wX == 0, wI == 0, wC == 0, wH == 0, mode == 1);
    p.grp = o.tc_group;
    if ((rc = ensure_workspace(c, p.total)) != LBG_OK) return rc;
    DevState *st = c.at<DevState>(p.state);
    // host X: every piece's copy is issued up front (after C's); the search takes the
    // pieces as they land
    if (wX == 0 && !host_copy_begin(c)) {
        (void)cudaGetLastError();
        return LBG_ERR_CUDA;
    }
    const float *dX = wX == 0 ? c.at<float>(p.Xs) : X;
    const float *dC = C;
    if (wC == 0) {
        CK(cudaMemcpyAsync(c.at<float>(p.Cin), C, sizeof(float) * (size_t)N * L,
                           cudaMemcpyHostToDevice, c.s));
        dC = c.at<float>(p.Cin);
    }
    if (wX == 0 && !host_copy_pieces(c, p, X, c.at<float>(p.Xs))) {
        (void)cudaGetLastError();
        return LBG_ERR_CUDA;
    }
    int32_t *dI = wI ? idx : c.at<int32_t>(p.assign);
    float *dH = Xhat ? (wH ? Xhat : c.at<float>(p.Xhat)) : nullptr;
    const bool wantD = D || res;
    // host X and idx (always issued directly): idx goes back while the distortion is summed
    const bool d2h_early = wX == 0 && wI == 0;
    bool host_ok = true;
    Timer tm;
    if ((rc = tm.init(o.phase_ms != nullptr)) != LBG_OK) return rc;
    float *mu = c.at<float>(p.mu);
    auto issue = [&](cudaStream_t s) {
        Call k = c;
        k.s = s;
        tm.mark(0, s);
        launch_begin(dC, N, L, mu, p.tc, st, s);   // also the initial state (cmax, rho zero)
        run_prepare(k, p, dC, nullptr, N, mu, st, false);
        tm.mark(1, s);
        if (wX == 0) {
            if (!run_assign_host(k, p, c.at<float>(p.Xs), dC, nullptr, N, mu, st, dI, o.test_expire_wait))
                host_ok = false;
        } else {
            run_assign(k, p, dX, dC, nullptr, N, mu, st, dI, 0, -1, o.test_expire_wait);
        }
        tm.mark(2, s);
        run_exact(k, p, dX, nullptr, N, st, dI);
        tm.mark(3, s);
        if (d2h_early && !host_d2h_after(k, idx, dI, sizeof(int32_t) * M)) host_ok = false;
        if (wantD) launch_hist_ctl(dI, k.at<float>(p.e), M, p.R, p.CH, N, false, nullptr, k.at<double>(p.dpart), st, s);
        if (dH) launch_decode(dI, M, L, dC, dH, s);
        if (res) LBG_COUNTED k_step_report<<<1, 1, 0, s>>>(st, res, 1);
        tm.mark(4, s);
    };
    if (o.phase_ms || wX == 0 || o.test_expire_wait) {   // direct: timed phases, host X pieces, test hook
        issue(c.s);
        if (!host_ok) return LBG_ERR_CUDA;
        CK(cudaGetLastError());
    } else {
        const SeqKey key{c.dev, 1, mode, (wantD ? 2 : 0) | (dH ? 4 : 0) | (p.grp << 8), M, L, N, p.total, 0.0,
                         dX, dC, nullptr, dI, dH, res, c.ws};
        if ((rc = seq_run(c, key, issue)) != LBG_OK) return rc;
    }
    if (res) return end_async(c);
    if (d2h_early && !host_d2h_join(c)) return LBG_ERR_CUDA;
    if (wI == 0 && !d2h_early) CK(cudaMemcpyAsync(idx, dI, sizeof(int32_t) * M, cudaMemcpyDeviceToHost, c.s));
    if (Xhat && wH == 0)
        CK(cudaMemcpyAsync(Xhat, dH, sizeof(float) * M * L, cudaMemcpyDeviceToHost, c.s));
    DevState h;
    CK(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, c.s));
    CK(cudaStreamSynchronize(c.s));
    tm.report(o.phase_ms, true);
    if (D) *D = h.D;
    if (o.n_exact) *o.n_exact = D ? h.n_exact_last : h.nflag;
    return finish_status(h);
}

lbg_status lbg_lloyd_step(const float *X, int64_t M, int32_t L, int32_t N, const float *C_in,
                          float *C_out, int32_t *assign, double *D, const lbg_opts *opts)
{
    lbg_status rc = check_dims(M, L, N);
    if (rc != LBG_OK) return rc;
    if (!C_in || !C_out || (M > 0 && !X)) return LBG_ERR_ARG;
    const lbg_opts o = resolve(opts);
    const int mode = precision_mode(o, L);
    if (mode < 0) return (lbg_status)mode;
    lbg_step_result *res = o.result_dev;
    if (res && (D || o.n_exact || o.phase_ms)) return LBG_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    Call c;
    if ((rc = begin(c, o)) != LBG_OK) return rc;
    const int wX = M > 0 ? where(X, c.dev) : 1, wCi = where(C_in, c.dev), wCo = where(C_out, c.dev);
    const int wA = assign ? where(assign, c.dev) : 0;
    if (wX < 0 || wCi < 0 || wCo < 0 || wA < 0) return LBG_ERR_ARG;
    if (res && (wX != 1 || wCi != 1 || wCo != 1 || (assign && wA != 1) || where(res, c.dev) != 1))
        return LBG_ERR_ARG;
    const bool hostC = (wCi == 0) || (wCo == 0);
    const bool wsA = !(assign && wA == 1);
    Plan p = make_plan(M, L, N, 0, wX == 0, wsA, hostC, false, mode == 1);
    p.grp = o.tc_group;
    if ((rc = ensure_workspace(c, p.total)) != LBG_OK) return rc;
    const size_t cbytes = sizeof(float) * (size_t)N * L;
    if (M == 0) {
        if (C_out != C_in) CK(cudaMemcpyAsync(C_out, C_in, cbytes, cudaMemcpyDefault, c.s));
        if (res) {
            CK(cudaMemsetAsync(res, 0, sizeof(*res), c.s));   // D = 0, n_exact = 0, LBG_OK
            return end_async(c);
        }
        CK(cudaStreamSynchronize(c.s));
        if (D) *D = 0.0;
        if (o.n_exact) *o.n_exact = 0;
        if (o.phase_ms)
            for (int i = 0; i < LBG_NUM_PHASES; ++i) o.phase_ms[i] = 0.f;
        return LBG_OK;
    }
    DevState *st = c.at<DevState>(p.state);
    // host X: every piece's copy is issued up front (after C's); the search takes the
    // pieces as they land
    if (wX == 0 && !host_copy_begin(c)) {
        (void)cudaGetLastError();
        return LBG_ERR_CUDA;
    }
    const float *dX = wX == 0 ? c.at<float>(p.Xs) : X;
    const float *dCi = C_in;
    float *dCo = C_out;
    if (hostC) {
        CK(cudaMemcpyAsync(c.at<float>(p.Cin), C_in, cbytes, cudaMemcpyDefault, c.s));
        dCi = c.at<float>(p.Cin);
        dCo = c.at<float>(p.Cout);
    }
    if (wX == 0 && !host_copy_pieces(c, p, X, c.at<float>(p.Xs))) {
        (void)cudaGetLastError();
        return LBG_ERR_CUDA;
    }
    int32_t *dA = wsA ? c.at<int32_t>(p.assign) : assign;
    // host X and assignment (always issued directly): the assignment goes back during the update
    const bool d2h_early = wX == 0 && assign && wA == 0 && !res;
    bool host_ok = true;
    Timer tm;
    if ((rc = tm.init(o.phase_ms != nullptr)) != LBG_OK) return rc;
    float *mu = c.at<float>(p.mu);
    auto issue = [&](cudaStream_t s) {
        Call k = c;
        k.s = s;
        tm.mark(0, s);
        launch_begin(dCi, N, L, mu, p.tc, st, s);   // also the initial state (cmax, rho zero)
        run_prepare(k, p, dCi, nullptr, N, mu, st, false);
        tm.mark(1, s);
        if (wX == 0) {
            if (!run_assign_host(k, p, c.at<float>(p.Xs), dCi, nullptr, N, mu, st, dA, o.test_expire_wait))
                host_ok = false;
        } else {
            run_assign(k, p, dX, dCi, nullptr, N, mu, st, dA, 0, -1, o.test_expire_wait);
        }
        tm.mark(2, s);
        run_exact(k, p, dX, nullptr, N, st, dA);
        tm.mark(3, s);
        if (d2h_early && !host_d2h_after(k, assign, dA, sizeof(int32_t) * M)) host_ok = false;
        launch_hist_ctl(dA, k.at<float>(p.e), M, p.R, p.CH, N, true, k.at<int32_t>(p.table),
                        k.at<double>(p.dpart), st, s);
        run_update(k, p, dX, nullptr, N, st, dA, dCi, dCo, false);
        if (o.reseed_empty)
            launch_reseed(k.at<int32_t>(p.off), nullptr, N, L, o.delta_reseed, dCo, st, false, s);
        if (res) LBG_COUNTED k_step_report<<<1, 1, 0, s>>>(st, res, 1);
        tm.mark(4, s);
    };
    if (o.phase_ms || wX == 0 || o.test_expire_wait) {   // direct: timed phases, host X pieces, test hook
        issue(c.s);
        if (!host_ok) return LBG_ERR_CUDA;
        CK(cudaGetLastError());
    } else {
        const SeqKey key{c.dev, 0, mode, (o.reseed_empty ? 1 : 0) | (p.grp << 8), M, L, N, p.total,
                         o.reseed_empty ? o.delta_reseed : 0.0, dX, dCi, dCo, dA, nullptr, res, c.ws};
        if ((rc = seq_run(c, key, issue)) != LBG_OK) return rc;
    }
    if (res) return end_async(c);
    if (hostC) CK(cudaMemcpyAsync(C_out, dCo, cbytes, cudaMemcpyDefault, c.s));
    if (d2h_early && !host_d2h_join(c)) return LBG_ERR_CUDA;
    if (assign && wA == 0 && !d2h_early)
        CK(cudaMemcpyAsync(assign, dA, sizeof(int32_t) * M, cudaMemcpyDeviceToHost, c.s));
    DevState h;
    CK(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, c.s));
    CK(cudaStreamSynchronize(c.s));
    tm.report(o.phase_ms, true);
    if (D) *D = h.D;
    if (o.n_exact) *o.n_exact = h.n_exact_last;
    return finish_status(h);
}

lbg_status lbg_distortion_backward(const float *X, int64_t M, int32_t L, const float *C, int32_t N,
                                   const int32_t *assign, float gD, float *dC, float *dX, double *D,
                                   const lbg_opts *opts)
{
    lbg_status rc = check_dims(M, L, N);
    if (rc != LBG_OK) return rc;
    if (!C || (M > 0 && (!X || !assign))) return LBG_ERR_ARG;
    const lbg_opts o = resolve(opts);
    const float *gdev = o.grad_scale_dev;
    lbg_step_result *res = o.result_dev;
    if (!gdev && !isfinite(gD)) return LBG_ERR_ARG;
    if (res && (D || o.phase_ms)) return LBG_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    Call c;
    if ((rc = begin(c, o)) != LBG_OK) return rc;
    const int wX = M > 0 ? where(X, c.dev) : 1, wC = where(C, c.dev);
    const int wA = M > 0 ? where(assign, c.dev) : 1;
    const int wdC = dC ? where(dC, c.dev) : 1, wdX = dX ? where(dX, c.dev) : 1;
    if (wX < 0 || wC < 0 || wA < 0 || wdC < 0 || wdX < 0) return LBG_ERR_ARG;
    if ((gdev || res) && (wX != 1 || wC != 1 || wA != 1 || wdC != 1 || wdX != 1 ||
                          (gdev && where(gdev, c.dev) != 1) || (res && where(res, c.dev) != 1)))
        return LBG_ERR_ARG;
    const bool hostC = wC == 0 || wdC == 0;
    const Plan p = make_plan(M, L, N, 0, wX == 0, wA == 0, hostC, wdX == 0, false);
    if ((rc = ensure_workspace(c, p.total)) != LBG_OK) return rc;
    const size_t cbytes = sizeof(float) * (size_t)N * L;
    DevState *st = c.at<DevState>(p.state);
    DevState h;
    CK(cudaMemsetAsync(st, 0, sizeof(DevState), c.s));   // no host memory: stays asynchronous
    const float *dXin = X;
    if (M > 0 && wX == 0) {
        CK(cudaMemcpyAsync(c.at<float>(p.Xs), X, sizeof(float) * M * L, cudaMemcpyHostToDevice, c.s));
        dXin = c.at<float>(p.Xs);
    }
    const float *dCin = C;
    if (wC == 0) {
        CK(cudaMemcpyAsync(c.at<float>(p.Cin), C, cbytes, cudaMemcpyHostToDevice, c.s));
        dCin = c.at<float>(p.Cin);
    }
    const int32_t *dA = assign;
    if (M > 0 && wA == 0) {
        CK(cudaMemcpyAsync(c.at<int32_t>(p.assign), assign, sizeof(int32_t) * M, cudaMemcpyHostToDevice,
                           c.s));
        dA = c.at<int32_t>(p.assign);
    }
    float *gX = dX ? (wdX ? dX : c.at<float>(p.Xhat)) : nullptr;
    float *gC = dC ? (wdC ? dC : c.at<float>(p.Cout)) : nullptr;
    Timer tm;
    if ((rc = tm.init(o.phase_ms != nullptr)) != LBG_OK) return rc;
    tm.mark(0, c.s);
    tm.mark(1, c.s);
    launch_grad_x(dXin, M, L, dCin, N, dA, gD, gdev, c.at<float>(p.e), gX, st, c.s);
    tm.mark(2, c.s);
    tm.mark(3, c.s);
    if (M > 0) {
        launch_hist_ctl(dA, c.at<float>(p.e), M, p.R, p.CH, N, gC != nullptr, c.at<int32_t>(p.table),
                        c.at<double>(p.dpart), st, c.s);
    }
    if (gC) {
        if (M > 0) {
            int32_t *table = c.at<int32_t>(p.table), *off = c.at<int32_t>(p.off);
            launch_scan_offsets(table, p.CH, N, c.at<int32_t>(p.counts), off, st, c.s);
            launch_scatter(dA, p.M, p.R, p.CH, table, off, nullptr, N, c.at<int32_t>(p.perm), st, false,
                           c.s);
            launch_cellsum(dXin, p.M, p.L, c.at<int32_t>(p.perm), off, nullptr, N, p.S,
                           c.at<float>(p.pieces), st, false, c.s);
            launch_combine_grad(c.at<float>(p.pieces), off, N, L, p.S, dCin, gD, gdev, gC, c.s);
        } else {
            CK(cudaMemsetAsync(gC, 0, cbytes, c.s));
        }
    }
    tm.mark(4, c.s);
    if (res) {
        if (M > 0)
            LBG_COUNTED k_step_report<<<1, 1, 0, c.s>>>(st, res, 1);
        else
            CK(cudaMemsetAsync(res, 0, sizeof(*res), c.s));   // D = 0, LBG_OK
        CK(cudaGetLastError());
        return end_async(c);
    }
    CK(cudaGetLastError());
    if (dC && wdC == 0) CK(cudaMemcpyAsync(dC, gC, cbytes, cudaMemcpyDeviceToHost, c.s));
    if (dX && wdX == 0 && M > 0)
        CK(cudaMemcpyAsync(dX, gX, sizeof(float) * M * L, cudaMemcpyDeviceToHost, c.s));
    CK(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, c.s));
    CK(cudaStreamSynchronize(c.s));
    tm.report(o.phase_ms, true);
    if (D) *D = M > 0 ? h.D : 0.0;
    return finish_status(h);
}

// ---- autotuner of the batched nearest-codevector launch
// Candidates: rows per work item x resident CTAs per SM.  A bucket (device, L,
// log2 of the largest N, log2 of the total rows) is calibrated once: every
// problem gets a full-size provisional codebook (its first rows, cyclically),
// the batched preparation runs, and one batched assignment per candidate is
// timed with CUDA events (best of two); the fastest is cached.  The choice
// changes only the speed: every row is computed the same way in each tile.
static std::map<std::array<int, 4>, std::pair<int, int>> g_tune;
static const int kTuneRows[4] = {128, 128, 64, 64};
static const int kTuneCtas[4] = {2, 1, 4, 2};

int ilog2_ceil(int64_t v)
{
    int k = 0;
    while (((int64_t)1 << k) < v) ++k;
    return k;
}

lbg_status calibrate_batched(const Call &c, int S, const std::vector<BatchSet> &hs, const BatchSet *dsets,
                             const int32_t *const *dP, int32_t *const *P, const int64_t *dtiles,
                             const int64_t *dtiles64, const std::vector<int64_t> &tiles,
                             const std::vector<int64_t> &tiles64, int *counter, const int32_t *N,
                             const int64_t *row_off, const float *dX, int L, int Lp, int &best_rows,
                             int &best_ctas, lbg_tune_report &rep)
{
    // data means (the centring of the preparation), then provisional codebooks
    launch_b_mean(dsets, S, dP[7], P[7][S], L, c.s);
    for (int s = 0; s < S; ++s) {
        const int64_t Ms = row_off[s + 1] - row_off[s];
        for (int64_t n = 0; n < N[s]; n += Ms) {
            const int64_t rows = (int64_t)N[s] - n < Ms ? (int64_t)N[s] - n : Ms;
            CK(cudaMemcpyAsync(hs[s].C + n * L, dX + row_off[s] * L, sizeof(float) * rows * L,
                               cudaMemcpyDeviceToDevice, c.s));
        }
    }
    std::vector<DevState> cal(S);
    for (int s = 0; s < S; ++s) init_state(cal[s], N[s]);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LBG_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LBG_ERR_CUDA;
    }
    lbg_status rc = LBG_OK;
    float best = INFINITY;
    rep.n_candidates = 4;
    for (int k = 0; k < 4 && rc == LBG_OK; ++k) {
        const int rows = kTuneRows[k], ctas = kTuneCtas[k];
        float t_best = INFINITY;
        for (int r = 0; r < 2 && rc == LBG_OK; ++r) {
            for (int s = 0; s < S; ++s)
                if (cudaMemcpyAsync(hs[s].st, &cal[s], sizeof(DevState), cudaMemcpyHostToDevice, c.s) !=
                    cudaSuccess)
                    rc = LBG_ERR_CUDA;
            launch_b_reset(dsets, S, counter, c.s);
            launch_b_prep(dsets, S, dP[2], P[2][S], L, Lp, c.s);
            cudaEventRecord(e0, c.s);
            launch_b_assign(dsets, S, rows == 64 ? dtiles64 : dtiles, rows == 64 ? tiles64[S] : tiles[S], L, Lp,
                            counter, rows, ctas, c.s);
            cudaEventRecord(e1, c.s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = LBG_ERR_CUDA;
            t_best = ms < t_best ? ms : t_best;
        }
        rep.cand_tile_rows[k] = rows;
        rep.cand_ctas_per_sm[k] = ctas;
        rep.cand_ms[k] = t_best;
        if (t_best < best) {
            best = t_best;
            best_rows = rows;
            best_ctas = ctas;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == LBG_OK && cudaGetLastError() != cudaSuccess) rc = LBG_ERR_CUDA;
    return rc;
}

lbg_status lbg_train_batched(int32_t S, const float *X, const int64_t *row_off, int32_t L,
                             const int32_t *N, double delta, double theta, float *C,
                             int32_t *assign, double *D, const lbg_opts *opts)
{
    if (S < 1 || !X || !row_off || !N || !C) return LBG_ERR_ARG;
    if (L < 1 || L > LBG_MAX_DIM) return LBG_ERR_ARG;
    if (!(delta >= 0.0) || !(theta >= 0.0) || !isfinite(delta) || !isfinite(theta))
        return LBG_ERR_ARG;
    if (row_off[0] != 0) return LBG_ERR_ARG;
    int64_t Mtot = 0, Ntot = 0;
    int NMAXB = 1;
    for (int s = 0; s < S; ++s) {
        const int64_t Ms = row_off[s + 1] - row_off[s];
        if (Ms < 1 || Ms > INT32_MAX) return LBG_ERR_ARG;
        if (N[s] < 1 || N[s] > LBG_MAX_CODEBOOK) return LBG_ERR_ARG;
        if (!is_pow2(N[s])) return LBG_ERR_NOT_POW2;
        Mtot += Ms;
        Ntot += N[s];
        NMAXB = N[s] > NMAXB ? N[s] : NMAXB;
    }
    const lbg_opts o = resolve(opts);
    if (o.precision != LBG_PREC_FP32) return LBG_ERR_UNSUPPORTED;
    if (o.tile_rows != 0 && o.tile_rows != 64 && o.tile_rows != 128) return LBG_ERR_ARG;
    if (o.ctas_per_sm != 0 && o.ctas_per_sm != 1 && o.ctas_per_sm != 2 && o.ctas_per_sm != 4)
        return LBG_ERR_ARG;
    if (o.ctas_per_sm == 4 && o.tile_rows != 64) return LBG_ERR_ARG;
    lbg_status rc;
    std::lock_guard<std::mutex> lock(g_mu);
    Call c;
    if ((rc = begin(c, o)) != LBG_OK) return rc;
    const int wX = where(X, c.dev), wC = where(C, c.dev), wA = assign ? where(assign, c.dev) : 0;
    if (wX < 0 || wC < 0 || wA < 0) return LBG_ERR_ARG;
    const int Lp = round_up(L, 4);

    // ---- workspace: one plan per problem, laid out one after another
    struct Sub {
        Plan p;
        size_t base;
    };
    std::vector<Sub> sub(S);
    size_t total = 0;
    auto take = [&](size_t bytes) {
        const size_t at = total;
        total += (bytes + 255) / 256 * 256;
        return at;
    };
    const size_t o_sets = take(sizeof(BatchSet) * S);
    const size_t o_pre = take(sizeof(int32_t) * (size_t)(S + 1) * 8);
    const size_t o_tiles = take(sizeof(int64_t) * (size_t)(S + 1));
    const size_t o_tiles64 = take(sizeof(int64_t) * (size_t)(S + 1));
    const size_t o_counter = take(sizeof(int) * 4);
    const size_t o_bar = take(sizeof(unsigned) * 4);   // grid barrier of the persistent pass
    const size_t o_X = wX == 0 ? take(sizeof(float) * (size_t)Mtot * L) : 0;
    const size_t o_C = wC == 0 ? take(sizeof(float) * (size_t)Ntot * L) : 0;
    const size_t o_A = take(sizeof(int32_t) * (size_t)Mtot);
    for (int s = 0; s < S; ++s) {
        const int64_t Ms = row_off[s + 1] - row_off[s];
        sub[s].p = make_plan(Ms, L, N[s], 0, false, true, false, false, false);
        sub[s].base = take(sub[s].p.total);
    }
    if ((rc = ensure_workspace(c, total)) != LBG_OK) return rc;
    char *ws = c.ws;
    const float *dX = X;
    if (wX == 0) {
        CK(cudaMemcpyAsync(ws + o_X, X, sizeof(float) * Mtot * L, cudaMemcpyHostToDevice, c.s));
        dX = reinterpret_cast<const float *>(ws + o_X);
    }
    float *dC = wC ? C : reinterpret_cast<float *>(ws + o_C);
    int32_t *dA = (assign && wA == 1) ? assign : reinterpret_cast<int32_t *>(ws + o_A);

    // ---- descriptors, states, block maps
    std::vector<BatchSet> hs(S);
    std::vector<int32_t> pre(8 * (S + 1), 0);
    std::vector<int64_t> tiles(S + 1, 0), tiles64(S + 1, 0);
    int32_t *P[8];
    for (int k = 0; k < 8; ++k) P[k] = pre.data() + k * (S + 1);
    std::vector<DevState> st0(S);
    int64_t coff = 0;
    for (int s = 0; s < S; ++s) {
        const Plan &p = sub[s].p;
        char *b = ws + sub[s].base;
        BatchSet &q = hs[s];
        q.X = dX + row_off[s] * L;
        q.M = p.M;
        q.N = p.N;
        q.NP = p.NP;
        q.CH = p.CH;
        q.G = p.G;
        q.R = p.R;
        q.S = p.S;
        q.C = dC + coff * L;
        q.Calt = reinterpret_cast<float *>(b + p.Calt);
        q.Cp = reinterpret_cast<float *>(b + p.Cp);
        q.kn = reinterpret_cast<float *>(b + p.kn);
        q.CT = reinterpret_cast<float *>(b + p.CT);
        q.mu = reinterpret_cast<float *>(b + p.mu);
        q.st = reinterpret_cast<DevState *>(b + p.state);
        q.assign = dA + row_off[s];
        q.flags = reinterpret_cast<int32_t *>(b + p.flags);
        q.table = reinterpret_cast<int32_t *>(b + p.table);
        q.counts = reinterpret_cast<int32_t *>(b + p.counts);
        q.off = reinterpret_cast<int32_t *>(b + p.off);
        q.perm = reinterpret_cast<int32_t *>(b + p.perm);
        q.e = reinterpret_cast<float *>(b + p.e);
        q.pieces = reinterpret_cast<float *>(b + p.pieces);
        q.qcell = reinterpret_cast<int32_t *>(b + p.qcell);
        q.cell_done = reinterpret_cast<int32_t *>(b + p.cell_done);
        q.nq = p.nq;
        q.dpart = reinterpret_cast<double *>(b + p.dpart);
        q.mpart = reinterpret_cast<double *>(b + p.mpart);
        coff += N[s];
        init_state(st0[s], 1);
        // blocks per problem of each batched launch
        const int64_t nq = p.nq;
        const int cnt[8] = {p.CH,
                            (N[s] + 31) / 32,
                            p.NP / 32,
                            (int)((nq + 7) / 8),
                            (int)(((int64_t)N[s] * L + 255) / 256),
                            (int)(((int64_t)(N[s] / 2 > 0 ? N[s] / 2 : 1) * L + 255) / 256),
                            (int)(((int64_t)N[s] * L + 255) / 256),
                            p.G};
        for (int k = 0; k < 8; ++k) P[k][s + 1] = P[k][s] + cnt[k];
        tiles[s + 1] = tiles[s] + (p.M + BM - 1) / BM;
        tiles64[s + 1] = tiles64[s] + (p.M + 63) / 64;
    }
    for (int s = 0; s < S; ++s)
        CK(cudaMemcpyAsync(hs[s].st, &st0[s], sizeof(DevState), cudaMemcpyHostToDevice, c.s));
    BatchSet *dsets = reinterpret_cast<BatchSet *>(ws + o_sets);
    int32_t *dpre = reinterpret_cast<int32_t *>(ws + o_pre);
    int64_t *dtiles = reinterpret_cast<int64_t *>(ws + o_tiles);
    int64_t *dtiles64 = reinterpret_cast<int64_t *>(ws + o_tiles64);
    int *counter = reinterpret_cast<int *>(ws + o_counter);
    CK(cudaMemcpyAsync(dsets, hs.data(), sizeof(BatchSet) * S, cudaMemcpyHostToDevice, c.s));
    CK(cudaMemcpyAsync(dpre, pre.data(), sizeof(int32_t) * pre.size(), cudaMemcpyHostToDevice, c.s));
    CK(cudaMemcpyAsync(dtiles, tiles.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice, c.s));
    CK(cudaMemcpyAsync(dtiles64, tiles64.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice, c.s));
    const int32_t *dP[8];
    for (int k = 0; k < 8; ++k) dP[k] = dpre + k * (S + 1);
    int max_groups = 0;
    for (int s = 0; s < S; ++s) max_groups += (int)((sub[s].p.M + 7) / 8);
    const bool vec = (reinterpret_cast<uintptr_t>(dX) & 15u) == 0;

    // ---- one persistent launch per pass, unless asked otherwise or it does not fit
    size_t pass_smem = 0, pass_phase_smem = 0;
    int pass_ctas = 0;
    if (!o.batched_per_phase && o.tile_rows == 0 && o.ctas_per_sm == 0) {
        pass_ctas = batch_pass_fit(S, L, NMAXB, &pass_phase_smem, &pass_smem);
        if (pass_ctas > 2) pass_ctas = 2;
    }
    unsigned *dbar = reinterpret_cast<unsigned *>(ws + o_bar);
    CK(cudaMemsetAsync(dbar, 0, sizeof(unsigned) * 4, c.s));
    CK(cudaMemsetAsync(counter, 0, sizeof(int) * 4, c.s));   // the persistent pass zeroes it after each pass
    BatchPass bp = {};
    bp.sets = dsets;
    bp.S = S;
    bp.L = L;
    bp.Lp = Lp;
    bp.NMAXB = NMAXB;
    bp.pre_prep = dP[2];
    bp.tot_prep = P[2][S];
    bp.pre_hist = dP[0];
    bp.tot_hist = P[0][S];
    bp.pre_scan = dP[1];
    bp.tot_scan = P[1][S];
    bp.pre_cellsum = dP[3];
    bp.tot_cellsum = P[3][S];
    bp.pre_combine = dP[4];
    bp.tot_combine = P[4][S];
    bp.pre_split = dP[5];
    bp.tot_split = P[5][S];
    bp.pre_copy = dP[6];
    bp.tot_copy = P[6][S];
    bp.pre_tiles = dtiles64;
    bp.ntiles = tiles64[S];
    bp.counter = counter;
    bp.bar = dbar;
    bp.theta = theta;
    bp.delta = delta;
    bp.max_passes = o.max_passes;
    bp.mult = o.split_multiplicative != 0;
    bp.vec = vec && (reinterpret_cast<uintptr_t>(dC) & 15u) == 0;
    // small stages in the one-launch pass: every row against every codevector (the per-phase
    // launches keep the tiled search; both give the same bits)
    bp.direct_max = bp.vec && (L & 3) == 0 && L <= 64 ? DIRECT_MAX_F32 : 0;
    bp.phase_smem = pass_phase_smem;

    // ---- tile of the batched nearest-codevector launch (lbg_opts.autotune)
    int tile_rows = 128, ctas = 2;
    lbg_tune_report report;
    memset(&report, 0, sizeof(report));
    if (pass_ctas > 0) {
        tile_rows = 64;     // the persistent pass: two 64-row tiles per CTA, its resident CTAs
        ctas = pass_ctas;
    } else if (o.tile_rows != 0 || o.ctas_per_sm != 0) {
        tile_rows = o.tile_rows != 0 ? o.tile_rows : 128;
        ctas = o.ctas_per_sm != 0 ? o.ctas_per_sm : (tile_rows == 64 ? 4 : 2);
    } else if (o.autotune) {
        const std::array<int, 4> key = {c.dev, L, ilog2_ceil(NMAXB), ilog2_ceil((int64_t)Mtot)};
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            tile_rows = it->second.first;
            ctas = it->second.second;
            report.from_cache = 1;
        } else if ((rc = calibrate_batched(c, S, hs, dsets, dP, P, dtiles, dtiles64, tiles, tiles64, counter,
                                           N, row_off, dX, L, Lp, tile_rows, ctas, report)) != LBG_OK) {
            return rc;
        } else {
            g_tune[key] = {tile_rows, ctas};
            // the calibration ran passes on scratch states: start from the initial ones
            for (int s = 0; s < S; ++s)
                CK(cudaMemcpyAsync(hs[s].st, &st0[s], sizeof(DevState), cudaMemcpyHostToDevice, c.s));
        }
    }
    report.tile_rows = tile_rows;
    report.ctas_per_sm = ctas;
    const int64_t *dtiles_use = tile_rows == 64 ? dtiles64 : dtiles;
    const int64_t ntiles_use = tile_rows == 64 ? tiles64[S] : tiles[S];
    Timer tm;
    if ((rc = tm.init(o.phase_ms != nullptr)) != LBG_OK) return rc;
    tm.mark(0, c.s);
    launch_b_mean(dsets, S, dP[7], P[7][S], L, c.s);

    // ---- one batched pass, recorded once into a graph and replayed
    bool pass_refused = false, in_capture = false, capture_refused = false;
    auto pass = [&](cudaStream_t st) {
        if (pass_ctas > 0 && !pass_refused) {
            if (launch_b_pass(bp, pass_ctas, pass_smem, st)) return;
            // refused while recording: the recording is dropped and the pass launched directly;
            // refused directly: the per-phase launches from now on
            if (in_capture) {
                capture_refused = true;
                return;
            }
            pass_refused = true;
        }
        launch_b_reset(dsets, S, counter, st);
        launch_b_prep(dsets, S, dP[2], P[2][S], L, Lp, st);
        launch_b_assign(dsets, S, dtiles_use, ntiles_use, L, Lp, counter, tile_rows, ctas, st);
        launch_b_exact(dsets, S, L, Lp, max_groups, st);
        launch_b_hist(dsets, S, dP[0], P[0][S], NMAXB, st);
        launch_b_ctl(dsets, S, theta, o.max_passes, st);
        launch_b_scan(dsets, S, dP[1], P[1][S], st);
        launch_b_offsets(dsets, S, st);
        launch_b_scatter(dsets, S, dP[0], P[0][S], NMAXB, st);
        launch_b_cellsum(dsets, S, dP[3], P[3][S], L, vec, st);
        launch_b_combine(dsets, S, dP[4], P[4][S], L, st);
        launch_b_split(dsets, S, dP[5], P[5][S], L, delta, o.split_multiplicative != 0, st);
        launch_b_advance(dsets, S, dP[6], P[6][S], L, st);
    };
    int stages = 1;
    for (int s = 0; s < S; ++s) {
        int k = 1;
        for (int n = 1; n < N[s]; n *= 2) ++k;
        stages = k > stages ? k : stages;
    }
    const int64_t max_total = (int64_t)stages * o.max_passes;
    GraphPass gp;
    in_capture = true;
    gp.build(c.s, pass);   // falls back to direct launches if capture is not possible
    in_capture = false;
    if (capture_refused) gp.drop();
    std::vector<DevState> hst(S);
    lbg_status out = LBG_OK;
    int64_t issued = 0;
    int batch = 2;
    for (;;) {
        for (int b = 0; b < batch && issued < max_total; ++b, ++issued) gp.run(c.s, pass);
        if (cudaGetLastError() != cudaSuccess) {
            out = LBG_ERR_CUDA;
            break;
        }
        bool all = true;
        uint32_t err = 0;
        for (int s = 0; s < S; ++s)
            if (cudaMemcpyAsync(&hst[s], hs[s].st, sizeof(DevState), cudaMemcpyDeviceToHost, c.s) !=
                cudaSuccess)
                out = LBG_ERR_CUDA;
        if (cudaStreamSynchronize(c.s) != cudaSuccess) out = LBG_ERR_CUDA;
        if (out != LBG_OK) {
            (void)cudaGetLastError();
            break;
        }
        for (int s = 0; s < S; ++s) {
            all = all && hst[s].finished;
            err |= hst[s].err;
        }
        if (all || err || issued >= max_total) break;
        if (batch < 32) batch *= 2;
    }
    tm.mark(4, c.s);
    report.persistent = pass_ctas > 0 && !pass_refused;
    if (o.tune_report) *o.tune_report = report;
    if (out != LBG_OK) return out;
    if (wC == 0) CK(cudaMemcpyAsync(C, dC, sizeof(float) * Ntot * L, cudaMemcpyDeviceToHost, c.s));
    if (assign && wA == 0)
        CK(cudaMemcpyAsync(assign, dA, sizeof(int32_t) * Mtot, cudaMemcpyDeviceToHost, c.s));
    CK(cudaStreamSynchronize(c.s));
    tm.report(o.phase_ms, false);
    DevState agg;
    init_state(agg, 0);
    int maxp = 0;
    for (int s = 0; s < S; ++s) {
        if (D) D[s] = hst[s].D;
        agg.err |= hst[s].err;
        agg.warn |= hst[s].warn;
        maxp = hst[s].total > maxp ? hst[s].total : maxp;
        if (!hst[s].finished && !hst[s].err) return LBG_ERR_CUDA;
    }
    if (o.n_records) *o.n_records = maxp;
    return finish_status(agg);
}

lbg_status lbg_train(const float *X, int64_t M, int32_t L, int32_t N, double delta, double theta,
                     float *C, int32_t n_init, int32_t *assign, double *D, const lbg_opts *opts)
{
    lbg_status rc = check_dims(M, L, N);
    if (rc != LBG_OK) return rc;
    if (M < 1 || !X || !C) return LBG_ERR_ARG;
    if (!(delta >= 0.0) || !(theta >= 0.0) || !isfinite(delta) || !isfinite(theta))
        return LBG_ERR_ARG;
    if (!is_pow2(N)) return LBG_ERR_NOT_POW2;
    if (n_init < 0 || n_init > N) return LBG_ERR_ARG;
    if (n_init > 0 && !is_pow2(n_init)) return LBG_ERR_NOT_POW2;
    const lbg_opts o = resolve(opts);
    const int mode = precision_mode(o, L);
    if (mode < 0) return (lbg_status)mode;
    std::lock_guard<std::mutex> lock(g_mu);
    Call c;
    if ((rc = begin(c, o)) != LBG_OK) return rc;
    const int wX = where(X, c.dev), wC = where(C, c.dev);
    const int wA = assign ? where(assign, c.dev) : 0;
    if (wX < 0 || wC < 0 || wA < 0) return LBG_ERR_ARG;
    // pass trace buffers: device memory of this device, with room for >= 1 pass
    if ((o.trace_C || o.trace_assign) &&
        (o.trace_cap < 1 || (o.trace_C && where(o.trace_C, c.dev) != 1) ||
         (o.trace_assign && where(o.trace_assign, c.dev) != 1)))
        return LBG_ERR_ARG;
    const bool tracing = o.records || o.trace_C || o.trace_assign;
    int stages = 1;
    for (int n = n_init > 0 ? n_init : 1; n < N; n *= 2) ++stages;
    const int64_t max_total = (int64_t)stages * o.max_passes;
    const int max_rec = o.max_records < max_total ? o.max_records : (int)max_total;
    Plan p = make_plan(M, L, N, max_rec, wX == 0, !(assign && wA == 1), false, false, mode == 1);
    p.grp = o.tc_group;
    if ((rc = ensure_workspace(c, p.total)) != LBG_OK) return rc;
    DevState *st = c.at<DevState>(p.state);
    DevState h;
    init_state(h, n_init > 0 ? n_init : 1);
    // stages of at most direct_max cells: every row against every codevector
    // (k_assign_direct) instead of the tiled search, its certificate and re-scoring
    const int direct_max = direct_supported(L, wX == 0 ? c.at<float>(p.Xs) : X, c.at<float>(p.Ccur))
                               ? (p.tc ? DIRECT_MAX_TC : DIRECT_MAX_F32)
                               : 0;
    h.direct_max = direct_max;
    CK(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, c.s));
    const float *dX = X;
    if (wX == 0) {
        CK(cudaMemcpyAsync(c.at<float>(p.Xs), X, sizeof(float) * M * L, cudaMemcpyHostToDevice, c.s));
        dX = c.at<float>(p.Xs);
    }
    float *Ccur = c.at<float>(p.Ccur), *Calt = c.at<float>(p.Calt), *mu = c.at<float>(p.mu);
    int32_t *dA = (assign && wA == 1) ? assign : c.at<int32_t>(p.assign);
    if (n_init > 0)
        CK(cudaMemcpyAsync(Ccur, C, sizeof(float) * (size_t)n_init * L, cudaMemcpyDefault, c.s));
    Timer tm;
    if ((rc = tm.init(o.phase_ms != nullptr)) != LBG_OK) return rc;
    tm.mark(0, c.s);
    // Initialization (Algorithm 1): centroid of the training set; it is also
    // the centring vector of every allocation of the run.
    launch_mean(dX, M, L, c.at<double>(p.mpart), p.G, mu, n_init > 0 ? nullptr : Ccur, st, c.s);
    if (p.tc) launch_round_mu(mu, L, c.s);   // integer centring keeps integer samples exact in BF16
    const int32_t *n_dev = &st->n_cur;
    PassRecord *rec = c.at<PassRecord>(p.rec);
    int64_t issued = 0;
    int batch = 2;
    DevState *hs = nullptr;
    CK(cudaMallocHost(&hs, sizeof(DevState)));
    lbg_status out = LBG_OK;
    auto pass = [&](cudaStream_t sst) {
        Call cs = c;
        cs.s = sst;
        if (tracing) launch_trace_begin(st, Ccur, N, L, o.trace_C, o.trace_cap, sst);
        run_prepare(cs, p, Ccur, n_dev, N, mu, st);
        run_assign(cs, p, dX, Ccur, n_dev, N, mu, st, dA);
        if (direct_max > 0) launch_assign_direct(dX, M, L, Ccur, n_dev, N, st, dA, cs.at<float>(p.e), sst);
        run_exact(cs, p, dX, n_dev, N, st, dA);
        launch_hist(dA, cs.at<float>(p.e), M, p.R, p.CH, n_dev, N, true, cs.at<int32_t>(p.table),
                    cs.at<double>(p.dpart), st, true, sst);
        launch_ctl(cs.at<double>(p.dpart), p.CH, st, MODE_TRAIN, theta, o.max_passes, N, rec,
                   max_rec, sst);
        run_update(cs, p, dX, n_dev, N, st, dA, Ccur, Ccur, true);
        if (o.reseed_empty)
            launch_reseed(cs.at<int32_t>(p.off), n_dev, N, L, delta, Ccur, st, true, sst);
        launch_split(Ccur, Calt, N, L, delta, o.split_multiplicative != 0, st, sst);
        launch_advance(Calt, Ccur, N, L, st, sst);
        if (tracing)
            launch_trace_end(st, dA, M, cs.at<int32_t>(p.counts), o.records ? rec : nullptr, max_rec,
                             o.trace_assign, o.trace_cap, sst);
    };
    GraphPass gp;
    gp.build(c.s, pass);
    for (;;) {
        for (int b = 0; b < batch && issued < max_total; ++b, ++issued) gp.run(c.s, pass);
        if (cudaGetLastError() != cudaSuccess) {
            out = LBG_ERR_CUDA;
            break;
        }
        if (cudaMemcpyAsync(hs, st, sizeof(DevState), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
            cudaStreamSynchronize(c.s) != cudaSuccess) {
            (void)cudaGetLastError();
            out = LBG_ERR_CUDA;
            break;
        }
        if (hs->finished || hs->err || issued >= max_total) break;
        if (batch < 32) batch *= 2;
    }
    tm.mark(4, c.s);
    if (out == LBG_OK) {
        h = *hs;
        if (!h.finished && !h.err) out = LBG_ERR_CUDA;   // pass bound reached without finishing
    }
    cudaFreeHost(hs);
    if (out != LBG_OK) return out;
    CK(cudaMemcpyAsync(C, Ccur, sizeof(float) * (size_t)N * L, cudaMemcpyDefault, c.s));
    if (assign && wA == 0)
        CK(cudaMemcpyAsync(assign, dA, sizeof(int32_t) * M, cudaMemcpyDeviceToHost, c.s));
    const int nrec = h.total < max_rec ? h.total : max_rec;
    if (o.records && nrec > 0) {
        static_assert(sizeof(PassRecord) == sizeof(lbg_pass_record), "record layout");
        CK(cudaMemcpyAsync(o.records, rec, sizeof(PassRecord) * nrec, cudaMemcpyDeviceToHost, c.s));
    }
    CK(cudaStreamSynchronize(c.s));
    tm.report(o.phase_ms, false);
    if (o.n_records) *o.n_records = h.total;
    if (D) *D = h.D;
    return finish_status(h);
}

}  // extern "C"
