// lbg_noalloc.cu -- vq_encode_noalloc: nearest-codevector encoding that
// allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need to
// encode: a serving loop that reserved its whole memory budget up front and
// must not take a cudaMalloc latency spike (cudaMalloc can synchronise the
// device) in steady state; a process whose framework allocator already holds
// nearly all device memory, so a raw cudaMalloc would fail; or code that is
// certified to allocate only during initialisation.  For them this entry
// point keeps every scratch array in one fixed file-scope __device__ array,
// which exists on every GPU that loads the library until the process exits.
//
// The scratch (prepared codebook, per-row distances and uncertified-row list
// of one chunk of rows, distortion partials, call state) lives in
// g_noalloc_scratch.  Host code cannot use that symbol as a device address:
// the address is looked up with cudaGetSymbolAddress once per device (on the
// first call made with that device current) and passed to the kernels.
// Every call reuses the same array and leaves its contents behind; each call
// re-initialises what must start at zero.  Calls whose work overlaps on the
// GPU (two streams, or two host threads) race on the array.
#include "lbgvq.h"
#include "lbg_internal.cuh"

#include <mutex>

using namespace lbg;

namespace {

// Limits of the fixed scratch (stated in include/lbgvq.h).
constexpr int NA_MAX_N = 4096;
constexpr int NA_MAX_L = LBG_MAX_DIM;            // 128
constexpr int64_t NA_ROWS = 1 << 20;             // rows per chunk of the input
constexpr int NA_NP = NA_MAX_N;                  // padded codebook rows (multiple of BN)
constexpr int NA_LP = NA_MAX_L;                  // padded dimension (multiple of 4)

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t OFF_STATE = 0;
constexpr size_t OFF_DTOT = OFF_STATE + align256(sizeof(DevState));
constexpr size_t OFF_MU = OFF_DTOT + align256(sizeof(double));
constexpr size_t OFF_DPART = OFF_MU + align256(sizeof(float) * NA_LP);
constexpr size_t OFF_KN = OFF_DPART + align256(sizeof(double) * HIST_CHUNKS_MAX);
constexpr size_t OFF_CP = OFF_KN + align256(sizeof(float) * NA_NP);
constexpr size_t OFF_CT = OFF_CP + align256(sizeof(float) * (size_t)(NA_NP / BN) * (NA_LP + 1) * BN);
constexpr size_t OFF_E = OFF_CT + align256(sizeof(float) * (size_t)NA_LP * NA_NP);
constexpr size_t OFF_FLAGS = OFF_E + align256(sizeof(float) * (size_t)NA_ROWS);
constexpr size_t NA_USED = OFF_FLAGS + align256(sizeof(int32_t) * (size_t)NA_ROWS);
constexpr size_t NA_BYTES = (size_t)16 << 20;    // 16 MiB
static_assert(NA_USED <= NA_BYTES, "fixed scratch too small for its stated limits");

}  // namespace

// The fixed scratch of vq_encode_noalloc (16 MiB on every device that loads the library).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {

std::mutex g_na_mu;
char *g_na_ptr[64] = {};

__global__ void k_noalloc_begin(DevState *st, double *dtot, int N)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DevState s = {};
    s.n_cur = N;
    s.D_prev = INFINITY;
    *st = s;
    *dtot = 0.0;
}

// After each chunk: add its distortion (k_ctl has already reset the row counters).
__global__ void k_noalloc_accum(DevState *st, double *dtot)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *dtot += st->D;
}

struct NaResult {
    uint32_t err;
    double D;
};

__global__ void k_noalloc_end(const DevState *st, const double *dtot, NaResult *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    out->err = st->err;
    out->D = *dtot;
}

// Device address of g_noalloc_scratch on the current device (looked up once).
lbg_status scratch_address(int dev, char **out)
{
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (dev < 0 || dev >= 64) return LBG_ERR_UNSUPPORTED;
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return LBG_ERR_CUDA;
        }
        g_na_ptr[dev] = static_cast<char *>(p);
    }
    *out = g_na_ptr[dev];
    return LBG_OK;
}

bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" lbg_status vq_encode_noalloc(const float *X, int64_t M, int32_t L, const float *C,
                                        int32_t N, int32_t *idx, double *D, void *stream)
{
    if (M < 0 || M > INT32_MAX || L < 1 || N < 1) return LBG_ERR_ARG;
    if (!C || (M > 0 && (!X || !idx))) return LBG_ERR_ARG;
    if (N > NA_MAX_N || L > NA_MAX_L) return LBG_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return LBG_ERR_CUDA;
    }
    if (!on_device(C, dev) || (M > 0 && (!on_device(X, dev) || !on_device(idx, dev))))
        return LBG_ERR_ARG;
    char *base = nullptr;
    lbg_status rc = scratch_address(dev, &base);
    if (rc != LBG_OK) return rc;
    if (M == 0) {
        if (D) *D = 0.0;
        return LBG_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevState *st = reinterpret_cast<DevState *>(base + OFF_STATE);
    double *dtot = reinterpret_cast<double *>(base + OFF_DTOT);
    float *mu = reinterpret_cast<float *>(base + OFF_MU);
    double *dpart = reinterpret_cast<double *>(base + OFF_DPART);
    float *kn = reinterpret_cast<float *>(base + OFF_KN);
    float *Cp = reinterpret_cast<float *>(base + OFF_CP);
    float *CT = reinterpret_cast<float *>(base + OFF_CT);
    float *e = reinterpret_cast<float *>(base + OFF_E);
    int32_t *flags = reinterpret_cast<int32_t *>(base + OFF_FLAGS);
    const int Lp = round_up(L, 4);

    LBG_COUNTED k_noalloc_begin<<<1, 32, 0, s>>>(st, dtot, N);
    launch_codebook_mean(C, N, L, mu, s);
    launch_prep(C, N, nullptr, N, L, Lp, mu, Cp, kn, CT, NA_NP, st, s);
    for (int64_t r0 = 0; r0 < M; r0 += NA_ROWS) {
        const int64_t mc = M - r0 < NA_ROWS ? M - r0 : NA_ROWS;
        const float *Xc = X + r0 * L;
        int32_t *ic = idx + r0;
        launch_assign(Xc, mc, L, Lp, Cp, kn, nullptr, N, mu, C, st, ic, e, flags, s);
        launch_exact(Xc, L, Lp, CT, nullptr, N, st, flags, ic, e, mc, s);
        // distortion of the chunk: same chunking rule as the cached-workspace path
        int64_t ch = (mc + 1023) / 1024;
        if (ch > HIST_CHUNKS_MAX) ch = HIST_CHUNKS_MAX;
        if (ch < 1) ch = 1;
        int64_t R = round_up64((mc + ch - 1) / ch, 256);
        if (R < 256) R = 256;
        const int CH = (int)((mc + R - 1) / R);
        launch_hist(ic, e, mc, R, CH, nullptr, N, false, nullptr, dpart, st, false, s);
        launch_ctl(dpart, CH, st, MODE_STEP, 0.0, 1, N, nullptr, 0, s);
        LBG_COUNTED k_noalloc_accum<<<1, 32, 0, s>>>(st, dtot);
    }
    NaResult *res = reinterpret_cast<NaResult *>(base + OFF_DPART);   // dpart is free again
    LBG_COUNTED k_noalloc_end<<<1, 32, 0, s>>>(st, dtot, res);
    NaResult h;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return LBG_ERR_CUDA;
    }
    if (h.err & ERR_NONFINITE) return LBG_ERR_NONFINITE;
    if (h.err & ERR_TIMEOUT) return LBG_ERR_TIMEOUT;
    if (h.err & ERR_INTERNAL) return LBG_ERR_CUDA;
    if (D) *D = h.D;
    return LBG_OK;
}
