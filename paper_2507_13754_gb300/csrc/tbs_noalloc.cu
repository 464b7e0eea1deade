// tbs_noalloc.cu -- one application of G that allocates no device memory.
//
// tbs_apply_green needs a plan, and creating a plan calls cudaMalloc.  Some
// callers cannot do that: code running while a CUDA graph is being captured,
// code inside a memory pool or allocator that must not re-enter the
// allocator, and real-time or embedded loops where every device allocation
// is made once at start-up by someone else.  For them this file provides
// tbs_apply_green_noalloc: the same row and column kernels, but their scratch
// (the two N x M intermediates of the FFT convolution and the twiddle
// tables) lives in one file-scope __device__ array of fixed size instead of
// plan-owned buffers.
//
// Limits and sharing:
//   * N <= TBS_NOALLOC_MAX_N (256), hence M <= 512.  The array holds
//     2 x 256 x 512 complex64 intermediates, twiddle tables for every M
//     from 16 to 512, a copy of the caller's spectrum quadrant at the
//     kernels' row stride and an error word: 2,635,680 bytes, kept by every
//     GPU that loads the library until the process exits.
//   * All calls share the array, so calls that overlap on the GPU (on
//     different streams, or from different host threads without ordering)
//     race on it.  Of its contents only the error word has to start at
//     zero, and each call clears it on its stream (cudaMemsetAsync, which
//     allocates nothing); every other row a call reads, it wrote before.
//   * The kernels' waits for their copies are bounded; one that runs out
//     (a lost copy, never expected) records it in the error word and leaves
//     `out` undefined.  The call returns before its kernels run, so it
//     cannot report that.
//   * The set-up below is per device and per process lifetime of the
//     library's module: after cudaDeviceReset the array and the kernels'
//     attributes are gone, and this entry point must not be used again in
//     that process.
//   * The first call on a device sets that device up (it takes the array's
//     device address with cudaGetSymbolAddress, fills the twiddle tables and
//     waits for that on the call's stream, and sets the kernels' shared
//     memory limits).  Make that first call outside any stream capture.
#include "tbs.h"
#include "tbs_fft.cuh"
#include "tbs_internal.h"

#include <mutex>
#include <stdio.h>
#include <string.h>

using namespace tbs;

namespace {

constexpr int NA_MAX_N = TBS_NOALLOC_MAX_N;
constexpr int NA_MAX_M = 2 * NA_MAX_N;                 // padded size for N = 256
constexpr size_t NA_PLANE = (size_t)NA_MAX_N * NA_MAX_M;  // complex64 per intermediate
// twiddle tables for M = 16, 32, ..., 512; the table of M starts at M - 16
constexpr size_t NA_TW = 2 * NA_MAX_M - 16;
// the caller's spectrum quadrant, repacked to the kernels' row stride
constexpr size_t NA_GHAT = (size_t)(NA_MAX_M / 2 + 1) * ghat_stride(NA_MAX_M);
constexpr size_t NA_DATA = 2 * NA_PLANE + NA_TW + NA_GHAT;
constexpr size_t NA_TOTAL = NA_DATA + 2;  // + the error word (16 bytes)

// the scratch: [X plane][W plane][twiddle tables][repacked quadrant][error word]
static __device__ __align__(256) float2 g_noalloc_scratch[NA_TOTAL];

constexpr int NA_MAX_DEVICES = 64;

struct NoallocDevice {
    bool ready = false;
    cudaError_t err = cudaSuccess;
    float2 *base = nullptr;      // device address of g_noalloc_scratch
    int grid[10] = {0};          // persistent column grid for M = 16 << i
};

std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[NA_MAX_DEVICES];

// exp(-2 pi i k / M) for every M, straight from FP64 sincospi
__global__ void noalloc_twiddle_kernel(float2 *tables) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int)NA_TW) return;
    int M = 16;
    while (i >= 2 * M - 16) M *= 2;  // table of M covers [M - 16, 2M - 16)
    const int k = i - (M - 16);
    double s, c;
    sincospi(2.0 * (double)k / (double)M, &s, &c);
    tables[i] = make_float2((float)c, (float)-s);
}

int padded(int n) {
    int m = 16;
    while (m < 2 * n - 1) m *= 2;
    return m;
}

int log2_16(int m) {
    int i = 0;
    while ((16 << i) < m) i++;
    return i;
}

tbs_status na_fail(tbs_status s, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess)
        snprintf(buf, sizeof(buf), "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof(buf), "%s", msg);
    set_last_error(buf);  // reported by tbs_last_error()
    return s;
}

// One-time set-up of the current device; returns its state or nullptr.
NoallocDevice *noalloc_device(cudaStream_t s, cudaError_t *err) {
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice &d = g_noalloc_dev[dev];
    if (d.ready) return &d;
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
        *err = e;
        return nullptr;
    }
    d.base = (float2 *)ptr;
    noalloc_twiddle_kernel<<<(int)((NA_TW + 255) / 256), 256, 0, s>>>(d.base + 2 * NA_PLANE);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        *err = e;
        return nullptr;
    }
    int sms = 1;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
        *err = e;
        return nullptr;
    }
    for (int i = 0, M = 16; M <= NA_MAX_M; i++, M *= 2) {
        if ((e = set_row_smem_attr(M)) != cudaSuccess || (e = set_col_smem_attr(M)) != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        d.grid[i] = sms * col_resident_blocks_per_sm(M, 0);
    }
    d.ready = true;
    return &d;
}

}  // namespace

extern "C" tbs_status tbs_apply_green_noalloc(int32_t n, const float *ghat, const float *f, float *out,
                                              int32_t conj_kernel, void *stream) {
    if (n < 2 || n > NA_MAX_N)
        return na_fail(TBS_ERR_UNSUPPORTED_SIZE,
                       "tbs_apply_green_noalloc: n outside [2, TBS_NOALLOC_MAX_N = 256]");
    if (!ghat || !f || !out) return na_fail(TBS_ERR_INVALID_ARG, "tbs_apply_green_noalloc: NULL pointer");
    if (f == out) return na_fail(TBS_ERR_INVALID_ARG, "tbs_apply_green_noalloc: f and out may not alias");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    NoallocDevice *d = noalloc_device(s, &e);
    if (!d) return na_fail(TBS_ERR_CUDA, "tbs_apply_green_noalloc: device set-up failed", e);
    const int M = padded(n);
    float2 *X = d->base;
    float2 *W = d->base + NA_PLANE;
    const float2 *tw = d->base + 2 * NA_PLANE + (M - 16);

    RowArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.W = W;
    ra.src = (const float2 *)f;
    ra.X = X;
    ra.psi = (float2 *)out;
    ra.tw = tw;
    ra.gate.mode = GATE_ALL;
    ra.n = n;
    ra.max_terms = 1;
    ra.l1_row = -1;
    ColArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.X = X;
    ca.W = W;
    // the caller's quadrant rows (M/2 + 1 wide) -> the kernels' stride
    float2 *ghq = d->base + 2 * NA_PLANE + NA_TW;
    const size_t qw = (size_t)(M / 2 + 1) * sizeof(float2);
    if ((e = cudaMemcpy2DAsync(ghq, (size_t)ghat_stride(M) * sizeof(float2), ghat, qw, qw, M / 2 + 1,
                               cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return na_fail(TBS_ERR_CUDA, "tbs_apply_green_noalloc: spectrum copy", e);
    ca.ghq = ghq;
    ca.tw = tw;
    ca.gate.mode = GATE_ALL;
    ca.n = n;
    ca.nrhs = 1;
    ca.num_sms = d->grid[log2_16(M)];
    // the error word, cleared for this call (stream-ordered after any earlier call)
    int *errw = reinterpret_cast<int *>(d->base + NA_DATA);
    if ((e = cudaMemsetAsync(errw, 0, 4 * sizeof(int), s)) != cudaSuccess)
        return na_fail(TBS_ERR_CUDA, "tbs_apply_green_noalloc: error word", e);
    ra.err = errw;
    ca.err = errw;
    ColMaps maps;  // host-side descriptors, passed by value to the kernel
    if ((e = col_tensor_maps(&maps, X, W, n, M, 1, 0)) != cudaSuccess)
        return na_fail(TBS_ERR_CUDA, "tbs_apply_green_noalloc: tensor maps", e);
    if ((e = launch_row(ROW_SRC, M, 1, ra, s)) != cudaSuccess ||
        (e = launch_col(M, 1, conj_kernel != 0, ca, &maps, 0, s)) != cudaSuccess ||
        (e = launch_row(ROW_OUT, M, 1, ra, s)) != cudaSuccess)
        return na_fail(TBS_ERR_CUDA, "tbs_apply_green_noalloc: launch failed", e);
    return TBS_OK;
}
