// Allocation-free conserved totals.
//
// weno_conserved_totals_noalloc sums sum_cells U dV per variable of a state
// the caller owns, like weno_conserved_totals does for a context's state, but
// without allocating anything: its per-block partial sums live in the
// file-scope device array below, which every GPU that loads the library
// holds until the process exits.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// want the totals -- applications whose device memory belongs to their own
// pool or allocator, and time-stepping loops with a fixed memory budget that
// must not allocate (cudaMalloc can also synchronize the device, which such
// a loop cannot afford mid-step).  Such a caller passes the state and a
// device buffer for the result; nothing else is needed.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/weno_is.h"

namespace {

constexpr int kChunk = 4096;                 // cells summed by one block
constexpr int kMaxBlocks = 16384;            // partial-sum slots per variable
constexpr int kMaxVars = 5;
constexpr long long kMaxCells = (long long)kChunk * kMaxBlocks;   // 67,108,864

// Partial sums [block][variable].  Shared by every call on a device; each
// call overwrites the slots it uses before reading them.
static __device__ __align__(256) double g_partial_scratch[kMaxBlocks * kMaxVars];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

template <typename T, int NV>
__global__ void __launch_bounds__(256) k_totals_chunk(const T* __restrict__ U, long long cells,
                                                      double* __restrict__ partial)
{
    const long long c0 = (long long)blockIdx.x * kChunk;
    long long c1 = c0 + kChunk;
    if (c1 > cells) c1 = cells;
    double s[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = 0.0;
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] += (double)U[v * cells + c];
    }
    __shared__ double red[8][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double w = s[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][v] = w;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double w = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) w += red[q][threadIdx.x];
        partial[(long long)blockIdx.x * NV + threadIdx.x] = w;
    }
}

template <int NV>
__global__ void k_totals_chunk_final(const double* __restrict__ partial, int nblk, double dV,
                                     double* __restrict__ out)
{
    // one warp per variable; lanes stride over the blocks, fixed-order tree
    const int v = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += partial[(long long)b * NV + v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[v] = s * dV;
}

template <typename T, int NV>
cudaError_t launch_totals(const void* U, long long cells, int nblk, double dV, double* scratch, double* out,
                          cudaStream_t s)
{
    k_totals_chunk<T, NV><<<nblk, 256, 0, s>>>(reinterpret_cast<const T*>(U), cells, scratch);
    k_totals_chunk_final<NV><<<NV, 32, 0, s>>>(scratch, nblk, dV, out);
    return cudaGetLastError();
}

// Device address of the scratch array for the current device.  The address
// is looked up (cudaGetSymbolAddress, with the device current) on every call
// made while `s` is not being captured, so a module reloaded after a device
// reset is found again; while `s` is being captured the address cached by
// the last lookup on this device is used, and without one the call fails.
cudaError_t scratch_for_current_device(cudaStream_t s, double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partial_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    } else if (g_scratch_addr[dev] == nullptr) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" weno_status weno_conserved_totals_noalloc(int dim, const int* n, const double* dx, int precision,
                                                     const void* U_dev, double* totals_dev, void* stream)
{
    if (dim < 1 || dim > 3 || !n || !dx || !U_dev || !totals_dev) return WENO_ERR_INVALID_ARG;
    if (precision < WENO_FP64 || precision > WENO_MIXED) return WENO_ERR_INVALID_ARG;
    long long cells = 1;
    double dV = 1.0;
    for (int d = 0; d < dim; ++d) {
        // cells stays <= kMaxCells, so the product cannot overflow
        if (n[d] < 1 || n[d] > kMaxCells / cells) return WENO_ERR_INVALID_ARG;
        cells *= n[d];
        dV *= dx[d];
    }
    cudaStream_t s = (cudaStream_t)stream;
    double* scratch = nullptr;
    if (scratch_for_current_device(s, &scratch) != cudaSuccess) return WENO_ERR_CUDA;
    const int nblk = (int)((cells + kChunk - 1) / kChunk);
    cudaError_t e;
    const bool f64 = precision == WENO_FP64;
    if (dim == 1) e = f64 ? launch_totals<double, 3>(U_dev, cells, nblk, dV, scratch, totals_dev, s)
                          : launch_totals<float, 3>(U_dev, cells, nblk, dV, scratch, totals_dev, s);
    else if (dim == 2) e = f64 ? launch_totals<double, 4>(U_dev, cells, nblk, dV, scratch, totals_dev, s)
                               : launch_totals<float, 4>(U_dev, cells, nblk, dV, scratch, totals_dev, s);
    else e = f64 ? launch_totals<double, 5>(U_dev, cells, nblk, dV, scratch, totals_dev, s)
                 : launch_totals<float, 5>(U_dev, cells, nblk, dV, scratch, totals_dev, s);
    return e == cudaSuccess ? WENO_OK : WENO_ERR_CUDA;
}
