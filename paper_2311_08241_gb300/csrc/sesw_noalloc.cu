// Allocation-free variant of the FP64 volume/energy reduction (sesw_diagnostics).
//
// Some callers cannot allocate device memory at the point where they need the
// diagnostics: code running inside another framework's memory pool or under its
// allocator lock, real-time loops that must not touch the driver's allocator, or
// hosts that hand this library nothing but pre-allocated buffers. For them this entry
// point takes every input and the output from the caller and keeps its only scratch
// (the per-chunk partial sums of the two-pass reduction) in a fixed array in the
// library's device memory. That array exists once per GPU that loads the library
// and stays allocated until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/sesw.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItemsPerThread = 16;
constexpr int64_t kItemsPerBlock = (int64_t)kThreads * kItemsPerThread;   // 4096

// Scratch: one (volume, energy) partial pair per chunk of 4096 items.
static __device__ __align__(256) double g_partials[2 * SESW_NOALLOC_MAX_CHUNKS];

// Host-side view of the scratch: its device address, looked up once per device and kept
// for the life of the process (a cudaDeviceReset would invalidate it).
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch[kMaxDevices] = {nullptr};

__device__ __forceinline__ void block_sum_pair(double &x, double &y)
{
    __shared__ double sh[2][kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = x;
        sh[1][wid] = y;
    }
    __syncthreads();
    if (wid == 0) {
        x = lane < kThreads / 32 ? sh[0][lane] : 0.0;
        y = lane < kThreads / 32 ? sh[1][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
    }
}

// Chunk b sums vertices and elements with index in [b*4096, (b+1)*4096); every chunk
// writes its own partial pair, so the scratch needs no clearing between calls.
__global__ void __launch_bounds__(kThreads)
k_diag_chunks(int64_t nv, int64_t ne, const double *__restrict__ area_v, const double *__restrict__ eta,
              const double *__restrict__ area_e, const double *__restrict__ h_e, const double *__restrict__ U,
              double g, double *__restrict__ partials)
{
    const int64_t base = (int64_t)blockIdx.x * kItemsPerBlock;
    double vol = 0.0, en = 0.0;
    for (int k = 0; k < kItemsPerThread; k++) {
        const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < nv) {
            const double e = eta[i];
            vol += area_v[i] * e;
            en += area_v[i] * 0.5 * g * e * e;
        }
        if (i < ne) {
            const double ux = U[2 * i], uy = U[2 * i + 1];
            en += area_e[i] * (ux * ux + uy * uy) / (2.0 * h_e[i]);
        }
    }
    block_sum_pair(vol, en);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = vol;
        partials[2 * blockIdx.x + 1] = en;
    }
}

__global__ void __launch_bounds__(kThreads)
k_diag_chunks_final(const double *__restrict__ partials, int nchunks, double *__restrict__ out)
{
    double vol = 0.0, en = 0.0;
    for (int i = threadIdx.x; i < nchunks; i += kThreads) {
        vol += partials[2 * i];
        en += partials[2 * i + 1];
    }
    block_sum_pair(vol, en);
    if (threadIdx.x == 0) {
        out[0] = vol;
        out[1] = en;
    }
}

}  // namespace

extern "C" int sesw_diagnostics_noalloc(int64_t nv, int64_t ne, const double *area_v, const double *eta,
                                        const double *area_e, const double *h_e, const double *U, double g,
                                        double *out, void *cuda_stream)
{
    if (nv < 0 || ne < 0 || !out || !(g > 0.0) || (nv > 0 && (!area_v || !eta)) ||
        (ne > 0 && (!area_e || !h_e || !U)))
        return SESW_EINVAL;
    const int64_t n = nv > ne ? nv : ne;
    const int64_t nchunks = (n + kItemsPerBlock - 1) / kItemsPerBlock;
    if (nchunks > SESW_NOALLOC_MAX_CHUNKS) return SESW_EINVAL;   // more than SESW_NOALLOC_MAX_ITEMS items

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SESW_ECUDA;
    }
    double *scratch = nullptr;
    {
        // First call on this device: translate the array's host-side name into its
        // device address (with this device current). Later calls reuse the address.
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
                cudaGetLastError();
                return SESW_ECUDA;
            }
            g_scratch[dev] = (double *)p;
        }
        scratch = g_scratch[dev];
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int blocks = nchunks > 0 ? (int)nchunks : 1;
    k_diag_chunks<<<blocks, kThreads, 0, stream>>>(nv, ne, area_v, eta, area_e, h_e, U, g, scratch);
    k_diag_chunks_final<<<1, kThreads, 0, stream>>>(scratch, blocks, out);
    return cudaGetLastError() == cudaSuccess ? SESW_OK : SESW_ECUDA;
}
