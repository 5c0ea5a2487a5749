// Dense layer of the learned surrogate on the fifth-generation tensor cores (sm_103a):
//     Y[n][j] = act( sum_k X[n][k] W[k][j] + b[j] ),  j < 64,
// with X already rounded to bfloat16 values (stored as float) and W in bfloat16; the
// products accumulate in FP32 in tensor memory.
//
// One CTA of 256 threads computes 128 rows. It stages its X tile and the whole W (as
// W^T, from a copy packed once per weight update by k_pack_wt) in shared memory in the
// K-major layout without swizzle that tcgen05.mma reads:
// core matrices of 8 rows x 8 bf16 (16 bytes per row, 128 bytes each), core matrices
// adjacent along K 128 bytes apart, along M (or N) K * 16 bytes apart. One thread
// issues K/16 MMAs of shape 128 x 64 x 16 into a 64-column TMEM accumulator and commits
// them to an mbarrier; after a bounded wait every warp reads 32 rows x 32 columns back
// with tcgen05.ld, applies bias and activation, and stores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sesw_device.cuh"
#include "sesw_internal.h"

namespace sesw {

namespace {

constexpr int TC_M = 128;        // rows per CTA: one MMA with M = 128
constexpr int TC_N = 64;         // output columns: the hidden width
constexpr int TC_THREADS = 256;  // eight warps: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns 32 (w / 4) .. + 31

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05) of a K-major operand without swizzle: start
// address, leading byte offset (between core matrices adjacent along K), stride byte
// offset (along M or N), all in 16-byte units; bit 46 is the descriptor version.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1),
// BF16 A and B (bits 7-9 and 10-12 = 1), both K-major, N / 8 at bit 17, M / 16 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Bounded wait on phase 0 of an mbarrier; false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, long long budget)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(0)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > budget) return false;
    }
}

// W (K x 64, row-major bf16) as the shared-memory image of W^T that k_linear_tc copies:
// 16-byte chunk c = (jg * K/8 + kc) * 8 + jl holds W[8 kc .. 8 kc + 7][8 jg + jl].
__global__ void k_pack_wt(int K, const __nv_bfloat16 *__restrict__ W, uint4 *__restrict__ out)
{
    const int KC = K / 8;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < TC_N * KC; c += gridDim.x * blockDim.x) {
        const int jl = c & 7, kc = (c >> 3) % KC, jg = (c >> 3) / KC;
        const int j = jg * 8 + jl;
        unsigned short h[8];
#pragma unroll
        for (int t = 0; t < 8; t++) h[t] = __bfloat16_as_ushort(W[(size_t)(kc * 8 + t) * TC_N + j]);
        out[c] = make_uint4((uint32_t)h[0] | ((uint32_t)h[1] << 16), (uint32_t)h[2] | ((uint32_t)h[3] << 16),
                            (uint32_t)h[4] | ((uint32_t)h[5] << 16), (uint32_t)h[6] | ((uint32_t)h[7] << 16));
    }
}

template <int K>
__global__ void __launch_bounds__(TC_THREADS)
k_linear_tc(int N, const float *__restrict__ X, const uint4 *__restrict__ Wp, const float *__restrict__ bias,
            int act, float *__restrict__ Y, unsigned *__restrict__ status, long long wait_cycles)
{
    static_assert(K % 16 == 0 && K <= 256, "K must be a multiple of 16");
    constexpr int KC = K / 8;    // core matrices along K
    extern __shared__ __align__(1024) unsigned char smem[];
    uint4 *As = reinterpret_cast<uint4 *>(smem);                              // 128 x K bf16
    uint4 *Bs = reinterpret_cast<uint4 *>(smem + (size_t)TC_M * K * 2);       // 64 x K bf16 (W^T)
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.x * TC_M;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // A tile: chunk c is row r = 8 rg + rl, columns 8 kc .. 8 kc + 7; consecutive threads
    // fill consecutive 16-byte rows of one core matrix. Four chunks' loads are issued
    // before any is converted, so that their latencies overlap.
    constexpr int PER = TC_M * KC / TC_THREADS;
    static_assert(PER % 4 == 0, "chunks per thread must be a multiple of 4");
#pragma unroll
    for (int b = 0; b < PER; b += 4) {
        float4 va[4], vb[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int c = tid + (b + u) * TC_THREADS;
            const int rl = c & 7, kc = (c >> 3) % KC, rg = (c >> 3) / KC;
            const int n = n0 + rg * 8 + rl;
            va[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            vb[u] = va[u];
            if (n < N) {
                va[u] = *reinterpret_cast<const float4 *>(X + (size_t)n * K + kc * 8);
                vb[u] = *reinterpret_cast<const float4 *>(X + (size_t)n * K + kc * 8 + 4);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int c = tid + (b + u) * TC_THREADS;
            const int rl = c & 7, kc = (c >> 3) % KC, rg = (c >> 3) / KC;
            As[(rg * KC + kc) * 8 + rl] =
                make_uint4(pack_bf16x2(va[u].x, va[u].y), pack_bf16x2(va[u].z, va[u].w),
                           pack_bf16x2(vb[u].x, vb[u].y), pack_bf16x2(vb[u].z, vb[u].w));
        }
    }
    // B tile: the packed image of W^T, copied as is
#pragma unroll 4
    for (int c = tid; c < TC_N * KC; c += TC_THREADS) Bs[c] = Wp[c];
    // make the generic-proxy writes of the tiles visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const uint32_t tmem = tmem_base;

    if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
        constexpr uint32_t idesc = idesc_bf16_f32(TC_M, TC_N);
#pragma unroll
        for (int ks = 0; ks < K / 16; ks++) {
            const uint64_t ad = umma_desc(a0 + ks * 256, 128, KC * 128);
            const uint64_t bd = umma_desc(b0 + ks * 256, 128, KC * 128);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(ks));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mbar))
                     : "memory");
        bool ok = mbar_wait(smem_u32(&mbar), wait_cycles);
        if (!ok) {
            atomicOr(status, 2u);
            // the MMAs may still be in flight: give them one more budget before TMEM is freed
            mbar_wait(smem_u32(&mbar), wait_cycles);
        }
        s_ok = ok;
    }
    __syncthreads();

    if (s_ok) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int quarter = warp & 3, half = warp >> 2;
        const int row = quarter * 32 + lane;
        const int n = n0 + row;
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
        for (int q = 2 * half; q < 2 * half + 2; q++) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr + q * 16));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (n < N) {
                float4 *dst = reinterpret_cast<float4 *>(Y + (size_t)n * TC_N + q * 16);
#pragma unroll
                for (int t = 0; t < 16; t += 4) {
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        float y = __uint_as_float(r[t + u]);
                        if (bias) y += bias[q * 16 + t + u];
                        if (act) y = tanhf(y);
                        v[u] = y;
                    }
                    dst[t / 4] = make_float4(v[0], v[1], v[2], v[3]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
    }
}

template <int K>
cudaError_t launch_k(int N, const float *X, const uint4 *Wp, const float *bias, int act, float *Y,
                     unsigned *status, cudaStream_t st)
{
    const size_t smem = (size_t)(TC_M + TC_N) * K * 2;
    // a per-kernel, per-device attribute: set on every launch (cheap) so that any device works
    cudaError_t e = cudaFuncSetAttribute(k_linear_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (N + TC_M - 1) / TC_M;
    if (grid == 0) return cudaSuccess;
    // about one second of SM clock for the MMA completion wait
    k_linear_tc<K><<<grid, TC_THREADS, smem, st>>>(N, X, Wp, bias, act, Y, status, 2000000000ll);
    return cudaGetLastError();
}

}  // namespace

bool linear_tc_supported(int K, int P) { return P == TC_N && (K == 128 || K == 192); }

size_t linear_tc_packed_elems(int K) { return (size_t)TC_N * K; }

cudaError_t pack_linear_tc(int K, const __nv_bfloat16 *W, __nv_bfloat16 *packed, cudaStream_t st)
{
    const int n = TC_N * K / 8;
    k_pack_wt<<<(n + 255) / 256, 256, 0, st>>>(K, W, reinterpret_cast<uint4 *>(packed));
    return cudaGetLastError();
}

cudaError_t launch_linear_tc(int N, int K, const float *X, const __nv_bfloat16 *packed, const float *bias, int act,
                             float *Y, unsigned *status, cudaStream_t st)
{
    const uint4 *Wp = reinterpret_cast<const uint4 *>(packed);
    if (K == 128) return launch_k<128>(N, X, Wp, bias, act, Y, status, st);
    if (K == 192) return launch_k<192>(N, X, Wp, bias, act, Y, status, st);
    return cudaErrorInvalidValue;
}

}  // namespace sesw
