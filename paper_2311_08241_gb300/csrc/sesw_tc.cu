// Message layers of the learned surrogate on the fifth-generation tensor cores (sm_103a).
// Forward (k_msg_layer_tc):
//     Y[n][j] = tanh( sum_k Z[n][k] W[k][j] + b[j] ),  h_next[n][j] = h[n][j] + Y[n][j],  j < 64,
// where the CTA forms its rows of Z (bfloat16 values) from the hidden states while staging
// them, so Z never goes to memory; W is bfloat16 and the products accumulate in FP32 in
// tensor memory.
//
// One CTA of 256 threads computes 128 rows. It stages its Z tile and the whole W (as W^T,
// from a copy packed once per weight update by k_pack_wt) in shared memory in the K-major
// layout without swizzle that tcgen05.mma reads: core matrices of 8 rows x 8 bf16 (16 bytes
// per row, 128 bytes each), core matrices adjacent along K 128 bytes apart, along M (or N)
// K * 16 bytes apart. One thread issues K/16 MMAs of shape 128 x 64 x 16 into a 64-column
// TMEM accumulator and commits them to an mbarrier; after a bounded wait every warp reads 32
// rows x 32 columns back with tcgen05.ld, applies bias, activation and the residual, and
// stores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sesw_device.cuh"
#include "sesw_internal.h"
#include "sesw_msg.cuh"

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

// Read 16 FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int t = 0; t < 16; t++) v[t] = __uint_as_float(r[t]);
}

// W (K x 64, row-major bf16) as the shared-memory image of W^T that k_msg_layer_tc copies:
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

__device__ __forceinline__ uint4 pack_bf16x8(const float *v)
{
    return make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                      pack_bf16x2(v[6], v[7]));
}

__device__ __forceinline__ void load8(const float *p, float *v)
{
    const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Element incidences of a vertex-layer CTA's rows held in shared memory (more go through
// global memory, in the same order).
constexpr int MSG_INC_CAP = 1536;

// Shared memory of k_msg_layer_tc: the A tile (128 x K bf16), W^T (64 x K bf16), then the
// rows' graph data: KIND 0 the three corners of 128 elements (three CTAs of 75.3 KB fit an
// SM); KIND 1 the 129 CSR offsets of the rows and the element ids and areas of up to
// MSG_INC_CAP incidences.
__host__ __device__ constexpr size_t msg_layer_smem(int kind)
{
    return (size_t)(TC_M + TC_N) * (kind == 0 ? 3 * TC_N : 2 * TC_N) * 2 +
           (kind == 0 ? (size_t)TC_M * 12 : (size_t)(TC_M + 4) * 4 + (size_t)MSG_INC_CAP * 8);
}

// One message layer of the surrogate's forward pass (KIND 0: element rows, K = 192; KIND 1:
// vertex rows, K = 128): the CTA forms its 128 rows of Z from the hidden states while it
// stages them as the A tile, so Z never goes to memory, then Y = tanh(Z W + b) and
// h_next = h + Y in the epilogue. The rows' graph data go to shared memory first, so that
// every gather of the hidden states has its address at hand; each thread then gathers two
// rows' inputs at a time.
template <int KIND>
__global__ void __launch_bounds__(TC_THREADS, 3)
k_msg_layer_tc(const MsgLayerArgs a, const uint4 *__restrict__ Wp, const float *__restrict__ bias,
               unsigned *__restrict__ status, long long wait_cycles)
{
    constexpr int K = KIND == 0 ? 3 * TC_N : 2 * TC_N;
    constexpr int KC = K / 8;    // core matrices along K
    extern __shared__ __align__(1024) unsigned char smem[];
    uint4 *As = reinterpret_cast<uint4 *>(smem);                              // 128 x K bf16
    uint4 *Bs = reinterpret_cast<uint4 *>(smem + (size_t)TC_M * K * 2);       // 64 x K bf16 (W^T)
    unsigned char *gdata = smem + (size_t)(TC_M + TC_N) * K * 2;
    int *s_tri = reinterpret_cast<int *>(gdata);                              // KIND 0: [3][128]
    int *s_off = reinterpret_cast<int *>(gdata);                              // KIND 1
    int *s_inc = s_off + TC_M + 4;
    float *s_area = reinterpret_cast<float *>(s_inc + MSG_INC_CAP);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.N, n0 = blockIdx.x * TC_M;

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
    // the rows' graph data (rows past N: element 0's corners; empty CSR rows)
    if (KIND == 0) {
        for (int r = tid; r < TC_M; r += TC_THREADS) {
            const int4 v = n0 + r < N ? a.etri[n0 + r] : make_int4(0, 0, 0, 0);
            s_tri[r] = v.x;
            s_tri[TC_M + r] = v.y;
            s_tri[2 * TC_M + r] = v.z;
        }
    } else {
        for (int r = tid; r <= TC_M; r += TC_THREADS) s_off[r] = a.voff[min(n0 + r, N)];
    }
    // B tile: the packed image of W^T, copied as is
#pragma unroll 4
    for (int c = tid; c < TC_N * KC; c += TC_THREADS) Bs[c] = Wp[c];
    __syncthreads();
    const int qbase = KIND == 1 ? s_off[0] : 0;
    const bool inc_smem = KIND == 1 && s_off[TC_M] - qbase <= MSG_INC_CAP;
    if (KIND == 1 && inc_smem) {
        for (int t = tid; t < s_off[TC_M] - qbase; t += TC_THREADS) {
            const int e = a.vinc[qbase + t] >> 2;
            s_inc[t] = e;
            s_area[t] = a.earea[e];
        }
        __syncthreads();
    }
    // A tile: item it is row r = 8 rg + rl and the 8 hidden channels 8 cg .. 8 cg + 7; it forms
    // the row's 16-byte chunk of each block of Z for those channels (chunk kc of row r sits at
    // (rg KC + kc) 8 + rl). Consecutive threads take consecutive rows of one core matrix, so
    // the shared-memory stores do not conflict.
    constexpr int PER = TC_M * (TC_N / 8) / TC_THREADS;
    static_assert(PER % 2 == 0, "items per thread must be even");
#pragma unroll 1
    for (int u = 0; u < PER; u += 2) {
        int r[2], cg[2], n[2];
#pragma unroll
        for (int w = 0; w < 2; w++) {
            const int it = tid + (u + w) * TC_THREADS;
            r[w] = (it >> 6) * 8 + (it & 7);
            cg[w] = (it >> 3) & 7;
            n[w] = n0 + r[w];
        }
        float hs[2][8], m0[2][8], m1[2][8];
        if (KIND == 0) {
            float h0[2][8], h1[2][8], h2[2][8];
            float4 g[2];
#pragma unroll
            for (int w = 0; w < 2; w++) {
                const int c8 = cg[w] * 8, nc = min(n[w], N - 1);
                g[w] = a.egrad[nc];
                load8(a.hself + (size_t)nc * TC_N + c8, hs[w]);
                load8(a.hother + (size_t)s_tri[r[w]] * TC_N + c8, h0[w]);
                load8(a.hother + (size_t)s_tri[TC_M + r[w]] * TC_N + c8, h1[w]);
                load8(a.hother + (size_t)s_tri[2 * TC_M + r[w]] * TC_N + c8, h2[w]);
            }
#pragma unroll
            for (int w = 0; w < 2; w++) {
#pragma unroll
                for (int t = 0; t < 8; t++) {
                    const float2 m = msg_elem_grad(g[w], h0[w][t], h1[w][t], h2[w][t], a.L);
                    m0[w][t] = m.x;
                    m1[w][t] = m.y;
                }
            }
        } else {
#pragma unroll
            for (int w = 0; w < 2; w++) load8(a.hself + (size_t)min(n[w], N - 1) * TC_N + cg[w] * 8, hs[w]);
#pragma unroll
            for (int w = 0; w < 2; w++) {
                const int c8 = cg[w] * 8;
                const int q0 = s_off[r[w]], q1 = s_off[r[w] + 1];
#pragma unroll
                for (int t = 0; t < 8; t++) m0[w][t] = 0.0f;
                // four incidences' rows in flight, summed in incidence order
                int q = q0;
                for (; q + 4 <= q1; q += 4) {
                    float h[4][8], ar[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const int e = inc_smem ? s_inc[q + j - qbase] : a.vinc[q + j] >> 2;
                        ar[j] = inc_smem ? s_area[q + j - qbase] : a.earea[e];
                        load8(a.hother + (size_t)e * TC_N + c8, h[j]);
                    }
#pragma unroll
                    for (int j = 0; j < 4; j++)
#pragma unroll
                        for (int t = 0; t < 8; t++) m0[w][t] = msg_vert_acc(m0[w][t], ar[j], h[j][t]);
                }
                for (; q < q1; q++) {
                    const int e = inc_smem ? s_inc[q - qbase] : a.vinc[q] >> 2;
                    const float ar = inc_smem ? s_area[q - qbase] : a.earea[e];
                    float h[8];
                    load8(a.hother + (size_t)e * TC_N + c8, h);
#pragma unroll
                    for (int t = 0; t < 8; t++) m0[w][t] = msg_vert_acc(m0[w][t], ar, h[t]);
                }
                const float inv = a.vinvA[min(n[w], N - 1)];
#pragma unroll
                for (int t = 0; t < 8; t++) m0[w][t] = msg_vert_mean(m0[w][t], inv);
            }
        }
#pragma unroll
        for (int w = 0; w < 2; w++) {
            if (n[w] >= N) {
#pragma unroll
                for (int t = 0; t < 8; t++) hs[w][t] = m0[w][t] = m1[w][t] = 0.0f;
            }
            uint4 *chunk = As + (size_t)(r[w] >> 3) * KC * 8 + (r[w] & 7);    // chunk kc at chunk[kc * 8]
            chunk[cg[w] * 8] = pack_bf16x8(hs[w]);
            chunk[(8 + cg[w]) * 8] = pack_bf16x8(m0[w]);
            if (KIND == 0) chunk[(16 + cg[w]) * 8] = pack_bf16x8(m1[w]);
        }
    }
    // make the generic-proxy writes of the tiles visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const uint32_t tmem = tmem_base;
    // the epilogue's residual rows, requested before the MMAs are issued: this thread's row and
    // 32 columns (rows past N read row N - 1 and store nothing)
    const int quarter = warp & 3, half = warp >> 2;
    const int erow = n0 + quarter * 32 + lane;
    float4 hres[8];
    {
        const float4 *hsrc = reinterpret_cast<const float4 *>(a.hself + (size_t)min(erow, N - 1) * TC_N + half * 32);
#pragma unroll
        for (int t = 0; t < 8; t++) hres[t] = hsrc[t];
    }

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
        const int n = erow;
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
        for (int q = 2 * half; q < 2 * half + 2; q++) {
            float acc[16];
            tmem_ld16(taddr + q * 16, acc);
            if (n < N) {
                float4 *dy = a.Y ? reinterpret_cast<float4 *>(a.Y + (size_t)n * TC_N + q * 16) : nullptr;
                float4 *dh = reinterpret_cast<float4 *>(a.hnext + (size_t)n * TC_N + q * 16);
#pragma unroll
                for (int t = 0; t < 16; t += 4) {
                    float y[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) y[u] = tanhf(__fadd_rn(acc[t + u], bias[q * 16 + t + u]));
                    const float4 h = hres[(q - 2 * half) * 4 + t / 4];
                    if (dy) dy[t / 4] = make_float4(y[0], y[1], y[2], y[3]);
                    dh[t / 4] = make_float4(__fadd_rn(h.x, y[0]), __fadd_rn(h.y, y[1]), __fadd_rn(h.z, y[2]),
                                            __fadd_rn(h.w, y[3]));
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

// ---------------------------------------------------------------------------------
// The two backward contractions of a message layer (inputs Z [N][K] holding bfloat16 values,
// K = 128 or 192; weights W [K][64]; dA = dL/d(pre-activation) [N][64], FP32):
//   weight gradient  G[i][j] = sum_n Z[n][i] dA[n][j]           (k_wgrad_tc)
//   input gradient   dZ[n][i] = sum_j dA[n][j] W[i][j]           (k_dgrad_tc)
// dA is not a bfloat16 value, so each of its elements is split into two bfloat16 parts,
// hi = bf16(dA) and lo = bf16(dA - hi), which carry 16 significant bits, and both parts
// are multiplied: the products accumulate in FP32 in tensor memory. Operand tiles are
// staged in the same K-major layout without swizzle as k_msg_layer_tc's (core matrices of 8
// rows x 16 bytes, 128 bytes apart along K, KC * 128 bytes apart along M or N).

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Bounded wait on phase `parity` of an mbarrier; false when the budget ran out.
__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity, long long budget)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > budget) return false;
    }
}

constexpr int WG_THREADS = 256;
constexpr int WG_NC = 64;          // rows n of one staged chunk: 4 MMA steps of 16
constexpr int WG_KC = WG_NC / 8;   // core matrices along the reduction in a chunk

// Weight gradient: CTA b sums rows [b R, b R + R) of Z^T dA into partial[b][i * 64 + j], and
// the bias gradient (the column sums of dA) into partial[b][K * 64 + j]. D is one (K = 128)
// or two (K = 192: rows 128..191 and 64 rows of zeros) tiles of 128 x 64 in TMEM.
template <int K>
__global__ void __launch_bounds__(WG_THREADS)
k_wgrad_tc(int N, int rows_per_cta, const float *__restrict__ Z, const float *__restrict__ dA,
           float *__restrict__ partial, unsigned *__restrict__ status, long long wait_cycles)
{
    constexpr int MT = (K + 127) / 128;
    constexpr int A_CHUNKS = MT * 128 * WG_KC;     // 16-byte chunks of the A tile (rows i, K-major)
    constexpr int B_CHUNKS = TC_N * WG_KC;         // of each B tile (rows j)
    extern __shared__ __align__(1024) unsigned char smem[];
    uint4 *As = reinterpret_cast<uint4 *>(smem);
    uint4 *Bh = As + A_CHUNKS;
    uint4 *Bl = Bh + B_CHUNKS;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;
    __shared__ float s_bias[WG_KC][TC_N];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.x * rows_per_cta, r1 = min(N, r0 + rows_per_cta);
    const int nchunk = r1 > r0 ? (r1 - r0 + WG_NC - 1) / WG_NC : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(MT * TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    // rows K .. MT * 128 - 1 of A stay zero
    for (int c = tid; c < A_CHUNKS; c += WG_THREADS) As[c] = make_uint4(0u, 0u, 0u, 0u);
    // bias: thread t < 128 owns row octet t / 16 and columns 4 (t % 16) .. + 3 of every chunk
    float bsum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    __syncthreads();
    const uint32_t tmem = tmem_base;
    const uint32_t bar = smem_u32(&mbar);
    const uint32_t a0 = smem_u32(As), bh0 = smem_u32(Bh), bl0 = smem_u32(Bl);
    constexpr uint32_t idesc = idesc_bf16_f32(128, TC_N);

    for (int ch = 0; ch < nchunk; ch++) {
        const int n0 = r0 + ch * WG_NC;
        // A: unit (octet oc, feature quad fq) reads Z[n0 + 8 oc + t][4 fq .. 4 fq + 3], t < 8,
        // and writes the core-matrix rows of features 4 fq .. 4 fq + 3
        for (int u = tid; u < WG_KC * (K / 4); u += WG_THREADS) {
            const int oc = u / (K / 4), fq = u % (K / 4);
            float4 v[8];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                const int n = n0 + 8 * oc + t;
                v[t] = n < r1 ? *reinterpret_cast<const float4 *>(Z + (size_t)n * K + 4 * fq)
                              : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            const float *f = reinterpret_cast<const float *>(v);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int i = 4 * fq + q;
                uint32_t w[4];
#pragma unroll
                for (int t = 0; t < 8; t += 2)
                    w[t / 2] = bf16x2_bits(__float2bfloat16_rn(f[4 * t + q]), __float2bfloat16_rn(f[4 * (t + 1) + q]));
                As[((i >> 3) * WG_KC + oc) * 8 + (i & 7)] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        // B: the same for dA, split into hi and lo parts
        if (tid < WG_KC * (TC_N / 4)) {
            const int oc = tid / (TC_N / 4), jq = tid % (TC_N / 4);
            float4 v[8];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                const int n = n0 + 8 * oc + t;
                v[t] = n < r1 ? *reinterpret_cast<const float4 *>(dA + (size_t)n * TC_N + 4 * jq)
                              : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            const float *f = reinterpret_cast<const float *>(v);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int j = 4 * jq + q;
                uint32_t wh[4], wl[4];
#pragma unroll
                for (int t = 0; t < 8; t += 2) {
                    __nv_bfloat16 h0, l0, h1, l1;
                    split_bf16(f[4 * t + q], h0, l0);
                    split_bf16(f[4 * (t + 1) + q], h1, l1);
                    wh[t / 2] = bf16x2_bits(h0, h1);
                    wl[t / 2] = bf16x2_bits(l0, l1);
                }
                const int c = ((j >> 3) * WG_KC + oc) * 8 + (j & 7);
                Bh[c] = make_uint4(wh[0], wh[1], wh[2], wh[3]);
                Bl[c] = make_uint4(wl[0], wl[1], wl[2], wl[3]);
#pragma unroll
                for (int t = 0; t < 8; t++) bsum[q] += f[4 * t + q];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int ks = 0; ks < WG_KC / 2; ks++) {
                const uint64_t bdh = umma_desc(bh0 + ks * 256, 128, WG_KC * 128);
                const uint64_t bdl = umma_desc(bl0 + ks * 256, 128, WG_KC * 128);
#pragma unroll
                for (int mt = 0; mt < MT; mt++) {
                    const uint64_t ad = umma_desc(a0 + mt * 16 * WG_KC * 128 + ks * 256, 128, WG_KC * 128);
                    mma_bf16(tmem + mt * TC_N, ad, bdh, idesc, ch > 0 || ks > 0);
                    mma_bf16(tmem + mt * TC_N, ad, bdl, idesc, 1);
                }
            }
            mma_commit(bar);
            // the tiles are overwritten by the next chunk only after the products have read them
            if (!mbar_wait_parity(bar, ch & 1, wait_cycles)) {
                atomicOr(status, 2u);
                mbar_wait_parity(bar, ch & 1, wait_cycles);
                s_ok = 0;
            }
        }
        __syncthreads();
        if (!s_ok) break;
    }

    // bias partial: the 8 row octets' sums in a fixed order
    if (tid < WG_KC * (TC_N / 4)) {
        const int oc = tid / (TC_N / 4), jq = tid % (TC_N / 4);
#pragma unroll
        for (int q = 0; q < 4; q++) s_bias[oc][4 * jq + q] = bsum[q];
    }
    __syncthreads();
    float *out = partial + (size_t)blockIdx.x * ((size_t)K * TC_N + TC_N);
    if (tid < TC_N) {
        float b = 0.0f;
        for (int oc = 0; oc < WG_KC; oc++) b += s_bias[oc][tid];
        out[(size_t)K * TC_N + tid] = b;
    }
    // G rows i = 128 mt + 32 (warp % 4) + lane, columns 32 (warp / 4) .. + 31
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int quarter = warp & 3, half = warp >> 2;
#pragma unroll
    for (int mt = 0; mt < MT; mt++) {
        const int i = mt * 128 + quarter * 32 + lane;
#pragma unroll
        for (int q = 2 * half; q < 2 * half + 2; q++) {
            float v[16];
            if (nchunk > 0 && s_ok) {
                tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + mt * TC_N + q * 16, v);
            } else {
#pragma unroll
                for (int t = 0; t < 16; t++) v[t] = 0.0f;
            }
            if (i < K) {
                float4 *dst = reinterpret_cast<float4 *>(out + (size_t)i * TC_N + q * 16);
#pragma unroll
                for (int t = 0; t < 16; t += 4) dst[t / 4] = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MT * TC_N));
    }
}

// Input gradient: dZ[n][i] = sum_j dA[n][j] W[i][j] for 128 rows n per CTA; the reduction is
// over the 64 output channels j (4 MMA steps, each on the hi and the lo part of dA), the MMA's
// N is the layer's K (128 or 192 TMEM columns). W (K x 64 bfloat16, row-major) is already the
// K-major image of the B operand: row i holds W[i][0 .. 63].
template <int K>
__global__ void __launch_bounds__(WG_THREADS)
k_dgrad_tc(int N, const float *__restrict__ dA, const __nv_bfloat16 *__restrict__ W, float *__restrict__ dZ,
           unsigned *__restrict__ status, long long wait_cycles)
{
    constexpr int KC = TC_N / 8;                   // core matrices along the reduction (8)
    constexpr int TCOLS = K <= 128 ? 128 : 256;    // TMEM allocation (a power of two)
    extern __shared__ __align__(1024) unsigned char smem[];
    uint4 *Ah = reinterpret_cast<uint4 *>(smem);   // 128 x 64 bf16
    uint4 *Al = Ah + TC_M * KC;
    uint4 *Bs = Al + TC_M * KC;                    // K x 64 bf16
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.x * TC_M;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // A: chunk (row r = 8 rg + rl, channels 8 kc .. + 7) of dA, split into hi and lo
    for (int c = tid; c < TC_M * KC; c += WG_THREADS) {
        const int rl = c & 7, kc = (c >> 3) % KC, rg = (c >> 3) / KC;
        const int n = n0 + rg * 8 + rl;
        float4 va = make_float4(0.0f, 0.0f, 0.0f, 0.0f), vb = va;
        if (n < N) {
            va = *reinterpret_cast<const float4 *>(dA + (size_t)n * TC_N + kc * 8);
            vb = *reinterpret_cast<const float4 *>(dA + (size_t)n * TC_N + kc * 8 + 4);
        }
        const float f[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf16(f[t], h0, l0);
            split_bf16(f[t + 1], h1, l1);
            wh[t / 2] = bf16x2_bits(h0, h1);
            wl[t / 2] = bf16x2_bits(l0, l1);
        }
        Ah[(rg * KC + kc) * 8 + rl] = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        Al[(rg * KC + kc) * 8 + rl] = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    }
    // B: chunk (row i = 8 ig + il, channels 8 kc .. + 7) is 16 contiguous bytes of W
    const uint4 *Wv = reinterpret_cast<const uint4 *>(W);
    for (int c = tid; c < K * KC; c += WG_THREADS) {
        const int il = c & 7, kc = (c >> 3) % KC, ig = (c >> 3) / KC;
        Bs[c] = Wv[(size_t)(ig * 8 + il) * KC + kc];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), b0 = smem_u32(Bs);
        constexpr uint32_t idesc = idesc_bf16_f32(TC_M, K);
#pragma unroll
        for (int ks = 0; ks < KC / 2; ks++) {
            const uint64_t bd = umma_desc(b0 + ks * 256, 128, KC * 128);
            mma_bf16(tmem, umma_desc(ah + ks * 256, 128, KC * 128), bd, idesc, ks > 0);
            mma_bf16(tmem, umma_desc(al + ks * 256, 128, KC * 128), bd, idesc, 1);
        }
        mma_commit(smem_u32(&mbar));
        bool ok = mbar_wait_parity(smem_u32(&mbar), 0, wait_cycles);
        if (!ok) {
            atomicOr(status, 2u);
            mbar_wait_parity(smem_u32(&mbar), 0, wait_cycles);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (s_ok) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int quarter = warp & 3, half = warp >> 2;
        const int n = n0 + quarter * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
        constexpr int GROUPS = K / 16;             // 16-column groups, split between the two halves
        for (int q = half; q < GROUPS; q += 2) {
            float v[16];
            tmem_ld16(taddr + q * 16, v);
            if (n < N) {
                float4 *dst = reinterpret_cast<float4 *>(dZ + (size_t)n * K + q * 16);
#pragma unroll
                for (int t = 0; t < 16; t += 4) dst[t / 4] = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
    }
}

}  // namespace

bool linear_tc_supported(int K, int P) { return P == TC_N && (K == 128 || K == 192); }

size_t wgrad_tc_smem(int K) { return (size_t)((K + 127) / 128) * 128 * WG_NC * 2 + 2 * (size_t)TC_N * WG_NC * 2; }

cudaError_t launch_wgrad_tc(int N, int K, int rows_per_cta, const float *Z, const float *dA, float *partial,
                            unsigned *status, cudaStream_t st)
{
    if (rows_per_cta <= 0 || rows_per_cta % WG_NC) return cudaErrorInvalidValue;
    const int grid = std::max(1, (N + rows_per_cta - 1) / rows_per_cta);
    const size_t smem = wgrad_tc_smem(K);
    cudaError_t e;
    if (K == 128) {
        if ((e = cudaFuncSetAttribute(k_wgrad_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        k_wgrad_tc<128><<<grid, WG_THREADS, smem, st>>>(N, rows_per_cta, Z, dA, partial, status, 2000000000ll);
    } else if (K == 192) {
        if ((e = cudaFuncSetAttribute(k_wgrad_tc<192>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        k_wgrad_tc<192><<<grid, WG_THREADS, smem, st>>>(N, rows_per_cta, Z, dA, partial, status, 2000000000ll);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_dgrad_tc(int N, int K, const float *dA, const __nv_bfloat16 *W, float *dZ, unsigned *status,
                            cudaStream_t st)
{
    const int grid = (N + TC_M - 1) / TC_M;
    if (grid == 0) return cudaSuccess;
    const size_t smem = 2 * (size_t)TC_M * TC_N * 2 + (size_t)K * TC_N * 2;
    cudaError_t e;
    if (K == 128) {
        if ((e = cudaFuncSetAttribute(k_dgrad_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        k_dgrad_tc<128><<<grid, WG_THREADS, smem, st>>>(N, dA, W, dZ, status, 2000000000ll);
    } else if (K == 192) {
        if ((e = cudaFuncSetAttribute(k_dgrad_tc<192>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        k_dgrad_tc<192><<<grid, WG_THREADS, smem, st>>>(N, dA, W, dZ, status, 2000000000ll);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

size_t linear_tc_packed_elems(int K) { return (size_t)TC_N * K; }

cudaError_t pack_linear_tc(int K, const __nv_bfloat16 *W, __nv_bfloat16 *packed, cudaStream_t st)
{
    const int n = TC_N * K / 8;
    k_pack_wt<<<(n + 255) / 256, 256, 0, st>>>(K, W, reinterpret_cast<uint4 *>(packed));
    return cudaGetLastError();
}

cudaError_t launch_msg_layer_tc(const MsgLayerArgs &a, const __nv_bfloat16 *packed, const float *bias,
                                unsigned *status, cudaStream_t st)
{
    const uint4 *Wp = reinterpret_cast<const uint4 *>(packed);
    if (a.kind != 0 && a.kind != 1) return cudaErrorInvalidValue;
    const int grid = (a.N + TC_M - 1) / TC_M;
    if (grid == 0) return cudaSuccess;
    const size_t smem = msg_layer_smem(a.kind);
    const void *fn = a.kind == 0 ? (const void *)k_msg_layer_tc<0> : (const void *)k_msg_layer_tc<1>;
    // a per-kernel, per-device attribute: set on every launch (cheap) so that any device works
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // about one second of SM clock for the MMA completion wait
    if (a.kind == 0)
        k_msg_layer_tc<0><<<grid, TC_THREADS, smem, st>>>(a, Wp, bias, status, 2000000000ll);
    else
        k_msg_layer_tc<1><<<grid, TC_THREADS, smem, st>>>(a, Wp, bias, status, 2000000000ll);
    return cudaGetLastError();
}

}  // namespace sesw
