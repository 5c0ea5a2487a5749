// CUDA kernels of libsesw (sm_103a): the split-explicit barotropic substep of
// Eq. (4.10), the time-mean transport of Eq. (4.12), state transfer and FP64
// diagnostics.
//
// Substep kernel layout. One thread block per vertex patch (a contiguous range of
// Hilbert-ordered vertices). The block first updates every element slot of the
// patch (the elements it owns and guest copies of neighbouring patches' elements
// that touch its vertices), keeping the three per-corner flux contributions in
// shared memory, then updates its own vertices by summing those contributions in a
// fixed order. eta is double-buffered across substeps (neighbouring blocks read the
// old level while this block writes the new one); element state is only ever read
// and written by the block that holds the slot.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sesw_internal.h"

namespace sesw {

namespace {

constexpr int kSubstepMaxThreads = 1024;
constexpr int kAuxThreads = 256;

// Error-free accumulation of x into the pair (hi, lo): after the call hi + lo equals
// the old hi + lo + x up to the rounding of lo (Knuth's two-sum). The explicit
// round-to-nearest intrinsics keep the compiler from fusing or reassociating.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x)
{
    float s = __fadd_rn(hi, x);
    float bp = __fsub_rn(s, hi);
    float ap = __fsub_rn(s, bp);
    float err = __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// One substep of Eq. (4.10) for all slots and vertices of the patch blockIdx.x.
//
// Element part (per slot, corners v0, v1, v2, gradients g0, g1, g2 = -g0 - g1):
//   grad eta = (eta0 - eta2) g0 + (eta1 - eta2) g1
//   H        = H0_e (+ (eta0 + eta1 + eta2)/3 when nonlinear)
//   a        = f dt / 2
//   r        = (Ux + a Uy, Uy - a Ux) + dt (R - g H grad eta)
//   U'       = (rx + a ry, ry - a rx) / (1 + a^2)           Crank-Nicolson Coriolis
//   F        = (1 + theta) U' - theta U
//   c_k      = dt A_e F . g_k, k = 0, 1;  c_2 = -(c_0 + c_1)  flux into corner k's cell
// Vertex part: eta' = eta + (sum of c over the vertex's incidences) / A_v.
template <int NONLIN>
__global__ void __launch_bounds__(kSubstepMaxThreads)
k_substep(const int4 *__restrict__ sv, const float4 *__restrict__ sg, const float4 *__restrict__ sc,
          const float2 *__restrict__ R, float2 *__restrict__ U, float2 *__restrict__ Shi,
          float2 *__restrict__ Slo, const int *__restrict__ patch_slot, const int *__restrict__ patch_own,
          const int *__restrict__ patch_v, const int *__restrict__ vcsr_off,
          const uint32_t *__restrict__ vcsr, const float *__restrict__ inv_av,
          const float *__restrict__ eta_in, float *__restrict__ eta_out, StepArgs a,
          unsigned *__restrict__ status)
{
    extern __shared__ float sflux[];
    const int p = blockIdx.x;
    const int s0 = patch_slot[p];
    const int n = patch_slot[p + 1] - s0;
    const int nown = patch_own[p];
    const float one_p_theta = 1.0f + a.theta;

    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = s0 + i;
        const int4 v = sv[s];
        const float4 g = sg[s];
        const float4 c = sc[s];
        const float2 r = R[s];
        const float2 u = U[s];
        const float e0 = eta_in[v.x], e1 = eta_in[v.y], e2 = eta_in[v.z];
        const float d0 = e0 - e2, d1 = e1 - e2;
        const float gx = d0 * g.x + d1 * g.z;
        const float gy = d0 * g.y + d1 * g.w;
        float H = c.y;
        if (NONLIN) H += (e0 + e1 + e2) * (1.0f / 3.0f);
        const float gH = a.g * H;
        const float aa = c.z * a.half_dt;
        const float rx = u.x + aa * u.y + a.dt * (r.x - gH * gx);
        const float ry = u.y - aa * u.x + a.dt * (r.y - gH * gy);
        const float inv = 1.0f / (1.0f + aa * aa);
        const float nx = (rx + aa * ry) * inv;
        const float ny = (ry - aa * rx) * inv;
        U[s] = make_float2(nx, ny);
        const float fx = one_p_theta * nx - a.theta * u.x;
        const float fy = one_p_theta * ny - a.theta * u.y;
        if (i < nown) {
            float2 hi = Shi[s], lo = Slo[s];
            two_sum_acc(hi.x, lo.x, fx);
            two_sum_acc(hi.y, lo.y, fy);
            Shi[s] = hi;
            Slo[s] = lo;
        }
        const float w = a.dt * c.x;
        const float c0 = w * (fx * g.x + fy * g.y);
        const float c1 = w * (fx * g.z + fy * g.w);
        sflux[3 * i + 0] = c0;
        sflux[3 * i + 1] = c1;
        sflux[3 * i + 2] = -(c0 + c1);
    }
    __syncthreads();

    const int v1 = patch_v[p + 1];
    bool bad = false;
    for (int v = patch_v[p] + threadIdx.x; v < v1; v += blockDim.x) {
        const int k1 = vcsr_off[v + 1];
        float sum = 0.0f;
        for (int k = vcsr_off[v]; k < k1; k++) {
            const uint32_t q = vcsr[k];
            sum += sflux[3 * (q >> 2) + (q & 3u)];
        }
        const float e = eta_in[v] + sum * inv_av[v];
        eta_out[v] = e;
        bad |= !(fabsf(e) <= a.eta_bound);
    }
    if (bad) atomicOr(status, 1u);
}

// End of a baroclinic step: <<U>> = S / M for owned slots, then S is cleared.
__global__ void k_epilogue(const int4 *__restrict__ sv, float2 *__restrict__ Shi, float2 *__restrict__ Slo,
                           float2 *__restrict__ Umean, int nslot, float inv_M)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslot; s += gridDim.x * blockDim.x) {
        const int w = sv[s].w;
        if (w < 0) continue;
        const float2 hi = Shi[s], lo = Slo[s];
        Umean[w] = make_float2((hi.x + lo.x) * inv_M, (hi.y + lo.y) * inv_M);
        Shi[s] = make_float2(0.0f, 0.0f);
        Slo[s] = make_float2(0.0f, 0.0f);
    }
}

__global__ void k_scatter_eta(const int *__restrict__ vperm, const double *__restrict__ in, float *__restrict__ eta,
                              int nv)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
        eta[v] = (float)in[vperm[v]];
}

// Copy a caller-order [ne][2] field into every slot (owner and guest copies alike).
__global__ void k_scatter_slots(const int4 *__restrict__ sv, const int *__restrict__ eperm,
                                const double *__restrict__ in, float2 *__restrict__ out, int nslot)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslot; s += gridDim.x * blockDim.x) {
        const int w = sv[s].w;
        const int e = eperm[w >= 0 ? w : -1 - w];
        out[s] = make_float2((float)in[2 * (size_t)e], (float)in[2 * (size_t)e + 1]);
    }
}

__global__ void k_gather(const int4 *__restrict__ sv, const int *__restrict__ vperm, const int *__restrict__ eperm,
                         const float *__restrict__ eta, const float2 *__restrict__ U,
                         const float2 *__restrict__ Umean, double *__restrict__ eta_out,
                         double *__restrict__ U_out, double *__restrict__ Um_out, int nv, int nslot)
{
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (eta_out)
        for (int v = t0; v < nv; v += stride) eta_out[vperm[v]] = (double)eta[v];
    for (int s = t0; s < nslot; s += stride) {
        const int w = sv[s].w;
        if (w < 0) continue;
        const int e = eperm[w];
        if (U_out) {
            const float2 u = U[s];
            U_out[2 * (size_t)e] = (double)u.x;
            U_out[2 * (size_t)e + 1] = (double)u.y;
        }
        if (Um_out) {
            const float2 u = Umean[w];
            Um_out[2 * (size_t)e] = (double)u.x;
            Um_out[2 * (size_t)e + 1] = (double)u.y;
        }
    }
}

template <int N>
__device__ __forceinline__ void block_sum2(double &x, double &y, double (*sh)[N])
{
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
        const int nw = (blockDim.x + 31) >> 5;
        x = lane < nw ? sh[0][lane] : 0.0;
        y = lane < nw ? sh[1][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
    }
}

// Per-block partial sums of volume and energy (FP64). Fixed grid and order, so the
// result is reproducible run to run.
__global__ void __launch_bounds__(kAuxThreads)
k_diag_partial(const int4 *__restrict__ sv, const float4 *__restrict__ sc, const float2 *__restrict__ U,
               const double *__restrict__ area_v, const float *__restrict__ eta, int nv, int nslot, double g,
               int nonlinear_h, double *__restrict__ part)
{
    __shared__ double sh[2][32];
    double vol = 0.0, en = 0.0;
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
        const double e = (double)eta[v];
        vol += area_v[v] * e;
        en += area_v[v] * 0.5 * g * e * e;
    }
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslot; s += stride) {
        const int4 c = sv[s];
        if (c.w < 0) continue;
        const float4 k = sc[s];
        double H = (double)k.y;
        if (nonlinear_h) H += ((double)eta[c.x] + (double)eta[c.y] + (double)eta[c.z]) / 3.0;
        const float2 u = U[s];
        en += (double)k.x * ((double)u.x * u.x + (double)u.y * u.y) / (2.0 * H);
    }
    block_sum2<32>(vol, en, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = vol;
        part[2 * blockIdx.x + 1] = en;
    }
}

__global__ void __launch_bounds__(kAuxThreads)
k_diag_final(const double *__restrict__ part, int nparts, double *__restrict__ out)
{
    __shared__ double sh[2][32];
    double vol = 0.0, en = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        vol += part[2 * i];
        en += part[2 * i + 1];
    }
    block_sum2<32>(vol, en, sh);
    if (threadIdx.x == 0) {
        out[0] = vol;
        out[1] = en;
    }
}

int grid_for(int n, int threads)
{
    int b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return b;
}

}  // namespace

cudaError_t launch_substep(const DevMesh &m, const DevState &s, const StepArgs &a, int parity, int block,
                           cudaStream_t stream)
{
    const int threads = block > 0 ? block : 256;
    const size_t smem = sizeof(float) * 3 * (size_t)m.max_patch_slots;
    const float *ein = s.eta[parity];
    float *eout = s.eta[parity ^ 1];
    if (a.nonlinear_h)
        k_substep<1><<<m.npatch, threads, smem, stream>>>(
            m.slot_v, m.slot_g, m.slot_c, s.R, s.U, s.S_hi, s.S_lo, m.patch_slot, m.patch_own, m.patch_v,
            m.vcsr_off, m.vcsr, m.inv_av, ein, eout, a, s.status);
    else
        k_substep<0><<<m.npatch, threads, smem, stream>>>(
            m.slot_v, m.slot_g, m.slot_c, s.R, s.U, s.S_hi, s.S_lo, m.patch_slot, m.patch_own, m.patch_v,
            m.vcsr_off, m.vcsr, m.inv_av, ein, eout, a, s.status);
    return cudaGetLastError();
}

cudaError_t substep_smem_attr(const DevMesh &m)
{
    const size_t smem = sizeof(float) * 3 * (size_t)m.max_patch_slots;
    cudaError_t e = cudaFuncSetAttribute(k_substep<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_substep<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_step_epilogue(const DevMesh &m, const DevState &s, const StepArgs &a, cudaStream_t stream)
{
    k_epilogue<<<grid_for(m.nslot, kAuxThreads), kAuxThreads, 0, stream>>>(m.slot_v, s.S_hi, s.S_lo, s.Umean,
                                                                             m.nslot, a.inv_M);
    return cudaGetLastError();
}

cudaError_t launch_scatter_state(const DevMesh &m, const DevState &s, const double *eta, const double *U,
                                 int parity, cudaStream_t stream)
{
    if (eta)
        k_scatter_eta<<<grid_for(m.nv, kAuxThreads), kAuxThreads, 0, stream>>>(m.vperm, eta, s.eta[parity], m.nv);
    if (U)
        k_scatter_slots<<<grid_for(m.nslot, kAuxThreads), kAuxThreads, 0, stream>>>(m.slot_v, m.eperm, U, s.U,
                                                                                      m.nslot);
    return cudaGetLastError();
}

cudaError_t launch_scatter_forcing(const DevMesh &m, const DevState &s, const double *R, cudaStream_t stream)
{
    k_scatter_slots<<<grid_for(m.nslot, kAuxThreads), kAuxThreads, 0, stream>>>(m.slot_v, m.eperm, R, s.R,
                                                                                  m.nslot);
    return cudaGetLastError();
}

cudaError_t launch_gather_state(const DevMesh &m, const DevState &s, int parity, double *eta, double *U,
                                double *Umean, cudaStream_t stream)
{
    k_gather<<<grid_for(m.nv > m.nslot ? m.nv : m.nslot, kAuxThreads), kAuxThreads, 0, stream>>>(
        m.slot_v, m.vperm, m.eperm, s.eta[parity], s.U, s.Umean, eta, U, Umean, m.nv, m.nslot);
    return cudaGetLastError();
}

int diagnostics_blocks(const DevMesh &m)
{
    int n = m.nv > m.nslot ? m.nv : m.nslot;
    int b = (n + kAuxThreads - 1) / kAuxThreads;
    if (b > 4 * 152) b = 4 * 152;
    if (b < 1) b = 1;
    return b;
}

cudaError_t launch_diagnostics(const DevMesh &m, const DevState &s, const StepArgs &a, int parity, int nblocks,
                               cudaStream_t stream)
{
    k_diag_partial<<<nblocks, kAuxThreads, 0, stream>>>(m.slot_v, m.slot_c, s.U, m.area_v, s.eta[parity], m.nv,
                                                        m.nslot, a.g64, a.nonlinear_h, s.diag_part);
    k_diag_final<<<1, kAuxThreads, 0, stream>>>(s.diag_part, nblocks, s.diag_out);
    return cudaGetLastError();
}

}  // namespace sesw
