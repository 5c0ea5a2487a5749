// CUDA kernels of libsesw (sm_103a): the split-explicit barotropic substep of
// Eq. (4.10) (with the freshwater flux W of Eq. 4.5), the SESM substep of Eqs.
// (4.7)-(4.8), the barotropic viscous regularisation of Eq. (viscosity_BT), the
// time-mean transport of Eq. (4.12), state transfer and FP64 diagnostics.
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

#include <algorithm>

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

// Barotropic viscous regularisation, Eq. (viscosity_BT), of the element w held by a
// slot with depth H and transport Us: a two-point flux across each edge with a
// neighbour (owner slot nb.k, or -1 at a coast),
//   u = U / H here and on the neighbour, du = rot(u_nb) - u with rot the turn from the
//   neighbour's frame into this one, A = background + flow |du| L,
//   R_hV = (1/A_e) sum_edges (H + H_nb)/2 A (L/d) du,
// H_nb = H0 (+ corner mean of eta when nonlinear) of the neighbour. Every copy of an
// element evaluates this from the same owner-slot inputs, so guests stay equal to owners.
__device__ __forceinline__ float2 visc_of(int w, float H, float2 Us, float area, const int4 *__restrict__ sv,
                                          const float4 *__restrict__ sc, const float2 *U,
                                          const int4 *__restrict__ vnb, const float4 *__restrict__ vgeo,
                                          const float *__restrict__ eta, const ViscArgs va)
{
    const float ux = Us.x / H, uy = Us.y / H;
    const int4 nb = vnb[w];
    const int nbs[3] = {nb.x, nb.y, nb.z};
    float fx = 0.0f, fy = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int q = nbs[k];
        if (q < 0) continue;
        const float4 gq = vgeo[3 * (size_t)w + k];
        float Hn = sc[q].y;
        if (va.nonlinear_h) {
            const int4 vq = sv[q];
            Hn += (eta[vq.x] + eta[vq.y] + eta[vq.z]) * (1.0f / 3.0f);
        }
        const float2 Uq = U[q];
        const float nx = Uq.x / Hn, ny = Uq.y / Hn;
        const float dx = (gq.x * nx - gq.y * ny) - ux;
        const float dy = (gq.y * nx + gq.x * ny) - uy;
        const float A = va.background + va.flow * sqrtf(dx * dx + dy * dy) * gq.w;
        const float kq = 0.5f * (H + Hn) * A * gq.z;
        fx += kq * dx;
        fy += kq * dy;
    }
    return make_float2(fx / area, fy / area);
}

// Viscosity inputs of the substep kernel (VISC = 1): transports are read from U_in (level
// m, also the neighbours') and written to U_out (level m + 1), and the forcing of the
// substep is R + (R_hV - V0) with V0 the value at substep 0 of the step (start = 1
// stores it; Sect. 2.2 subtracts the term's start value).
struct SubstepVisc {
    const int4 *vnb;
    const float4 *vgeo;
    float2 *V0;
    ViscArgs va;
    int start;
};

// One substep of Eq. (4.10) for all slots and vertices of the patch blockIdx.x.
//
// Element part (per slot, corners v0, v1, v2, gradients g0, g1, g2 = -g0 - g1):
//   grad eta = (eta0 - eta2) g0 + (eta1 - eta2) g1
//   H        = H0_e (+ (eta0 + eta1 + eta2)/3 when nonlinear)
//   a        = f dt / 2
//   r        = (Ux + a Uy, Uy - a Ux) + dt (R' - g H grad eta),  R' = R (+ R_hV - V0 with VISC)
//   U'       = (rx + a ry, ry - a rx) / (1 + a^2)           Crank-Nicolson Coriolis
//   F        = (1 + theta) U' - theta U
//   c_k      = dt A_e F . g_k, k = 0, 1;  c_2 = -(c_0 + c_1)  flux into corner k's cell
// Vertex part: eta' = eta + (sum of c over the vertex's incidences) / A_v - dt W
// (W: freshwater flux of Eq. 4.5, positive out of the ocean; W == NULL means 0).
// Without VISC, U_in and U_out are the same array (each slot is read, then written, by
// one thread).
template <int NONLIN, int VISC>
__global__ void __launch_bounds__(kSubstepMaxThreads)
k_substep(const int4 *__restrict__ sv, const float4 *__restrict__ sg, const float4 *__restrict__ sc,
          const float2 *__restrict__ R, const float2 *U_in, float2 *U_out, float2 *__restrict__ Shi,
          float2 *__restrict__ Slo, const int *__restrict__ patch_slot, const int *__restrict__ patch_own,
          const int *__restrict__ patch_v, const int *__restrict__ vcsr_off,
          const uint32_t *__restrict__ vcsr, const float *__restrict__ inv_av,
          const float *__restrict__ eta_in, float *__restrict__ eta_out, const float *__restrict__ patch_dt,
          float *__restrict__ eta_sum, const float *__restrict__ W, SubstepVisc vis, StepArgs a,
          unsigned *__restrict__ status)
{
    extern __shared__ float sflux[];
    const int p = blockIdx.x;
    const float dt = patch_dt[p], half_dt = 0.5f * dt;
    const int s0 = patch_slot[p];
    const int n = patch_slot[p + 1] - s0;
    const int nown = patch_own[p];
    const float one_p_theta = 1.0f + a.theta;

    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = s0 + i;
        const int4 v = sv[s];
        const float4 g = sg[s];
        const float4 c = sc[s];
        float2 r = R[s];
        const float2 u = U_in[s];
        const float e0 = eta_in[v.x], e1 = eta_in[v.y], e2 = eta_in[v.z];
        const float d0 = e0 - e2, d1 = e1 - e2;
        const float gx = d0 * g.x + d1 * g.z;
        const float gy = d0 * g.y + d1 * g.w;
        float H = c.y;
        if (NONLIN) H += (e0 + e1 + e2) * (1.0f / 3.0f);
        if (VISC) {
            const float2 V = visc_of(v.w >= 0 ? v.w : -1 - v.w, H, u, c.x, sv, sc, U_in, vis.vnb, vis.vgeo, eta_in,
                                     vis.va);
            if (vis.start) {
                vis.V0[s] = V;      // R' = R + (V - V) = R
            } else {
                const float2 z = vis.V0[s];
                r = make_float2(r.x + (V.x - z.x), r.y + (V.y - z.y));
            }
        }
        const float gH = a.g * H;
        const float aa = c.z * half_dt;
        const float rx = u.x + aa * u.y + dt * (r.x - gH * gx);
        const float ry = u.y - aa * u.x + dt * (r.y - gH * gy);
        const float inv = 1.0f / (1.0f + aa * aa);
        const float nx = (rx + aa * ry) * inv;
        const float ny = (ry - aa * rx) * inv;
        U_out[s] = make_float2(nx, ny);
        const float fx = one_p_theta * nx - a.theta * u.x;
        const float fy = one_p_theta * ny - a.theta * u.y;
        if (i < nown) {
            float2 hi = Shi[s], lo = Slo[s];
            two_sum_acc(hi.x, lo.x, fx);
            two_sum_acc(hi.y, lo.y, fy);
            Shi[s] = hi;
            Slo[s] = lo;
        }
        const float w = dt * c.x;
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
        float e = eta_in[v] + sum * inv_av[v];
        if (W) e -= dt * W[v];
        if (eta_sum) eta_sum[v] += eta_in[v];     // sum of eta^0 .. eta^{M-1} (time mean of the step)
        eta_out[v] = e;
        bad |= !(fabsf(e) <= a.eta_bound);
    }
    if (bad) atomicOr(status, 1u);
}

// ---------------------------------------------------------------------------------
// SESM substep (AB3-AM4 with dissipative coefficients, Eqs. 4.7-4.8), one launch per
// substep in graph mode. Launch m first completes the momentum update of substep m-1,
//     U^m = U^{m-1} + dt ( -f e_z x U_AB^{m-1} - g H_AM grad(eta_AM) + R ),
//     eta_AM = am0 eta^m + am1 eta^{m-1} + am2 eta^{m-2} + am3 eta^{m-3},
//     U_AB^{m-1} = ab0 U^{m-1} + ab1 U^{m-2} + ab2 U^{m-3}
// (skipped for m = 0), then forms U_AB^m = ab0 U^m + ab1 U^{m-1} + ab2 U^{m-2}, adds it
// to the compensated sum S and updates eta^{m+1} = eta^m - dt (div(U_AB^m) + W). Levels before
// the start of the subcycle are passed as aliases of level 0.
struct SesmLevels {
    const float2 *u1, *u2, *u3;      // U^{m-1}, U^{m-2}, U^{m-3}
    float2 *u0;                      // U^m (written when update != 0, else read)
    const float *e0, *e1, *e2, *e3;  // eta^m, eta^{m-1}, eta^{m-2}, eta^{m-3}
    float *enew;                     // eta^{m+1}
    int update;                      // 1: compute U^m first
    int vertex;                      // 1: continuity update (0 only in the closing launch)
};

template <int NONLIN>
__global__ void __launch_bounds__(kSubstepMaxThreads)
k_sesm(const int4 *__restrict__ sv, const float4 *__restrict__ sg, const float4 *__restrict__ sc,
       const float2 *__restrict__ R, float2 *__restrict__ Shi, float2 *__restrict__ Slo,
       const int *__restrict__ patch_slot, const int *__restrict__ patch_own, const int *__restrict__ patch_v,
       const int *__restrict__ vcsr_off, const uint32_t *__restrict__ vcsr, const float *__restrict__ inv_av,
       const float *__restrict__ patch_dt, const float *__restrict__ W, SesmLevels L, StepArgs a,
       unsigned *__restrict__ status)
{
    extern __shared__ float sflux[];
    const int p = blockIdx.x;
    const float dt = patch_dt[p];
    const int s0 = patch_slot[p];
    const int n = patch_slot[p + 1] - s0;
    const int nown = patch_own[p];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = s0 + i;
        const int4 v = sv[s];
        const float4 g = sg[s];
        const float2 u1 = L.u1[s], u2 = L.u2[s];
        float2 u0;
        if (L.update) {
            const float4 c = sc[s];
            const float2 u3 = L.u3[s], r = R[s];
            const float abx = a.ab0 * u1.x + a.ab1 * u2.x + a.ab2 * u3.x;
            const float aby = a.ab0 * u1.y + a.ab1 * u2.y + a.ab2 * u3.y;
            float em[3];
            const int vv[3] = {v.x, v.y, v.z};
#pragma unroll
            for (int k = 0; k < 3; k++)
                em[k] = a.am0 * L.e0[vv[k]] + a.am1 * L.e1[vv[k]] + a.am2 * L.e2[vv[k]] + a.am3 * L.e3[vv[k]];
            const float d0 = em[0] - em[2], d1 = em[1] - em[2];
            const float gx = d0 * g.x + d1 * g.z;
            const float gy = d0 * g.y + d1 * g.w;
            float H = c.y;
            if (NONLIN) H += (em[0] + em[1] + em[2]) * (1.0f / 3.0f);
            const float gH = a.g * H;
            // -f e_z x U_AB = (f U_AB_y, -f U_AB_x)
            u0.x = u1.x + dt * (c.z * aby - gH * gx + r.x);
            u0.y = u1.y + dt * (-c.z * abx - gH * gy + r.y);
            L.u0[s] = u0;
        } else {
            u0 = L.u0[s];
        }
        if (!L.vertex) continue;
        const float fx = a.ab0 * u0.x + a.ab1 * u1.x + a.ab2 * u2.x;
        const float fy = a.ab0 * u0.y + a.ab1 * u1.y + a.ab2 * u2.y;
        if (i < nown) {
            float2 hi = Shi[s], lo = Slo[s];
            two_sum_acc(hi.x, lo.x, fx);
            two_sum_acc(hi.y, lo.y, fy);
            Shi[s] = hi;
            Slo[s] = lo;
        }
        const float w = dt * sc[s].x;
        const float c0 = w * (fx * g.x + fy * g.y);
        const float c1 = w * (fx * g.z + fy * g.w);
        sflux[3 * i + 0] = c0;
        sflux[3 * i + 1] = c1;
        sflux[3 * i + 2] = -(c0 + c1);
    }
    if (!L.vertex) return;
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
        float e = L.e0[v] + sum * inv_av[v];
        if (W) e -= dt * W[v];
        L.enew[v] = e;
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

// R_hV of every element at (U, eta) into out[element] (the operator alone; the step
// evaluates it inside k_substep). One thread per owned slot.
__global__ void __launch_bounds__(kAuxThreads)
k_viscosity(const int4 *__restrict__ sv, const float4 *__restrict__ sc, const float2 *__restrict__ U,
            const int4 *__restrict__ vnb, const float4 *__restrict__ vgeo, const float *__restrict__ eta,
            ViscArgs va, float2 *__restrict__ out, int nslot)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslot; s += gridDim.x * blockDim.x) {
        const int4 v = sv[s];
        if (v.w < 0) continue;
        const float4 c = sc[s];
        float H = c.y;
        if (va.nonlinear_h) H += (eta[v.x] + eta[v.y] + eta[v.z]) * (1.0f / 3.0f);
        out[v.w] = visc_of(v.w, H, U[s], c.x, sv, sc, U, vnb, vgeo, eta, va);
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

__global__ void k_gather_scaled(const int *__restrict__ vperm, const float *__restrict__ x, double scale,
                                double *__restrict__ out, int nv)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
        out[vperm[v]] = (double)x[v] * scale;
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

// One block per basin: volume and energy of its vertex and owned-slot ranges.
__global__ void __launch_bounds__(kAuxThreads)
k_diag_basins(const int *__restrict__ basin_v, const int *__restrict__ basin_slot, const int4 *__restrict__ sv,
              const float4 *__restrict__ sc, const float2 *__restrict__ U, const double *__restrict__ area_v,
              const float *__restrict__ eta, double g, int nonlinear_h, double *__restrict__ out)
{
    __shared__ double sh[2][32];
    const int b = blockIdx.x;
    double vol = 0.0, en = 0.0;
    for (int v = basin_v[b] + threadIdx.x; v < basin_v[b + 1]; v += blockDim.x) {
        const double e = (double)eta[v];
        vol += area_v[v] * e;
        en += area_v[v] * 0.5 * g * e * e;
    }
    for (int s = basin_slot[b] + threadIdx.x; s < basin_slot[b + 1]; s += blockDim.x) {
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
        out[2 * b] = vol;
        out[2 * b + 1] = en;
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

// ---------------------------------------------------------------------------------
// Persistent kernel: one launch per baroclinic step, one block per patch, all blocks
// resident (cooperative launch). A block keeps the elevation of its own and halo
// vertices and the per-corner fluxes in shared memory, and the transport and the
// compensated flux sum of its slots in registers, for all M substeps. When it fits
// (CACHED), the patch's static slot data, incidence lists, 1/A_v and halo index list
// are also copied to shared memory once per step.
//
// Substep m: update the interior slots (corners all own vertices); wait until the
// patches owning the halo vertices have published elevation m; read it from the
// exchange buffer of parity m; update the other slots; vertex pass; write the own
// vertices' new elevation to the exchange buffer of parity m+1 and publish m+1.
// A block overwrites an exchange buffer two substeps later, after its neighbours
// have published a count that shows they finished reading it.
struct PArgs {
    const int *patch_slot, *patch_own, *patch_int, *patch_v, *patch_halo, *halo_v, *patch_nbr, *nbr;
    const int *vcsr_off;
    const uint32_t *vcsr;
    const int4 *sv;
    const ushort4 *sl;
    const float4 *sg, *sc;
    const float2 *R;
    float2 *U, *Umean;
    const float *inv_av;
    const float *patch_dt;
    const float *eta_in;
    float *eta_out;
    float *eta_sum;         // null, or sum over the substeps of eta^0 .. eta^{M-1} (own vertices)
    const float *W;         // null, or the freshwater flux of each vertex (Eq. 4.5)
    float *xb[2];
    unsigned *flags;        // [npatch], then the abort word
    unsigned *status;
    const int *pack_patch;  // patch of each block: pack_patch[pack_base + blockIdx.x]
    int pack_base;
    StepArgs a;
    int M, npatch;
    // shared-memory carve-up (CACHED), in bytes from the dynamic shared base
    int off_flux, off_g, off_c, off_r, off_l, off_off, off_csr, off_inv, off_halo;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Flags are padded to one 128-byte line each so that publishing and polling
// patches do not contend for the same L2 line.
constexpr int kFlagStride = 32;

// Warp 0 waits until every neighbour of patch p has published `target` substeps
// (lanes poll one neighbour each). Returns false when the wait gave up; it then sets
// the timeout bit and the abort word, which makes every other wait give up too.
__device__ bool warp0_wait_neighbours(const PArgs &P, int p, unsigned target)
{
    const int lane = threadIdx.x & 31;
    const int b = P.patch_nbr[p], e = P.patch_nbr[p + 1];
    const unsigned *abort_word = P.flags + (size_t)P.npatch * kFlagStride;
    bool ok = true;
    for (int k = b + lane; k < e && ok; k += 32) {
        const unsigned *f = P.flags + (size_t)P.nbr[k] * kFlagStride;
        const long long t0 = clock64();
        while (ld_acquire_gpu(f) < target) {
            if (ld_relaxed_gpu(abort_word) != 0u || clock64() - t0 > P.a.wait_cycles) {
                ok = false;
                break;
            }
            __nanosleep(20);
        }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && lane == 0) {
        atomicOr(P.status, 2u);
        atomicExch(P.flags + (size_t)P.npatch * kFlagStride, 1u);
    }
    return ok;
}

// Element update of one slot (Eq. 4.10, first row, and the theta-weighted flux);
// coef = (dt A_e, g H0_e, f dt / 2, 1 / (1 + (f dt / 2)^2)).
template <int NONLIN>
__device__ __forceinline__ void element_update(const float e0, const float e1, const float e2, const float4 g,
                                               const float4 coef, const float2 r, float2 &u, float2 &shi,
                                               float2 &slo, bool owned, float *flux3, float theta,
                                               float one_p_theta, float dt, float gconst)
{
    const float d0 = e0 - e2, d1 = e1 - e2;
    const float gx = d0 * g.x + d1 * g.z;
    const float gy = d0 * g.y + d1 * g.w;
    float gH = coef.y;
    if (NONLIN) gH += gconst * ((e0 + e1 + e2) * (1.0f / 3.0f));
    const float aa = coef.z;
    const float rx = u.x + aa * u.y + dt * (r.x - gH * gx);
    const float ry = u.y - aa * u.x + dt * (r.y - gH * gy);
    const float nx = (rx + aa * ry) * coef.w;
    const float ny = (ry - aa * rx) * coef.w;
    const float fx = one_p_theta * nx - theta * u.x;
    const float fy = one_p_theta * ny - theta * u.y;
    u = make_float2(nx, ny);
    if (owned) {
        two_sum_acc(shi.x, slo.x, fx);
        two_sum_acc(shi.y, slo.y, fy);
    }
    const float c0 = coef.x * (fx * g.x + fy * g.y);
    const float c1 = coef.x * (fx * g.z + fy * g.w);
    flux3[0] = c0;
    flux3[1] = c1;
    flux3[2] = -(c0 + c1);
}

__device__ __forceinline__ float4 slot_coef(const float4 c, const StepArgs &a, float dt)
{
    const float aa = c.z * (0.5f * dt);
    return make_float4(dt * c.x, a.g * c.y, aa, 1.0f / (1.0f + aa * aa));
}

template <int SPT, int NONLIN, int CACHED, int FW>
__global__ void __launch_bounds__(1024, 1) k_persistent(PArgs P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_ok;
    const int p = P.pack_patch[P.pack_base + blockIdx.x];
    const int T = blockDim.x;
    const int s0 = P.patch_slot[p], ns = P.patch_slot[p + 1] - s0;
    const int nown_s = P.patch_own[p], nint = P.patch_int[p];
    const int v0 = P.patch_v[p], nown = P.patch_v[p + 1] - v0;
    const int hb = P.patch_halo[p], nhalo = P.patch_halo[p + 1] - hb;
    const int c0 = P.vcsr_off[v0], ncsr = P.vcsr_off[v0 + nown] - c0;
    const StepArgs a = P.a;
    const float dt = P.patch_dt[p];

    float *seta = reinterpret_cast<float *>(smem_raw);
    float *sflux = reinterpret_cast<float *>(smem_raw + P.off_flux);
    float4 *s_g = reinterpret_cast<float4 *>(smem_raw + P.off_g);
    float4 *s_c = reinterpret_cast<float4 *>(smem_raw + P.off_c);
    float2 *s_r = reinterpret_cast<float2 *>(smem_raw + P.off_r);
    ushort4 *s_l = reinterpret_cast<ushort4 *>(smem_raw + P.off_l);
    unsigned short *s_off = reinterpret_cast<unsigned short *>(smem_raw + P.off_off);
    unsigned short *s_csr = reinterpret_cast<unsigned short *>(smem_raw + P.off_csr);
    float *s_inv = reinterpret_cast<float *>(smem_raw + P.off_inv);
    int *s_halo = reinterpret_cast<int *>(smem_raw + P.off_halo);

    for (int i = threadIdx.x; i < nown; i += T) seta[i] = P.eta_in[v0 + i];
    for (int i = threadIdx.x; i < nhalo; i += T) seta[nown + i] = P.eta_in[P.halo_v[hb + i]];
    if (CACHED) {
        for (int i = threadIdx.x; i < ns; i += T) {
            s_g[i] = P.sg[s0 + i];
            s_c[i] = slot_coef(P.sc[s0 + i], a, dt);
            s_r[i] = P.R[s0 + i];
            s_l[i] = P.sl[s0 + i];
        }
        for (int i = threadIdx.x; i <= nown; i += T) s_off[i] = (unsigned short)(P.vcsr_off[v0 + i] - c0);
        // cached incidence entries hold the flux index 3 * slot + corner directly
        for (int k = threadIdx.x; k < ncsr; k += T) {
            const uint32_t q = P.vcsr[c0 + k];
            s_csr[k] = (unsigned short)(3u * (q >> 2) + (q & 3u));
        }
        for (int i = threadIdx.x; i < nown; i += T) s_inv[i] = P.inv_av[v0 + i];
        for (int i = threadIdx.x; i < nhalo; i += T) s_halo[i] = P.halo_v[hb + i];
    }
    float2 u[SPT], shi[SPT], slo[SPT];
#pragma unroll
    for (int j = 0; j < SPT; j++) {
        const int i = threadIdx.x + j * T;
        u[j] = i < ns ? P.U[s0 + i] : make_float2(0.0f, 0.0f);
        shi[j] = make_float2(0.0f, 0.0f);
        slo[j] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();

    const float one_p_theta = 1.0f + a.theta;
    // Element update of the slots with local index in [lo, hi). Corner elevations of
    // own vertices come from shared memory; with `halo_src` set, those of halo vertices
    // are read from that exchange buffer (boundary slots, substeps m >= 1).
    auto elements = [&](int lo, int hi, const float *halo_src) {
#pragma unroll
        for (int j = 0; j < SPT; j++) {
            const int i = threadIdx.x + j * T;
            if (i >= lo && i < hi) {
                float4 g, coef;
                float2 r;
                ushort4 l;
                if (CACHED) {
                    g = s_g[i];
                    coef = s_c[i];
                    r = s_r[i];
                    l = s_l[i];
                } else {
                    g = P.sg[s0 + i];
                    coef = slot_coef(P.sc[s0 + i], a, dt);
                    r = P.R[s0 + i];
                    l = P.sl[s0 + i];
                }
                float e0, e1, e2;
                if (halo_src) {
                    const int *hid = CACHED ? s_halo : P.halo_v + hb;
                    e0 = l.x < nown ? seta[l.x] : __ldcg(halo_src + hid[l.x - nown]);
                    e1 = l.y < nown ? seta[l.y] : __ldcg(halo_src + hid[l.y - nown]);
                    e2 = l.z < nown ? seta[l.z] : __ldcg(halo_src + hid[l.z - nown]);
                } else {
                    e0 = seta[l.x];
                    e1 = seta[l.y];
                    e2 = seta[l.z];
                }
                element_update<NONLIN>(e0, e1, e2, g, coef, r, u[j], shi[j], slo[j], i < nown_s, sflux + 3 * i,
                                       a.theta, one_p_theta, dt, a.g);
            }
        }
    };

    for (int m = 0; m < P.M; m++) {
        if (m == 0) {
            elements(0, ns, nullptr);
        } else {
            elements(0, nint, nullptr);
            if (threadIdx.x < 32) {
                const bool ok = warp0_wait_neighbours(P, p, (unsigned)m);
                if (threadIdx.x == 0) s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) break;
            elements(nint, ns, P.xb[m & 1]);
        }
        __syncthreads();

        // vertex pass; the new elevation of own vertices also goes to the exchange buffer
        const bool more = m + 1 < P.M;
        float *xout = P.xb[(m + 1) & 1];
        bool bad = false;
        for (int i = threadIdx.x; i < nown; i += T) {
            float sum = 0.0f, inv;
            if (CACHED) {
                const int k1 = s_off[i + 1];
                for (int k = s_off[i]; k < k1; k++) sum += sflux[s_csr[k]];
                inv = s_inv[i];
            } else {
                const int k1 = P.vcsr_off[v0 + i + 1];
                for (int k = P.vcsr_off[v0 + i]; k < k1; k++) {
                    const uint32_t q = P.vcsr[k];
                    sum += sflux[3 * (q >> 2) + (q & 3u)];
                }
                inv = P.inv_av[v0 + i];
            }
            float e = seta[i] + sum * inv;
            if (FW) e -= dt * __ldg(P.W + v0 + i);
            if (P.eta_sum) P.eta_sum[v0 + i] += seta[i];
            seta[i] = e;
            if (more) __stcg(xout + v0 + i, e);
            bad |= !(fabsf(e) <= a.eta_bound);
        }
        if (bad) atomicOr(P.status, 1u);
        __syncthreads();
        if (!more) break;
        if (threadIdx.x == 0 && p != a.silent_patch) {
            __threadfence();
            st_release_gpu(P.flags + (size_t)p * kFlagStride, (unsigned)(m + 1));
        }
    }
    __syncthreads();

    for (int i = threadIdx.x; i < nown; i += T) P.eta_out[v0 + i] = seta[i];
#pragma unroll
    for (int j = 0; j < SPT; j++) {
        const int i = threadIdx.x + j * T;
        if (i < ns) {
            P.U[s0 + i] = u[j];
            if (i < nown_s) {
                const int w = P.sv[s0 + i].w;
                P.Umean[w] = make_float2((shi[j].x + slo[j].x) * a.inv_M, (shi[j].y + slo[j].y) * a.inv_M);
            }
        }
    }
}

// fw: the freshwater flux is set (a separate instantiation keeps the path without it
// free of the extra load and branch)
template <int SPT, int CACHED>
void *persistent_fn(int nonlin, int fw)
{
    if (fw) return nonlin ? (void *)k_persistent<SPT, 1, CACHED, 1> : (void *)k_persistent<SPT, 0, CACHED, 1>;
    return nonlin ? (void *)k_persistent<SPT, 1, CACHED, 0> : (void *)k_persistent<SPT, 0, CACHED, 0>;
}

void *persistent_kernel(int spt, int nonlin, int cached, int fw)
{
    if (cached) {
        switch (spt) {
        case 1: return persistent_fn<1, 1>(nonlin, fw);
        case 2: return persistent_fn<2, 1>(nonlin, fw);
        case 3: return persistent_fn<3, 1>(nonlin, fw);
        case 4: return persistent_fn<4, 1>(nonlin, fw);
        default: return nullptr;
        }
    }
    switch (spt) {
    case 1: return persistent_fn<1, 0>(nonlin, fw);
    case 2: return persistent_fn<2, 0>(nonlin, fw);
    case 3: return persistent_fn<3, 0>(nonlin, fw);
    case 4: return persistent_fn<4, 0>(nonlin, fw);
    case 6: return persistent_fn<6, 0>(nonlin, fw);
    case 8: return persistent_fn<8, 0>(nonlin, fw);
    default: return nullptr;
    }
}

size_t flag_bytes(int npatch) { return sizeof(unsigned) * ((size_t)npatch + 1) * kFlagStride; }

struct SmemLayout {
    int off_flux, off_g, off_c, off_r, off_l, off_off, off_csr, off_inv, off_halo;
    size_t total_plain, total_cached;
};

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

SmemLayout smem_layout(const DevMesh &m)
{
    SmemLayout L;
    size_t o = align16(sizeof(float) * (size_t)m.max_patch_local);
    L.off_flux = (int)o;
    o = align16(o + sizeof(float) * 3 * (size_t)m.max_patch_slots);
    L.total_plain = o;
    L.off_g = (int)o;
    o += sizeof(float4) * (size_t)m.max_patch_slots;
    L.off_c = (int)o;
    o += sizeof(float4) * (size_t)m.max_patch_slots;
    L.off_r = (int)o;
    o = align16(o + sizeof(float2) * (size_t)m.max_patch_slots);
    L.off_l = (int)o;
    o = align16(o + sizeof(ushort4) * (size_t)m.max_patch_slots);
    L.off_inv = (int)o;
    o = align16(o + sizeof(float) * (size_t)m.max_patch_vertices);
    L.off_halo = (int)o;
    o = align16(o + sizeof(int) * (size_t)m.max_patch_halo);
    L.off_off = (int)o;
    o = align16(o + sizeof(unsigned short) * ((size_t)m.max_patch_vertices + 1));
    L.off_csr = (int)o;
    o = align16(o + sizeof(unsigned short) * (size_t)m.max_patch_csr);
    L.total_cached = o;
    return L;
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
                           cudaStream_t stream, const SubstepViscArgs *visc)
{
    const int threads = block > 0 ? block : 256;
    const size_t smem = sizeof(float) * 3 * (size_t)m.max_patch_slots;
    const float *ein = s.eta[parity];
    float *eout = s.eta[parity ^ 1];
    SubstepVisc vis{};
    const float2 *uin = s.U;
    float2 *uout = s.U;
    if (visc) {
        vis.vnb = m.visc_nb;
        vis.vgeo = m.visc_geo;
        vis.V0 = s.V0;
        vis.va = visc->va;
        vis.start = visc->start;
        uin = visc->U_in;
        uout = visc->U_out;
    }
#define SESW_SUBSTEP(NL, VI)                                                                                      \
    k_substep<NL, VI><<<m.npatch, threads, smem, stream>>>(                                                      \
        m.slot_v, m.slot_g, m.slot_c, s.R, uin, uout, s.S_hi, s.S_lo, m.patch_slot, m.patch_own, m.patch_v,      \
        m.vcsr_off, m.vcsr, m.inv_av, ein, eout, m.patch_dt, s.eta_sum, s.W, vis, a, s.status)
    if (a.nonlinear_h) {
        if (visc) SESW_SUBSTEP(1, 1); else SESW_SUBSTEP(1, 0);
    } else {
        if (visc) SESW_SUBSTEP(0, 1); else SESW_SUBSTEP(0, 0);
    }
#undef SESW_SUBSTEP
    return cudaGetLastError();
}

// The dynamic shared-memory limit is a process-wide attribute of each kernel, shared by
// every context of the process; it is always raised to the device's opt-in maximum
// (a permission, nothing is reserved) so that contexts with different patch sizes
// never lower it under each other's launches.
int optin_smem()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}

// Raise a kernel's dynamic shared-memory limit to the most the device allows it (the
// opt-in maximum less the kernel's static shared memory); returns that limit or -1.
int raise_smem_limit(const void *fn)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    const int limit = optin_smem() - (int)fa.sharedSizeBytes;
    if (limit <= 0 || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return limit;
}

cudaError_t substep_smem_attr(const DevMesh &m)
{
    const size_t need = sizeof(float) * 3 * (size_t)m.max_patch_slots;
    const void *fns[6] = {(const void *)k_substep<0, 0>, (const void *)k_substep<1, 0>,
                          (const void *)k_substep<0, 1>, (const void *)k_substep<1, 1>,
                          (const void *)k_sesm<0>, (const void *)k_sesm<1>};
    for (const void *fn : fns) {
        const int l = raise_smem_limit(fn);
        if (l < 0 || (size_t)l < need) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_sesm(const DevMesh &m, const DevState &s, const StepArgs &a, const SesmPtrs &q, int block,
                        cudaStream_t stream)
{
    const int threads = block > 0 ? block : 256;
    const size_t smem = sizeof(float) * 3 * (size_t)m.max_patch_slots;
    SesmLevels L;
    L.u1 = q.u1;
    L.u2 = q.u2;
    L.u3 = q.u3;
    L.u0 = q.u0;
    L.e0 = q.e0;
    L.e1 = q.e1;
    L.e2 = q.e2;
    L.e3 = q.e3;
    L.enew = q.enew;
    L.update = q.update;
    L.vertex = q.vertex;
    if (a.nonlinear_h)
        k_sesm<1><<<m.npatch, threads, smem, stream>>>(m.slot_v, m.slot_g, m.slot_c, s.R, s.S_hi, s.S_lo,
                                                       m.patch_slot, m.patch_own, m.patch_v, m.vcsr_off, m.vcsr,
                                                       m.inv_av, m.patch_dt, s.W, L, a, s.status);
    else
        k_sesm<0><<<m.npatch, threads, smem, stream>>>(m.slot_v, m.slot_g, m.slot_c, s.R, s.S_hi, s.S_lo,
                                                       m.patch_slot, m.patch_own, m.patch_v, m.vcsr_off, m.vcsr,
                                                       m.inv_av, m.patch_dt, s.W, L, a, s.status);
    return cudaGetLastError();
}

cudaError_t launch_viscosity(const DevMesh &m, const DevState &s, const ViscArgs &v, int parity, float2 *out,
                             cudaStream_t stream)
{
    k_viscosity<<<grid_for(m.nslot, kAuxThreads), kAuxThreads, 0, stream>>>(
        m.slot_v, m.slot_c, s.U, m.visc_nb, m.visc_geo, s.eta[parity], v, out, m.nslot);
    return cudaGetLastError();
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

cudaError_t launch_gather_scaled(const DevMesh &m, const float *x, double scale, double *out, cudaStream_t stream)
{
    k_gather_scaled<<<grid_for(m.nv, kAuxThreads), kAuxThreads, 0, stream>>>(m.vperm, x, scale, out, m.nv);
    return cudaGetLastError();
}

cudaError_t launch_gather_state(const DevMesh &m, const DevState &s, int parity, double *eta, double *U,
                                double *Umean, cudaStream_t stream)
{
    k_gather<<<grid_for(m.nv > m.nslot ? m.nv : m.nslot, kAuxThreads), kAuxThreads, 0, stream>>>(
        m.slot_v, m.vperm, m.eperm, s.eta[parity], s.U, s.Umean, eta, U, Umean, m.nv, m.nslot);
    return cudaGetLastError();
}

size_t persistent_flag_bytes(int npatch) { return flag_bytes(npatch); }

PersistentPlan persistent_plan(const DevMesh &m, int blocks_per_sm)
{
    PersistentPlan plan;
    int dev = 0, smem_optin = 0, smem_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return plan;
    }
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    const int max_threads = 1024 / blocks_per_sm;
    // fewest slots per thread such that one block of at most max_threads covers the
    // largest patch; the block is then sized to that patch (multiple of 32)
    static const int spts[] = {1, 2, 3, 4, 6, 8};
    int spt = 0, t = 0;
    for (int cand : spts) {
        const int need = (m.max_patch_slots + cand - 1) / cand;
        const int tt = ((need + 31) / 32) * 32;
        if (tt <= max_threads) {
            spt = cand;
            t = tt < 32 ? 32 : tt;
            break;
        }
    }
    if (!spt) return plan;
    const SmemLayout L = smem_layout(m);
    // per block: the opt-in limit, and the SM's capacity shared by blocks_per_sm blocks
    // (1 KB of each block's share is reserved by the system, plus the kernel's static shared)
    size_t budget = (size_t)smem_optin - 1024;
    const size_t share = (size_t)smem_sm / (size_t)blocks_per_sm;
    if (share < 2048) return plan;
    budget = std::min(budget, share - 2048);
    // the cached variant indexes incidence entries and offsets with 16 bits
    int cached = (spt <= 4 && L.total_cached <= budget && m.max_patch_csr < 65536 && m.max_patch_slots < 16384) ? 1 : 0;
    const size_t smem = cached ? L.total_cached : L.total_plain;
    if (smem > budget) return plan;
    // every variant the plan may launch must reach blocks_per_sm resident blocks
    for (int nonlin = 0; nonlin < 2; nonlin++)
        for (int fw = 0; fw < 2; fw++) {
            void *fn = persistent_kernel(spt, nonlin, cached, fw);
            int occ = 0;
            if (!fn || raise_smem_limit(fn) < (int)smem ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, t, smem) != cudaSuccess ||
                occ < blocks_per_sm) {
                cudaGetLastError();
                return plan;
            }
        }
    plan.slots_per_thread = spt;
    plan.threads = t;
    plan.cached = cached;
    plan.smem = smem;
    return plan;
}

cudaError_t persistent_prepare(const PersistentPlan &plan)
{
    for (int nonlin = 0; nonlin < 2; nonlin++)
        for (int fw = 0; fw < 2; fw++) {
            void *fn = persistent_kernel(plan.slots_per_thread, nonlin, plan.cached, fw);
            if (!fn || raise_smem_limit(fn) < (int)plan.smem) return cudaErrorInvalidValue;
        }
    return cudaSuccess;
}

cudaError_t launch_persistent(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity,
                              const PersistentPlan &plan, cudaStream_t stream)
{
    PArgs P;
    P.patch_slot = m.patch_slot;
    P.patch_own = m.patch_own;
    P.patch_int = m.patch_int;
    P.patch_v = m.patch_v;
    P.patch_halo = m.patch_halo;
    P.halo_v = m.halo_v;
    P.patch_nbr = m.patch_nbr;
    P.nbr = m.nbr;
    P.vcsr_off = m.vcsr_off;
    P.vcsr = m.vcsr;
    P.sv = m.slot_v;
    P.sl = m.slot_l;
    P.sg = m.slot_g;
    P.sc = m.slot_c;
    P.R = s.R;
    P.U = s.U;
    P.Umean = s.Umean;
    P.inv_av = m.inv_av;
    P.patch_dt = m.patch_dt;
    P.eta_in = s.eta[parity];
    P.eta_out = s.eta[parity ^ 1];
    P.eta_sum = s.eta_sum;
    P.W = s.W;
    P.xb[0] = s.xbuf[0];
    P.xb[1] = s.xbuf[1];
    P.flags = s.flags;
    P.status = s.status;
    P.a = a;
    P.M = M;
    P.npatch = m.npatch;
    const SmemLayout L = smem_layout(m);
    P.off_flux = L.off_flux;
    P.off_g = L.off_g;
    P.off_c = L.off_c;
    P.off_r = L.off_r;
    P.off_l = L.off_l;
    P.off_off = L.off_off;
    P.off_csr = L.off_csr;
    P.off_inv = L.off_inv;
    P.off_halo = L.off_halo;
    P.pack_patch = m.pack_patch;
    void *fn = persistent_kernel(plan.slots_per_thread, a.nonlinear_h, plan.cached, s.W != nullptr);
    if (!fn) return cudaErrorInvalidValue;
    // one cooperative launch per pack; all packs of a step use the same elevation parity
    for (size_t k = 0; k + 1 < m.pack_off.size(); k++) {
        P.pack_base = m.pack_off[k];
        const int nblocks = m.pack_off[k + 1] - m.pack_off[k];
        void *args[] = {&P};
        cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(plan.threads), args, plan.smem, stream);
        if (e != cudaSuccess) return e;
    }
    // flags and the abort word start from zero in the next step
    return cudaMemsetAsync(s.flags, 0, flag_bytes(m.npatch), stream);
}

cudaError_t launch_diagnostics_basins(const DevMesh &m, const DevState &s, const StepArgs &a, int parity,
                                      double *out, cudaStream_t stream)
{
    k_diag_basins<<<m.nbasin, kAuxThreads, 0, stream>>>(m.basin_v, m.basin_slot, m.slot_v, m.slot_c, s.U, m.area_v,
                                                       s.eta[parity], a.g64, a.nonlinear_h, out);
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
