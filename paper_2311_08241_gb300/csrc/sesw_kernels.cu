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
// old level while this block writes the new one); element state is only ever written
// by the block that holds the slot (with the viscosity, transports are double-buffered
// too and neighbours are read at the old level). The persistent step kernel is in
// sesw_persistent.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sesw_device.cuh"
#include "sesw_internal.h"

namespace sesw {

namespace {

constexpr int kSubstepMaxThreads = 1024;
constexpr int kAuxThreads = 256;

// Per-slot tables of the barotropic viscosity (see DevMesh::visc_q).
struct ViscTables {
    const int4 *q, *c;
    const float4 *a, *b, *r;
    const float2 *r2;
};

// Barotropic viscous regularisation, Eq. (viscosity_BT), of slot s (depth H, transport
// Us, corner elevations e[3], area A_e): a two-point flux across each edge k (corners k
// and k+1) with a neighbour,
//   u = U / H here and on the neighbour, du = rot(u_nb) - u (ROT: the neighbour's frame
//   is turned; otherwise rot is the identity), flux = (H + H_nb)/2 (A_bg L/d + C_v |du| L^2/d) du,
//   R_hV = (1/A_e) sum_edges flux,
// with H_nb = H0_nb (+ the mean of eta over the edge's two corners and the neighbour's
// opposite corner when nonlinear). Neighbours are read from their owner slots, so every
// copy of an element computes the same value.
template <int ROT>
__device__ __forceinline__ float2 visc_of(int s, float H, float2 Us, const float e[3], float area, const ViscTables T,
                                          const float2 *U, const float *__restrict__ eta, const ViscArgs va)
{
    const float ux = Us.x / H, uy = Us.y / H;
    const int4 tq = T.q[s], tc = T.c[s];
    const float4 ta = T.a[s], tb = T.b[s];
    const int q[3] = {tq.x, tq.y, tq.z};
    const int oc[3] = {tc.x, tc.y, tc.z};
    const float h0[3] = {__int_as_float(tq.w), __int_as_float(tc.w), ta.w};
    const float la[3] = {ta.x, ta.y, ta.z};
    const float lb[3] = {tb.x, tb.y, tb.z};
    float cs[3] = {1.0f, 1.0f, 1.0f}, sn[3] = {0.0f, 0.0f, 0.0f};
    if (ROT) {
        const float4 r = T.r[s];
        const float2 r2 = T.r2[s];
        cs[0] = r.x; sn[0] = r.y; cs[1] = r.z; sn[1] = r.w; cs[2] = r2.x; sn[2] = r2.y;
    }
    float fx = 0.0f, fy = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (q[k] < 0) continue;
        float Hn = h0[k];
        if (va.nonlinear_h) Hn += (e[k] + e[(k + 1) % 3] + eta[oc[k]]) * (1.0f / 3.0f);
        const float2 Uq = U[q[k]];
        const float nx = Uq.x / Hn, ny = Uq.y / Hn;
        float dx, dy;
        if (ROT) {
            dx = (cs[k] * nx - sn[k] * ny) - ux;
            dy = (sn[k] * nx + cs[k] * ny) - uy;
        } else {
            dx = nx - ux;
            dy = ny - uy;
        }
        const float kq = 0.5f * (H + Hn) * (va.background * la[k] + va.flow * sqrtf(dx * dx + dy * dy) * lb[k]);
        fx += kq * dx;
        fy += kq * dy;
    }
    return make_float2(fx / area, fy / area);
}

// Viscosity inputs of the substep kernel (VISC = 1, or 2 with turned neighbour frames):
// transports are read from U_in (level m, also the neighbours') and written to U_out
// (level m + 1), and the forcing of the substep is R + (R_hV - V0) with V0 the value at
// substep 0 of the step (start = 1 stores it; Sect. 2.2 subtracts the term's start value).
struct SubstepVisc {
    ViscTables T;
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
    const float dt = patch_dt[p], half_dt = __fmul_rn(0.5f, dt);
    const int s0 = patch_slot[p];
    const int n = patch_slot[p + 1] - s0;
    const int nown = patch_own[p];
    const float one_p_theta = __fadd_rn(1.0f, a.theta);

    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = s0 + i;
        const int4 v = sv[s];
        const float4 g = sg[s];
        const float4 c = sc[s];
        float2 r = R[s];
        const float2 u = U_in[s];
        const float e0 = eta_in[v.x], e1 = eta_in[v.y], e2 = eta_in[v.z];
        if (VISC) {
            float H = c.y;
            if (NONLIN) H += (e0 + e1 + e2) * (1.0f / 3.0f);
            const float ev[3] = {e0, e1, e2};
            const float2 V = visc_of<VISC == 2>(s, H, u, ev, c.x, vis.T, U_in, eta_in, vis.va);
            if (vis.start) {
                vis.V0[s] = V;      // R' = R + (V - V) = R
            } else {
                const float2 z = vis.V0[s];
                r = make_float2(r.x + (V.x - z.x), r.y + (V.y - z.y));
            }
        }
        const float aa = __fmul_rn(c.z, half_dt);
        const float inv = __frcp_rn(__fmaf_rn(aa, aa, 1.0f));
        float2 un = u;
        const float2 F = se_transport<NONLIN>(e0, e1, e2, g, __fmul_rn(a.g, c.y), a.g, aa, inv, dt, r, one_p_theta,
                                              a.theta, un);
        U_out[s] = un;
        if (i < nown) {
            float2 hi = Shi[s], lo = Slo[s];
            two_sum_acc2(hi, lo, F);
            Shi[s] = hi;
            Slo[s] = lo;
        }
        corner_fluxes(F, g, __fmul_rn(dt, c.x), sflux + 3 * i);
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
        float e = vertex_eta(eta_in[v], sum, inv_av[v]);
        if (W) e = __fmaf_rn(-dt, W[v], e);
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
            const float2 uab = sesm_ab3(u1, u2, u3, a.ab0, a.ab1, a.ab2);
            float em[3];
            const int vv[3] = {v.x, v.y, v.z};
#pragma unroll
            for (int k = 0; k < 3; k++)
                em[k] = sesm_am4(L.e0[vv[k]], L.e1[vv[k]], L.e2[vv[k]], L.e3[vv[k]], a.am0, a.am1, a.am2, a.am3);
            u0 = sesm_momentum<NONLIN>(em[0], em[1], em[2], g, c.y, a.g, c.z, dt, r, u1, uab);
            L.u0[s] = u0;
        } else {
            u0 = L.u0[s];
        }
        if (!L.vertex) continue;
        const float2 F = sesm_ab3(u0, u1, u2, a.ab0, a.ab1, a.ab2);
        if (i < nown) {
            float2 hi = Shi[s], lo = Slo[s];
            two_sum_acc2(hi, lo, F);
            Shi[s] = hi;
            Slo[s] = lo;
        }
        corner_fluxes(F, g, __fmul_rn(dt, sc[s].x), sflux + 3 * i);
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
        float e = vertex_eta(L.e0[v], sum, inv_av[v]);
        if (W) e = __fmaf_rn(-dt, W[v], e);
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
template <int ROT>
__global__ void __launch_bounds__(kAuxThreads)
k_viscosity(const int4 *__restrict__ sv, const float4 *__restrict__ sc, const float2 *__restrict__ U,
            const ViscTables T, const float *__restrict__ eta, ViscArgs va, float2 *__restrict__ out, int nslot)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslot; s += gridDim.x * blockDim.x) {
        const int4 v = sv[s];
        if (v.w < 0) continue;
        const float4 c = sc[s];
        const float e[3] = {eta[v.x], eta[v.y], eta[v.z]};
        float H = c.y;
        if (va.nonlinear_h) H += (e[0] + e[1] + e[2]) * (1.0f / 3.0f);
        out[v.w] = visc_of<ROT>(s, H, U[s], e, c.x, T, U, eta, va);
    }
}

__global__ void k_scatter_eta(const int *__restrict__ vperm, const double *__restrict__ in, float *__restrict__ eta,
                              int nv)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
        eta[v] = (float)in[vperm[v]];
}

// Copy a caller-order [ne][2] field into every slot (owner and guest copies alike); slot_e
// holds each slot's caller element.
__global__ void k_scatter_slots(const int *__restrict__ slot_e, const double *__restrict__ in,
                                float2 *__restrict__ out, int nslot)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslot; s += gridDim.x * blockDim.x) {
        const size_t e = (size_t)slot_e[s];
        out[s] = make_float2((float)in[2 * e], (float)in[2 * e + 1]);
    }
}

__global__ void k_gather_scaled(const int *__restrict__ vperm, const float *__restrict__ x, double scale,
                                double *__restrict__ out, int nv)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
        out[vperm[v]] = (double)x[v] * scale;
}

// The state in caller order, written in order (the reads follow the inverse maps): eta of caller
// vertex v, U from the owner slot and <<U>> of caller element e.
__global__ void k_gather(const int *__restrict__ vinv, const int *__restrict__ einv, const int *__restrict__ eown,
                         const float *__restrict__ eta, const float2 *__restrict__ U,
                         const float2 *__restrict__ Umean, double *__restrict__ eta_out,
                         double *__restrict__ U_out, double *__restrict__ Um_out, int nv, int ne)
{
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (eta_out)
        for (int v = t0; v < nv; v += stride) eta_out[v] = (double)eta[vinv[v]];
    for (int e = t0; e < ne; e += stride) {
        if (U_out) {
            const float2 u = U[eown[e]];
            U_out[2 * (size_t)e] = (double)u.x;
            U_out[2 * (size_t)e + 1] = (double)u.y;
        }
        if (Um_out) {
            const float2 u = Umean[einv[e]];
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
k_diag_partial(const int4 *__restrict__ sv, const double *__restrict__ area_e, const double *__restrict__ h0_e,
               const float2 *__restrict__ U, const double *__restrict__ area_v, const float *__restrict__ eta, int nv,
               int nslot, double g, int nonlinear_h, double *__restrict__ part)
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
        double H = h0_e[c.w];
        if (nonlinear_h) H += ((double)eta[c.x] + (double)eta[c.y] + (double)eta[c.z]) / 3.0;
        const float2 u = U[s];
        en += area_e[c.w] * ((double)u.x * u.x + (double)u.y * u.y) / (2.0 * H);
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
              const double *__restrict__ area_e, const double *__restrict__ h0_e, const float2 *__restrict__ U,
              const double *__restrict__ area_v, const float *__restrict__ eta, double g, int nonlinear_h,
              double *__restrict__ out)
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
        double H = h0_e[c.w];
        if (nonlinear_h) H += ((double)eta[c.x] + (double)eta[c.y] + (double)eta[c.z]) / 3.0;
        const float2 u = U[s];
        en += area_e[c.w] * ((double)u.x * u.x + (double)u.y * u.y) / (2.0 * H);
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
        vis.T = ViscTables{m.visc_q, m.visc_c, m.visc_a, m.visc_b, m.visc_r, m.visc_r2};
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
    const int vk = visc ? (m.visc_rot ? 2 : 1) : 0;
    if (a.nonlinear_h) {
        if (vk == 2) SESW_SUBSTEP(1, 2); else if (vk == 1) SESW_SUBSTEP(1, 1); else SESW_SUBSTEP(1, 0);
    } else {
        if (vk == 2) SESW_SUBSTEP(0, 2); else if (vk == 1) SESW_SUBSTEP(0, 1); else SESW_SUBSTEP(0, 0);
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
    const void *fns[8] = {(const void *)k_substep<0, 0>, (const void *)k_substep<1, 0>,
                          (const void *)k_substep<0, 1>, (const void *)k_substep<1, 1>,
                          (const void *)k_substep<0, 2>, (const void *)k_substep<1, 2>,
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
    const ViscTables T{m.visc_q, m.visc_c, m.visc_a, m.visc_b, m.visc_r, m.visc_r2};
    if (m.visc_rot)
        k_viscosity<1><<<grid_for(m.nslot, kAuxThreads), kAuxThreads, 0, stream>>>(m.slot_v, m.slot_c, s.U, T,
                                                                                  s.eta[parity], v, out, m.nslot);
    else
        k_viscosity<0><<<grid_for(m.nslot, kAuxThreads), kAuxThreads, 0, stream>>>(m.slot_v, m.slot_c, s.U, T,
                                                                                  s.eta[parity], v, out, m.nslot);
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
        k_scatter_slots<<<grid_for(m.nslot, kAuxThreads), kAuxThreads, 0, stream>>>(m.slot_e, U, s.U, m.nslot);
    return cudaGetLastError();
}

cudaError_t launch_scatter_forcing(const DevMesh &m, const DevState &s, const double *R, cudaStream_t stream)
{
    k_scatter_slots<<<grid_for(m.nslot, kAuxThreads), kAuxThreads, 0, stream>>>(m.slot_e, R, s.R, m.nslot);
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
    k_gather<<<grid_for(m.nv > m.ne ? m.nv : m.ne, kAuxThreads), kAuxThreads, 0, stream>>>(
        m.vinv, m.einv, m.eown, s.eta[parity], s.U, s.Umean, eta, U, Umean, m.nv, m.ne);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics_basins(const DevMesh &m, const DevState &s, const StepArgs &a, int parity,
                                      double *out, cudaStream_t stream)
{
    k_diag_basins<<<m.nbasin, kAuxThreads, 0, stream>>>(m.basin_v, m.basin_slot, m.slot_v, m.area_e, m.h0_e, s.U,
                                                       m.area_v, s.eta[parity], a.g64, a.nonlinear_h, out);
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
    k_diag_partial<<<nblocks, kAuxThreads, 0, stream>>>(m.slot_v, m.area_e, m.h0_e, s.U, m.area_v, s.eta[parity],
                                                        m.nv, m.nslot, a.g64, a.nonlinear_h, s.diag_part);
    k_diag_final<<<1, kAuxThreads, 0, stream>>>(s.diag_part, nblocks, s.diag_out);
    return cudaGetLastError();
}

}  // namespace sesw
