// Device helpers shared by the kernel translation units of libsesw (not part of the
// public interface).
#pragma once

#include <cuda_runtime.h>

namespace sesw {

// Packed FP32 pairs. Blackwell issues one instruction for an (x, y) pair of FP32 additions,
// multiplications or fused multiply-adds (FADD2/FMUL2/FFMA2), each lane rounded exactly as
// the scalar __fadd_rn/__fmul_rn/__fmaf_rn would round it. The vector quantities of the
// substep (gradients, transports, sums) are (x, y) pairs, so they take half the instructions.
__device__ __forceinline__ float2 pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

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

// The same two-sum on both components of a pair at once (per lane identical to two_sum_acc;
// PACKED = 0 runs the two scalar ones).
template <int PACKED = 1>
__device__ __forceinline__ void two_sum_acc2(float2 &hi, float2 &lo, float2 x)
{
    if (!PACKED) {
        two_sum_acc(hi.x, lo.x, x.x);
        two_sum_acc(hi.y, lo.y, x.y);
        return;
    }
    const float2 m1 = splat(-1.0f);
    const float2 s = __fadd2_rn(hi, x);
    const float2 bp = __ffma2_rn(hi, m1, s);
    const float2 ap = __ffma2_rn(bp, m1, s);
    const float2 err = __fadd2_rn(__ffma2_rn(ap, m1, hi), __ffma2_rn(bp, m1, x));
    hi = s;
    lo = __fadd2_rn(lo, err);
}

// Element update of one slot in the dissipative forward-backward substep (Eq. 4.10, first
// row) and the theta-weighted transport that the continuity row and the time mean of
// Eq. (4.12) use. Every SE kernel calls this one function, and its roundings are spelled
// out, so that the same inputs give bitwise the same transport and flux whichever kernel
// or launch layout computes them.
//   e0, e1, e2  corner elevations; grad eta = (e0 - e2) dphi0 + (e1 - e2) dphi1
//   g           (dphi0/dx, dphi0/dy, dphi1/dx, dphi1/dy)
//   gH0         g H0_e; NONLIN adds g (e0 + e1 + e2) / 3 (H = H0 + eta)
//   aa, inv     f dt / 2 and 1 / (1 + aa^2) (Crank-Nicolson Coriolis)
//   r           frozen forcing R (m^2/s^2)
//   u           in: U^m, out: U^{m+1}
// Returns F = (1 + theta) U^{m+1} - theta U^m.
// PACKED = 0 computes the same roundings with scalar instructions (bitwise the same result).
template <int NONLIN, int PACKED = 1>
__device__ __forceinline__ float2 se_transport(float e0, float e1, float e2, float4 g, float gH0, float gconst,
                                               float aa, float inv, float dt, float2 r, float one_p_theta,
                                               float theta, float2 &u)
{
    const float d0 = __fsub_rn(e0, e2), d1 = __fsub_rn(e1, e2);
    if (!PACKED) {
        const float gx = __fmaf_rn(d1, g.z, __fmul_rn(d0, g.x));
        const float gy = __fmaf_rn(d1, g.w, __fmul_rn(d0, g.y));
        float gH = gH0;
        if (NONLIN) gH = __fmaf_rn(gconst, __fmul_rn(__fadd_rn(__fadd_rn(e0, e1), e2), 1.0f / 3.0f), gH0);
        const float rx = __fmaf_rn(dt, __fmaf_rn(-gH, gx, r.x), __fmaf_rn(aa, u.y, u.x));
        const float ry = __fmaf_rn(dt, __fmaf_rn(-gH, gy, r.y), __fmaf_rn(-aa, u.x, u.y));
        const float nx = __fmul_rn(__fmaf_rn(aa, ry, rx), inv);
        const float ny = __fmul_rn(__fmaf_rn(-aa, rx, ry), inv);
        const float2 F = make_float2(__fmaf_rn(one_p_theta, nx, __fmul_rn(-theta, u.x)),
                                     __fmaf_rn(one_p_theta, ny, __fmul_rn(-theta, u.y)));
        u = make_float2(nx, ny);
        return F;
    }
    const float2 grad = __ffma2_rn(splat(d1), pair(g.z, g.w), __fmul2_rn(splat(d0), pair(g.x, g.y)));
    float gH = gH0;
    if (NONLIN) gH = __fmaf_rn(gconst, __fmul_rn(__fadd_rn(__fadd_rn(e0, e1), e2), 1.0f / 3.0f), gH0);
    // right-hand side: U + aa (U_y, -U_x) + dt (R - g H grad eta)
    const float2 t = __ffma2_rn(splat(-gH), grad, r);
    const float2 w = __ffma2_rn(pair(aa, -aa), pair(u.y, u.x), u);
    const float2 rr = __ffma2_rn(splat(dt), t, w);
    // Crank-Nicolson solve: U' = (rr + aa (rr_y, -rr_x)) / (1 + aa^2)
    const float2 n = __fmul2_rn(__ffma2_rn(pair(aa, -aa), pair(rr.y, rr.x), rr), splat(inv));
    const float2 F = __ffma2_rn(splat(one_p_theta), n, __fmul2_rn(splat(-theta), u));
    u = n;
    return F;
}

// Contributions of the transport F of a triangle to the median-dual cells of its three
// corners: c_k = w F . dphi_k with w = dt A_e (k = 0, 1), c_2 = -(c_0 + c_1).
template <int PACKED = 1>
__device__ __forceinline__ void corner_fluxes(float2 F, float4 g, float w, float *out3)
{
    if (!PACKED) {
        const float c0 = __fmul_rn(w, __fmaf_rn(F.y, g.y, __fmul_rn(F.x, g.x)));
        const float c1 = __fmul_rn(w, __fmaf_rn(F.y, g.w, __fmul_rn(F.x, g.z)));
        out3[0] = c0;
        out3[1] = c1;
        out3[2] = -__fadd_rn(c0, c1);
        return;
    }
    const float c0 = __fmul_rn(w, __fmaf_rn(F.y, g.y, __fmul_rn(F.x, g.x)));
    const float c1 = __fmul_rn(w, __fmaf_rn(F.y, g.w, __fmul_rn(F.x, g.z)));
    out3[0] = c0;
    out3[1] = c1;
    out3[2] = -__fadd_rn(c0, c1);
}

// The vertex update of Eq. (4.10), second row: eta + (sum of the corner contributions,
// added in the vertex's incidence order) / A_v.
__device__ __forceinline__ float vertex_eta(float eta, float sum, float inv_area)
{
    return __fmaf_rn(sum, inv_area, eta);
}

// The SESM substep (Eqs. 4.7-4.8) in one form for every kernel, with its roundings
// spelled out like se_transport's.
// Momentum: U^m = U^{m-1} + dt (-f e_z x U_AB^{m-1} - g H_AM grad(eta_AM) + R), from the
// corner values of eta_AM; H_AM = H0_e (+ the corner mean of eta_AM with NONLIN).
template <int NONLIN>
__device__ __forceinline__ float2 sesm_momentum(float e0, float e1, float e2, float4 g, float H0, float gconst,
                                                float f, float dt, float2 r, float2 u1, float2 uab)
{
    const float d0 = __fsub_rn(e0, e2), d1 = __fsub_rn(e1, e2);
    const float2 grad = __ffma2_rn(splat(d1), pair(g.z, g.w), __fmul2_rn(splat(d0), pair(g.x, g.y)));
    float H = H0;
    if (NONLIN) H = __fadd_rn(H0, __fmul_rn(__fadd_rn(__fadd_rn(e0, e1), e2), 1.0f / 3.0f));
    const float gH = __fmul_rn(gconst, H);
    // -f e_z x U_AB = (f U_AB_y, -f U_AB_x)
    const float2 t = __fadd2_rn(__ffma2_rn(splat(-gH), grad, __fmul2_rn(pair(f, -f), pair(uab.y, uab.x))), r);
    return __ffma2_rn(splat(dt), t, u1);
}

// AB3 transport ab0 U^m + ab1 U^{m-1} + ab2 U^{m-2} (Eq. 4.7).
__device__ __forceinline__ float2 sesm_ab3(float2 u0, float2 ua, float2 ub, float ab0, float ab1, float ab2)
{
    return __ffma2_rn(splat(ab2), ub, __ffma2_rn(splat(ab1), ua, __fmul2_rn(splat(ab0), u0)));
}

// AM4 elevation am0 eta^{m+1} + am1 eta^m + am2 eta^{m-1} + am3 eta^{m-2} (Eq. 4.7).
__device__ __forceinline__ float sesm_am4(float e, float e1, float e2, float e3, float am0, float am1, float am2,
                                          float am3)
{
    return __fmaf_rn(am3, e3, __fmaf_rn(am2, e2, __fmaf_rn(am1, e1, __fmul_rn(am0, e))));
}

// The device's opt-in shared-memory limit per block (0 when it cannot be read).
int optin_smem();

// Raise a kernel's dynamic shared-memory limit to the most the device allows it (the
// opt-in maximum less the kernel's static shared memory); returns that limit or -1.
int raise_smem_limit(const void *fn);

}  // namespace sesw
