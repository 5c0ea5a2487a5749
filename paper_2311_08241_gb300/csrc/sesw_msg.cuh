// Message inputs of the surrogate's message layers, in one form for the fused tensor-core
// layer of the forward pass (sesw_tc.cu) and for the kernels that rebuild the inputs for the
// backward pass (sesw_surrogate.cu): both round the same way, so the weight gradients see
// the bfloat16 values the forward pass multiplied.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sesw {

// x rounded to the nearest bfloat16 value
__device__ __forceinline__ float bf16_value(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Element message of one hidden channel: L (sum_k dphi_k/dx h_k, sum_k dphi_k/dy h_k) over the
// corners, g = (dphi0/dx, dphi0/dy, dphi1/dx, dphi1/dy) and dphi_2 = -(dphi_0 + dphi_1).
__device__ __forceinline__ float2 msg_elem_grad(float4 g, float h0, float h1, float h2, float L)
{
    const float gx = __fmaf_rn(-__fadd_rn(g.x, g.z), h2, __fmaf_rn(g.z, h1, __fmul_rn(g.x, h0)));
    const float gy = __fmaf_rn(-__fadd_rn(g.y, g.w), h2, __fmaf_rn(g.w, h1, __fmul_rn(g.y, h0)));
    return make_float2(__fmul_rn(L, gx), __fmul_rn(L, gy));
}

// Vertex message: the area-weighted sum over the vertex's triangles, accumulated in incidence
// order (s <- s + A_e h_e), then scaled by 1 / sum A_e.
__device__ __forceinline__ float msg_vert_acc(float s, float area, float h) { return __fmaf_rn(area, h, s); }
__device__ __forceinline__ float msg_vert_mean(float s, float inv_area) { return __fmul_rn(s, inv_area); }

}  // namespace sesw
