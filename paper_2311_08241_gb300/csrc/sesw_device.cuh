// Device helpers shared by the kernel translation units of libsesw (not part of the
// public interface).
#pragma once

#include <cuda_runtime.h>

namespace sesw {

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

// The device's opt-in shared-memory limit per block (0 when it cannot be read).
int optin_smem();

// Raise a kernel's dynamic shared-memory limit to the most the device allows it (the
// opt-in maximum less the kernel's static shared memory); returns that limit or -1.
int raise_smem_limit(const void *fn);

}  // namespace sesw
