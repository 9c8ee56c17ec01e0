// The ratio test of Sec. 2.3.1 step (4), decided exactly.
#pragma once
#include <cstdint>

namespace cm {

// dis(q1) < t_r dis(q2) with t_r = num / den, on exact squared distances.
// FP32 when sqrt(d1 / d2) is at least 1e-3 away from t_r (FP32 error is ~1e-7
// there), FP64 re-check otherwise (d^2 < 2^24, so den^2 d1^2 and num^2 d2^2
// are exact in FP64).
__device__ __forceinline__ bool ratio_pass(uint32_t d1, uint32_t d2, int num, int den, uint32_t& rechecks) {
    if (d2 == 0u) return false;
    const float r = sqrtf((float)d1 / (float)d2);
    const float tr = (float)num / (float)den;
    if (fabsf(r - tr) >= 1e-3f) return r < tr;
    ++rechecks;
    return (double)den * (double)den * (double)d1 < (double)num * (double)num * (double)d2;
}

}  // namespace cm
