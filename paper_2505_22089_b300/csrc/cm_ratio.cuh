// The ratio test of Sec. 2.3.1 step (4), decided exactly.
#pragma once
#include <cstdint>

namespace cm {

// dis(q1) < t_r dis(q2) with t_r = num / den, on exact squared distances.
// Decided in FP32 when r = sqrt(d1 / d2) is at least 1e-3 away from t_r, by
// FP64 otherwise (a re-check, counted).  The band test needs no division or
// square root: r < t_r - 1e-3 exactly when d1 < (t_r - 1e-3)^2 d2, and
// r > t_r + 1e-3 when d1 > (t_r + 1e-3)^2 d2 (d1, d2 < 2^24 are exact in FP32
// and the products carry a relative error near 1e-7, far inside the band, so
// a pass or fail decided there is the exact one).  lo and hi are those two
// squares (ratio_band; lo = -1 when t_r <= 1e-3, as r >= 0).  In the band,
// den^2 d1 and num^2 d2 are exact in FP64.
__device__ __forceinline__ bool ratio_pass(uint32_t d1, uint32_t d2, int num, int den, float lo, float hi,
                                           uint32_t& rechecks) {
    if (d2 == 0u) return false;
    const float f1 = (float)d1, f2 = (float)d2;
    if (f1 < lo * f2) return true;
    if (f1 > hi * f2) return false;
    ++rechecks;
    return (double)den * (double)den * (double)d1 < (double)num * (double)num * (double)d2;
}

}  // namespace cm
