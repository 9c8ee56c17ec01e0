// Arithmetic of the SAO local constraint shared by the host form
// (cm_sao.cpp) and the GPU form (cm_sao_gpu.cu), so that both take every
// decision with the same operations and roundings: FP64 distances and cross
// products without fused multiply-adds, the angular order, and the cyclic
// edit distance of two label sequences.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define CM_SAO_HD __host__ __device__ __forceinline__
#else
#define CM_SAO_HD inline
#endif

namespace cm {
namespace sao {

constexpr int kMaxK = 32;   // neighbours per side at most (the GPU form takes up to 16)

CM_SAO_HD int imin(int a, int b) { return a < b ? a : b; }
CM_SAO_HD int imax(int a, int b) { return a > b ? a : b; }

// Correctly rounded FP64 operations that are never fused into an FMA (the
// host form is compiled without contraction).
CM_SAO_HD double mul(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
CM_SAO_HD double add(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
CM_SAO_HD double sub(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}

// Squared distance from (ax, ay) to (bx, by).
CM_SAO_HD double d2(double ax, double ay, double bx, double by) {
    const double dx = sub(bx, ax), dy = sub(by, ay);
    return add(mul(dx, dx), mul(dy, dy));
}

// true when ray a = (ax, ay) comes before ray b in angular order from the +x
// axis, in [0, 2 pi): half-planes first, then the sign of the cross product;
// a zero vector has angle 0; ties by label.
CM_SAO_HD bool ray_less(double ax, double ay, int al, double bx, double by, int bl) {
    const int ha = (ay < 0 || (ay == 0 && ax < 0)) ? 1 : 0;
    const int hb = (by < 0 || (by == 0 && bx < 0)) ? 1 : 0;
    if (ha != hb) return ha < hb;
    const bool za = ay == 0 && ax >= 0, zb = by == 0 && bx >= 0;   // angle exactly 0 (or a zero vector)
    if (za || zb) return za && zb ? al < bl : za;
    const double cr = sub(mul(ax, by), mul(ay, bx));
    if (cr != 0) return cr > 0;
    return al < bl;
}

// Unit-cost edit distance of a and b, or any value above `cap` once every
// entry of a DP row exceeds it (the distance can only grow from there).
CM_SAO_HD int levenshtein(const int32_t* a, int na, const int32_t* b, int nb, int cap) {
    int row[kMaxK + 1];
    for (int j = 0; j <= nb; ++j) row[j] = j;
    for (int i = 1; i <= na; ++i) {
        int diag = row[0];
        row[0] = i;
        int lo = i;
        for (int j = 1; j <= nb; ++j) {
            const int up = row[j];
            const int v = imin(imin(up + 1, row[j - 1] + 1), diag + (a[i - 1] == b[j - 1] ? 0 : 1));
            row[j] = v;
            diag = up;
            lo = imin(lo, v);
        }
        if (lo > cap) return lo;
    }
    return row[nb];
}

// Cyclic edit distance: the smallest edit distance over rotations of a (an
// alignment of two rotated sequences can be re-cut where b starts, giving one
// of the same cost between a rotation of a and b itself).  The rotation that
// starts with b's first label goes first (exact 0 for an unchanged order),
// the others are bounded by the best so far.
CM_SAO_HD int cyclic_edit_distance(const int32_t* a, int na, const int32_t* b, int nb) {
    if (na == 0 || nb == 0) return imax(na, nb);
    int r0 = 0;
    for (int t = 0; t < na; ++t)
        if (a[t] == b[0]) r0 = t;
    if (na == nb) {
        int t = 0;
        while (t < na && a[(r0 + t) % na] == b[t]) ++t;
        if (t == na) return 0;
    }
    int32_t rot[kMaxK];
    int best = na + nb;
    for (int step = 0; step < na && best > 0; ++step) {
        const int r = (r0 + step) % na;
        for (int t = 0; t < na; ++t) rot[t] = a[(r + t) % na];
        best = imin(best, levenshtein(rot, na, b, nb, best - 1));
    }
    return best;
}

}  // namespace sao
}  // namespace cm
