// Staging of uint8 descriptor rows as BF16 tensor-core operands (K-major, no
// swizzle, the layout of cm_tc.cuh).  An integer 0..255 is exact in BF16, so
// products of two such values and their sums below 2^24 are exact in the
// FP32 accumulator.
#pragma once
#include <cstdint>

#include "cm_internal.h"
#include "cm_tc.cuh"

namespace cm {
namespace stage {

// Bytes b0 and b0+1 of w as two BF16 values.  The byte is placed under the
// exponent of 2^23 by one byte permute (2^23 + b as FP32) and 2^23 subtracted;
// an integer 0..255 has at most 8 significant bits, so the FP32 upper half is
// its exact BF16.
__device__ __forceinline__ uint32_t u8x2_to_bf16x2(uint32_t w, int b0) {
    const float f0 = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540 + b0)) - 8388608.f;
    const float f1 = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7541 + b0)) - 8388608.f;
    return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// One uint8 row (8 x 16 bytes, or zeros) from global memory.
__device__ __forceinline__ void load_row(const uint8_t* src, bool have, uint4 (&v)[8]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = have ? __ldg(reinterpret_cast<const uint4*>(src) + c) : make_uint4(0, 0, 0, 0);
}

// The row into row r of a K-major BF16 operand tile of `rows` rows; returns
// its squared norm.
__device__ __forceinline__ uint32_t store_row(const uint4 (&v)[8], unsigned char* tile, int r, int rows) {
    uint32_t nn = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        nn = __dp4a(v[c].x, v[c].x, nn);
        nn = __dp4a(v[c].y, v[c].y, nn);
        nn = __dp4a(v[c].z, v[c].z, nn);
        nn = __dp4a(v[c].w, v[c].w, nn);
        uint4 lo, hi;
        lo.x = u8x2_to_bf16x2(v[c].x, 0); lo.y = u8x2_to_bf16x2(v[c].x, 2);
        lo.z = u8x2_to_bf16x2(v[c].y, 0); lo.w = u8x2_to_bf16x2(v[c].y, 2);
        hi.x = u8x2_to_bf16x2(v[c].z, 0); hi.y = u8x2_to_bf16x2(v[c].z, 2);
        hi.z = u8x2_to_bf16x2(v[c].w, 0); hi.w = u8x2_to_bf16x2(v[c].w, 2);
        *reinterpret_cast<uint4*>(tile + tc::chunk_off(r, 2 * c, rows)) = lo;
        *reinterpret_cast<uint4*>(tile + tc::chunk_off(r, 2 * c + 1, rows)) = hi;
    }
    return nn;
}

// The 8 MMAs (K = 16 each) of a 128 x N x 128 BF16 product of an A tile of
// 128 rows and a B tile of N rows, both staged by store_row.
__device__ __forceinline__ void mma_128xN(uint32_t tmem_d, const unsigned char* A, const unsigned char* B, int N) {
    const uint32_t lbo_a = (128 / 8) * 128, lbo_b = (uint32_t)(N / 8) * 128;
    const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B), idesc = tc::idesc_f16(128, N, 1);
#pragma unroll
    for (int ks = 0; ks < kDim / 16; ++ks)
        tc::mma_f16(tmem_d, tc::smem_desc(a0 + ks * 2 * lbo_a, lbo_a, 128), tc::smem_desc(b0 + ks * 2 * lbo_b, lbo_b, 128),
                    idesc, ks != 0);
}

}  // namespace stage
}  // namespace cm
