// lbm_half.cuh -- FP16 storage of the populations: stochastic rounding of
// the stored values (device side).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

// Stochastic rounding of FP16 stores.  Near a steady state the same value
// rounds the same way step after step, so round-to-nearest acts as a
// persistent source of heat and momentum at every node (larger than the
// buoyancy force per step at these Mach numbers).  Rounding up with
// probability equal to the discarded fraction keeps every stored value exact
// in expectation.  The random bits are counter based: the 32-bit integer hash
// "lowbias32" (constants from C. Wellons' hash prospector) of the node index
// and the step number gives one uniformly distributed word per node; value k
// of the node takes the top 13 bits of that word times the k-th odd constant
// (a bijection of the word, so each value's 13 bits are uniform; correlation
// between the values of one node changes only the variance of the rounding,
// not its mean).  13 bits = the FP32 mantissa bits below FP16's last bit.
struct Dither {
    uint32_t h;
    __device__ __forceinline__ Dither(uint32_t node, uint32_t step) {
        uint32_t x = node ^ (step * 0x9E3779B9u);
        x ^= x >> 16;
        x *= 0x7feb352du;
        x ^= x >> 15;
        x *= 0x846ca68bu;
        x ^= x >> 16;
        h = x;
    }
    // 13 random bits for value k (k < 17)
    __device__ __forceinline__ uint32_t bits(int k) const {
        constexpr uint32_t M[17] = {0x9E3779B1u, 0x85EBCA77u, 0xC2B2AE3Du, 0x27D4EB2Fu, 0x165667B1u,
                                    0xD3A2646Du, 0xFD7046C5u, 0xB55A4F09u, 0x68E31DA5u, 0x1B873593u,
                                    0xCC9E2D51u, 0xE6546B65u, 0xF1357AEBu, 0x2545F491u, 0x9B05688Bu,
                                    0x510E527Fu, 0x1F83D9ABu};
        return (h * M[k]) >> 19;
    }
};

// v (already divided by the storage scale) rounded to FP16 stochastically:
// add 13 random bits below FP16's last mantissa bit, then truncate.
__device__ __forceinline__ __half half_sr(float v, uint32_t r) {
    return __float2half_rz(__uint_as_float(__float_as_uint(v) + r));
}

// Store of the 17 post-collision values of one node into FP16 planes,
// rounded stochastically (dither != nullptr) or to nearest.
template <class R>
__device__ __forceinline__ void store_planes_half(__half* __restrict__ d, long long pl, const R* fo, const R* ho,
                                                  float inv_scale, Dither* dither) {
    if (dither) {
#pragma unroll
        for (int i = 1; i < 9; ++i) d[(i - 1) * pl] = half_sr(float(fo[i]) * inv_scale, dither->bits(i - 1));
#pragma unroll
        for (int i = 0; i < 9; ++i) d[(8 + i) * pl] = half_sr(float(ho[i]) * inv_scale, dither->bits(8 + i));
        return;
    }
#pragma unroll
    for (int i = 1; i < 9; ++i) d[(i - 1) * pl] = __float2half_rn(float(fo[i]) * inv_scale);
#pragma unroll
    for (int i = 0; i < 9; ++i) d[(8 + i) * pl] = __float2half_rn(float(ho[i]) * inv_scale);
}

}  // namespace lbm
