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
// in expectation.
//
// The rounding itself is the conversion instruction's stochastic mode
// (cvt.rs.f16x2.f32): it converts two FP32 values into the two halves of one
// 32-bit word and takes the random bits of both from a 32-bit operand.  The
// two x-neighbours 2m and 2m + 1 of a row (the row pitch is even, so node
// indices pair the same way) form pair m: plane k of both nodes is rounded
// by one conversion with the random word of (pair, plane, step), node 2m + 1
// in the upper half, node 2m in the lower one.  A kernel that updates one
// node alone runs the same conversion and keeps its own half, so the stored
// bits do not depend on how the nodes were grouped into threads.
//
// The random words are counter based: the 32-bit integer hash "lowbias32"
// (constants from C. Wellons' hash prospector) of the pair index and the step
// number gives one uniformly distributed word per pair, and plane k takes
// that word times the k-th odd constant (a bijection of the word, so every
// plane's word is uniform; correlation between the planes of one pair
// changes only the variance of the rounding, not its mean).
struct Dither {
    uint32_t h;
    uint32_t upper;  // the node is the odd member of its pair
    __device__ __forceinline__ Dither(uint32_t node, uint32_t step) {
        uint32_t x = (node >> 1) ^ (step * 0x9E3779B9u);
        x ^= x >> 16;
        x *= 0x7feb352du;
        x ^= x >> 15;
        x *= 0x846ca68bu;
        x ^= x >> 16;
        h = x;
        upper = node & 1u;
    }
    // random word of plane k (k < 17) for both nodes of the pair
    __device__ __forceinline__ uint32_t word(int k) const {
        constexpr uint32_t M[17] = {0x9E3779B1u, 0x85EBCA77u, 0xC2B2AE3Du, 0x27D4EB2Fu, 0x165667B1u,
                                    0xD3A2646Du, 0xFD7046C5u, 0xB55A4F09u, 0x68E31DA5u, 0x1B873593u,
                                    0xCC9E2D51u, 0xE6546B65u, 0xF1357AEBu, 0x2545F491u, 0x9B05688Bu,
                                    0x510E527Fu, 0x1F83D9ABu};
        return h * M[k];
    }
};

// hi, lo (already divided by the storage scale) rounded to FP16
// stochastically with the random bits of rbits: hi into the upper half of
// the result, lo into the lower half.
__device__ __forceinline__ uint32_t half2_sr(float hi, float lo, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}

// One node's value v of plane k, rounded as it is when stored with its pair.
__device__ __forceinline__ __half half_sr_node(float v, const Dither& d, int k) {
    const uint32_t r = half2_sr(v, v, d.word(k));
    return __ushort_as_half((unsigned short)(d.upper ? (r >> 16) : (r & 0xFFFFu)));
}

// Store of the 17 post-collision values of one node into FP16 planes,
// rounded stochastically (dither != nullptr) or to nearest.
template <class R>
__device__ __forceinline__ void store_planes_half(__half* __restrict__ d, long long pl, const R* fo, const R* ho,
                                                  float inv_scale, Dither* dither) {
    if (dither) {
#pragma unroll
        for (int i = 1; i < 9; ++i) d[(i - 1) * pl] = half_sr_node(float(fo[i]) * inv_scale, *dither, i - 1);
#pragma unroll
        for (int i = 0; i < 9; ++i) d[(8 + i) * pl] = half_sr_node(float(ho[i]) * inv_scale, *dither, 8 + i);
        return;
    }
#pragma unroll
    for (int i = 1; i < 9; ++i) d[(i - 1) * pl] = __float2half_rn(float(fo[i]) * inv_scale);
#pragma unroll
    for (int i = 0; i < 9; ++i) d[(8 + i) * pl] = __float2half_rn(float(ho[i]) * inv_scale);
}

// Store of the 17 values of the two nodes of one pair (a: the even node at
// d, b: the odd node at d + 1; d 4-byte aligned), one 32-bit store per
// plane.  dither: the pair's random words (constructed from either node).
template <class R>
__device__ __forceinline__ void store_pair_half(__half* __restrict__ d, int pl, const R* fa, const R* ha,
                                                const R* fb, const R* hb, float inv_scale, const Dither& dither) {
    uint32_t* w = reinterpret_cast<uint32_t*>(d);
    const int pw = pl >> 1;  // plane stride in 32-bit words (the plane size is even)
#pragma unroll
    for (int i = 1; i < 9; ++i)
        w[(i - 1) * pw] = half2_sr(float(fb[i]) * inv_scale, float(fa[i]) * inv_scale, dither.word(i - 1));
#pragma unroll
    for (int i = 0; i < 9; ++i)
        w[(8 + i) * pw] = half2_sr(float(hb[i]) * inv_scale, float(ha[i]) * inv_scale, dither.word(8 + i));
}

}  // namespace lbm
