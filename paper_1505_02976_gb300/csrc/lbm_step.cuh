// lbm_step.cuh -- device code shared by the single-lattice and the batched
// step kernels (internal): block size, the store of one node and the
// out-of-line wall-node update.
#pragma once

#include "lbm_diag.cuh"

namespace lbm {

constexpr int kStepBlock = 128;
// Resident blocks per SM the step kernel is compiled for: 8 x 128 threads
// caps the FP32 kernel at 64 registers; the FP64 kernel keeps room to avoid
// spilling.
#ifndef LBM_F32_STEP_BLOCKS
#define LBM_F32_STEP_BLOCKS 8
#endif
template <class R> struct StepOccupancy { static constexpr int blocks = LBM_F32_STEP_BLOCKS; };
template <> struct StepOccupancy<double> { static constexpr int blocks = 3; };

template <class R, class S>
__device__ __forceinline__ void store_node(const KConst<R>& k, S* __restrict__ dst, long long at,
                                           const R* fo, const R* ho, Dither* dither = nullptr) {
    store_planes<S, R>(dst + at, k.plane, fo, ho, k.inv_scale, dither);
}

// Wall node of one step: the generic update of its x_f neighbour's pulled
// populations (NEES rebuild and boundary collision, see
// node_update_generic).  Kept out of line: only the 4(N - 1) wall threads
// take it.
template <class R, class S>
__device__ __noinline__ void wall_update(const KConst<R>& k, const S* __restrict__ src,
                                         S* __restrict__ dst, int x, int y, uint32_t step) {
    const WallInfo w = classify(k, x, y);
    Pops<R> P;
    pull(k, src, w.xs, w.ys, P);
    R in[17], out[17];
#pragma unroll
    for (int i = 1; i < 9; ++i) in[i - 1] = P.f[i];
#pragma unroll
    for (int i = 0; i < 9; ++i) in[8 + i] = P.h[i];
    R thff = R(0);
    if (w.tside < 0) thff = (pull_hsum<R, R, S>(k, src, w.xff, w.yff) + R(0.5) * k.Q) * k.inv_sigma;
    const R thb = w.tside >= 0 ? k.T_bc[w.tside] - k.T0 : R(0);
    node_update_generic(k, w, in, node_eps(k, w.xs, w.ys), node_eps(k, x, y), thff, thb, row_ay(k, w.ys),
                        row_ay(k, y), out);
    if (!isfinite(out[0] + out[8])) atomicOr(k.flag, 1);
    R fo[9], ho[9];
#pragma unroll
    for (int i = 1; i < 9; ++i) fo[i] = out[i - 1];
#pragma unroll
    for (int i = 0; i < 9; ++i) ho[i] = out[8 + i];
    Dither dither((uint32_t)(y * k.pitch + x), step);
    store_node(k, dst, (long long)y * k.pitch + x, fo, ho, &dither);
}

}  // namespace lbm
