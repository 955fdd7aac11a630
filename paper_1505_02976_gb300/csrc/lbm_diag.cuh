// lbm_diag.cuh -- device helpers shared by the diagnostics kernels and the
// batched step's Nusselt kernel (internal).
#pragma once

#include "lbm_internal.h"

namespace lbm {

// Macroscopic state of node (x, y) after streaming: its own moments, or for
// a wall node the boundary state of Sec. 3.4.
template <class R, class S>
__device__ __forceinline__ State<R> node_state_at(const KConst<R>& k, const S* __restrict__ src, int x, int y) {
    const WallInfo w = classify(k, x, y);
    const int xs = w.wall ? w.xs : x, ys = w.wall ? w.ys : y;
    Pops<R> P;
    pull(k, src, xs, ys, P);
    CellC<R> cs = cell_consts(k, node_eps(k, xs, ys));
    cs.ay = row_ay(k, ys);
    const State<R> s = node_moments(k, cs, P.f, P.h);
    if (!w.wall) return s;
    R thff = R(0);
    if (w.tside < 0) thff = (pull_hsum<R, R, S>(k, src, w.xff, w.yff) + R(0.5) * k.Q) * k.inv_sigma;
    const R thb = w.tside >= 0 ? k.T_bc[w.tside] - k.T0 : R(0);
    CellC<R> cb = cell_consts(k, node_eps(k, x, y));
    cb.ay = row_ay(k, y);
    return wall_state(k, cb, w, s, thff, thb);
}

// (u_x, u_y, T - T0) of node (x, y) after streaming: the step's fast path
// for interior nodes (same moments as node_state_at up to rounding order),
// node_state_at for wall nodes.
template <class R, class S>
__device__ __forceinline__ void node_u_th(const KConst<R>& k, const S* __restrict__ src, int x, int y, R* ux,
                                          R* uy, R* th) {
    if (is_wall(k, x, y)) {
        const State<R> s = node_state_at(k, src, x, y);
        *ux = s.ux;
        *uy = s.uy;
        *th = s.th;
        return;
    }
    Pops<R> P;
    pull(k, src, x, y, P);
    FastState<R> s;
    if (k.eps_field) {
        KConst<R> kc = k;
        apply_eps(kc, node_eps(k, x, y));
        s = fast_moments(kc, P.f, P.h, y);
    } else {
        s = fast_moments(k, P.f, P.h, y);
    }
    *ux = s.ux;
    *uy = s.uy;
    *th = s.th;
}

// T of node (x, y) in FP64 from the stored populations, with the wall rules
// of Sec. 3.4 (Dirichlet value, or Eq. TNEESApGra on adiabatic walls).
template <class R, class S>
__device__ double node_T(const KConst<R>& k, const DiagConst& d, const S* __restrict__ src, int x, int y) {
    const WallInfo w = classify(k, x, y);
    if (!w.wall) return d.T0 + (pull_hsum<double, R, S>(k, src, x, y) + 0.5 * d.Q) * d.inv_sigma;
    if (w.tside >= 0) return d.T_bc[w.tside];
    const double tf = (pull_hsum<double, R, S>(k, src, w.xs, w.ys) + 0.5 * d.Q) * d.inv_sigma;
    const double tff = (pull_hsum<double, R, S>(k, src, w.xff, w.yff) + 0.5 * d.Q) * d.inv_sigma;
    return d.T0 + (4.0 * tf - tff) / 3.0;
}

constexpr int kReduceBlock = 256;

// Fixed-order block sum of one value per thread (deterministic).
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;  // valid in thread 0
}

// Grid of one block row per lattice row.
inline dim3 row_grid(int nx, int ny, int bx) { return dim3((unsigned)((nx + bx - 1) / bx), (unsigned)ny); }

}  // namespace lbm
