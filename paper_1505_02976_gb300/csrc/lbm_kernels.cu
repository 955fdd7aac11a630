// lbm_kernels.cu -- the fused step kernel of a single lattice.
//
// k_step: one thread per node, pull streaming from the ping buffer, all the
// per-node arithmetic of the step in registers, and one write of the 17
// post-collision planes to the pong buffer.  Wall nodes take the NEES rebuild
// inside the same launch (an out-of-line path that pulls the populations of
// the wall node's fluid neighbour x_f instead of its own).  FP32 and FP16
// lattices walled on all four sides run the kernel with TMA-staged rows
// (lbm_step_tma.cu) unless the global-load kernel is selected.
#include <math.h>

#include "lbm_step.cuh"

namespace lbm {



// The fused step: one thread per node; interior nodes take the fast path,
// wall nodes the NEES path.  TAU1: tau_f = tau_T = 1 (the paper's default,
// Sec. 4), where the (1 - 1/tau) terms vanish.
template <class R, class S, bool EPS_FIELD, bool TAU1>
__global__ void __launch_bounds__(kStepBlock, StepOccupancy<R>::blocks)
k_step(const __grid_constant__ KConst<R> k, const S* __restrict__ src, S* __restrict__ dst, uint32_t step) {
    // Programmatic dependent launch: let the next step's blocks be scheduled
    // while this grid drains, and wait here until the previous step's grid
    // has completed and its writes are visible (no-op without the launch
    // attribute).  Both are hardware-managed; nothing spins.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int x = blockIdx.x * kStepBlock + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= k.nx) return;
    if (is_wall(k, x, y)) {
        wall_update(k, src, dst, x, y, step);
        return;
    }
    if constexpr (EPS_FIELD) {
        KConst<R> kc = k;
        apply_eps(kc, node_eps(k, x, y));
        interior_update<R, S, TAU1>(kc, src, dst, x, y, step);
    } else {
        interior_update<R, S, TAU1>(k, src, dst, x, y, step);
    }
}

template <class R, class S>
__global__ void k_init(const __grid_constant__ KConst<R> k, S* __restrict__ dst,
                       const double* __restrict__ T, const double* __restrict__ ux,
                       const double* __restrict__ uy, double T_init) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= k.nx) return;
    const long long c = (long long)y * k.nx + x;
    State<R> s;
    s.th = R((T ? T[c] : T_init) - double(k.T0));
    s.ux = ux ? R(ux[c]) : R(0);
    s.uy = uy ? R(uy[c]) : R(0);
    s.p = R(0);
    s.Fx = s.Fy = R(0);
    s.Sxx = s.Sxy = s.Syy = R(0);
    s.gx = s.gy = R(0);
    EqTerms<R> e;
    eq_terms(k, cell_consts(k, node_eps(k, x, y)), s, e);
    store_node(k, dst, (long long)y * k.pitch + x, e.fe, e.he);
}

// ------------------------------------------------------------------ launchers

template <class R, class S>
cudaError_t launch_step(const KConst<R>& k, const S* src, S* dst, uint32_t step, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = row_grid(k.nx, k.ny, kStepBlock);
    cfg.blockDim = dim3(kStepBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool tau1 = k.omf == R(0) && k.omT == R(0);
    if (k.eps_field)
        return tau1 ? cudaLaunchKernelEx(&cfg, k_step<R, S, true, true>, k, src, dst, step)
                    : cudaLaunchKernelEx(&cfg, k_step<R, S, true, false>, k, src, dst, step);
    return tau1 ? cudaLaunchKernelEx(&cfg, k_step<R, S, false, true>, k, src, dst, step)
                : cudaLaunchKernelEx(&cfg, k_step<R, S, false, false>, k, src, dst, step);
}

template <class R, class S>
cudaError_t launch_init(const KConst<R>& k, S* dst, const double* T, const double* ux,
                        const double* uy, double T_init, cudaStream_t st) {
    k_init<R, S><<<row_grid(k.nx, k.ny, 128), 128, 0, st>>>(k, dst, T, ux, uy, T_init);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE(R, S)                                                                        \
    template cudaError_t launch_step<R, S>(const KConst<R>&, const S*, S*, uint32_t, cudaStream_t);  \
    template cudaError_t launch_init<R, S>(const KConst<R>&, S*, const double*, const double*,      \
                                           const double*, double, cudaStream_t);

LBM_INSTANTIATE(double, double)
LBM_INSTANTIATE(float, float)
LBM_INSTANTIATE(float, __half)

}  // namespace lbm
