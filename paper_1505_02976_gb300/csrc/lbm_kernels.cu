// lbm_kernels.cu -- the fused step kernel (single lattice and batches).
//
// k_step: one thread per node, pull streaming from the ping buffer, all the
// per-node arithmetic of the step in registers, and one write of the 17
// post-collision planes to the pong buffer.  Wall nodes take the NEES rebuild
// inside the same launch (an out-of-line path that pulls the populations of
// the wall node's fluid neighbour x_f instead of its own).
#include <math.h>

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


// The fused step: one thread per node; interior nodes take the fast path,
// wall nodes the NEES path.
template <class R, class S, bool EPS_FIELD>
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
        interior_update(kc, src, dst, x, y, step);
    } else {
        interior_update(k, src, dst, x, y, step);
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
    if (k.eps_field) return cudaLaunchKernelEx(&cfg, k_step<R, S, true>, k, src, dst, step);
    return cudaLaunchKernelEx(&cfg, k_step<R, S, false>, k, src, dst, step);
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

// ------------------------------------------------------------------ batches

// Batched step: a grid of resident blocks walks a work list of tiles drawn
// from many cavities of different size and parameters.  Each block takes one
// contiguous chunk of the list (items are sorted by cavity, so a block
// changes cavity rarely) and stages the current cavity's constants in shared
// memory; every node then runs the same interior / wall code as k_step.
// Small cavities have many wall nodes; the batched kernel runs better with a
// little more register room for their out-of-line path (6 x 128 threads).
template <class R> struct BatchOccupancy { static constexpr int blocks = 6; };
template <> struct BatchOccupancy<double> { static constexpr int blocks = 3; };

// Wall node idx of a cavity in perimeter order: S row, N row, W column, E
// column (walled sides only; the columns skip the rows' corner nodes).
template <class R>
__device__ __forceinline__ void perimeter_node(const KConst<R>& k, int idx, int& x, int& y) {
    const bool wS = k.bc[SS] != BC_PERIODIC, wN = k.bc[SN] != BC_PERIODIC;
    const int nS = wS ? k.nx : 0, nN = wN ? k.nx : 0;
    const int y0 = wS ? 1 : 0, y1 = wN ? k.ny - 1 : k.ny;
    const int nW = k.bc[SW] != BC_PERIODIC ? y1 - y0 : 0;
    if (idx < nS) { x = idx; y = 0; return; }
    idx -= nS;
    if (idx < nN) { x = idx; y = k.ny - 1; return; }
    idx -= nN;
    if (idx < nW) { x = 0; y = y0 + idx; return; }
    idx -= nW;
    x = k.nx - 1;
    y = y0 + idx;
}

// Batched step: a grid of resident blocks walks a work list drawn from many
// cavities of different size and parameters.  Each block takes one
// contiguous, cost-balanced range of the list (items are sorted by cavity,
// so a block changes cavity rarely) and stages the current cavity's
// constants in shared memory.  Interior tiles and packed wall nodes are
// separate items, so the out-of-line wall path never stalls a warp of
// interior nodes.
template <class R, class S, int TX>
__global__ void __launch_bounds__(kStepBlock, BatchOccupancy<R>::blocks)
k_step_batch(const BatchCavity<R>* __restrict__ cav, const BatchItem* __restrict__ items,
             const int* __restrict__ bounds, const S* __restrict__ src, S* __restrict__ dst, uint32_t step) {
    __shared__ KConst<R> ks;
    __shared__ long long off;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int begin = bounds[blockIdx.x];
    const int end = bounds[blockIdx.x + 1];
    int cur = -1;
    for (int it = begin; it < end; ++it) {
        const BatchItem w = items[it];
        if (w.cavity != cur) {
            __syncthreads();
            const int* from = reinterpret_cast<const int*>(&cav[w.cavity].k);
            int* to = reinterpret_cast<int*>(&ks);
            for (int q = threadIdx.x; q < (int)(sizeof(KConst<R>) / sizeof(int)); q += kStepBlock) to[q] = from[q];
            if (threadIdx.x == 0) off = cav[w.cavity].offset;
            __syncthreads();
            cur = w.cavity;
        }
        const S* s = src + off;
        S* d = dst + off;
        if (w.kind == 0) {
            const int x = w.a + tx, y = w.b + ty;
            if (x < ks.nx && y < ks.ny && !is_wall(ks, x, y)) interior_update(ks, s, d, x, y, step);
        } else if ((int)threadIdx.x < w.b) {
            int x, y;
            perimeter_node(ks, w.a + (int)threadIdx.x, x, y);
            wall_update(ks, s, d, x, y, step);
        }
    }
}

template <class R, class S>
__global__ void k_nusselt_batch(const BatchCavity<R>* __restrict__ cav, const S* __restrict__ src,
                                int side, double* __restrict__ out) {
    __shared__ double sh[kReduceBlock / 32];
    const BatchCavity<R>& c = cav[blockIdx.x];
    const KConst<R>& k = c.k;
    const S* s = src + c.offset;
    const int n = side <= SE ? k.ny : k.nx;
    double acc = 0.0;
    for (int j = threadIdx.x; j < n; j += kReduceBlock) {
        double t[3];
        for (int m = 0; m < 3; ++m) {
            int x, y;
            if (side == SW) { x = m; y = j; }
            else if (side == SE) { x = k.nx - 1 - m; y = j; }
            else if (side == SS) { x = j; y = m; }
            else { x = j; y = k.ny - 1 - m; }
            t[m] = node_T(k, c.d, s, x, y);
        }
        const double d_in = (-3.0 * t[0] + 4.0 * t[1] - t[2]) * 0.5;
        const double d_axis = (side == SW || side == SS) ? d_in : -d_in;
        acc += ((j == 0 || j == n - 1) ? 0.5 : 1.0) * (-c.d.L * d_axis / c.d.dT);
    }
    const double total = block_sum(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = total / double(n - 1);
}

template <class R, class S>
cudaError_t launch_step_batch(const BatchCavity<R>* cav, const BatchItem* items, const int* bounds, int tile_x,
                              int grid, const S* src, S* dst, uint32_t step, cudaStream_t st) {
    if (grid < 1) return cudaErrorInvalidValue;
    switch (tile_x) {
    case 32: k_step_batch<R, S, 32><<<grid, kStepBlock, 0, st>>>(cav, items, bounds, src, dst, step); break;
    case 64: k_step_batch<R, S, 64><<<grid, kStepBlock, 0, st>>>(cav, items, bounds, src, dst, step); break;
    case 128: k_step_batch<R, S, 128><<<grid, kStepBlock, 0, st>>>(cav, items, bounds, src, dst, step); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class R, class S>
cudaError_t launch_nusselt_batch(const BatchCavity<R>* cav, int n, const S* src, int side, double* out,
                                 cudaStream_t st) {
    k_nusselt_batch<R, S><<<n, kReduceBlock, 0, st>>>(cav, src, side, out);
    return cudaGetLastError();
}

template <class R, class S>
int batch_blocks_per_sm(int tile_x) {
    int b = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (tile_x == 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step_batch<R, S, 32>, kStepBlock, 0);
    if (tile_x == 64) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step_batch<R, S, 64>, kStepBlock, 0);
    if (tile_x == 128) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step_batch<R, S, 128>, kStepBlock, 0);
    return e == cudaSuccess ? b : 0;
}

#define LBM_INSTANTIATE_BATCH(R, S)                                                                  \
    template cudaError_t launch_step_batch<R, S>(const BatchCavity<R>*, const BatchItem*, const int*, \
                                                 int, int, const S*, S*, uint32_t, cudaStream_t);    \
    template cudaError_t launch_nusselt_batch<R, S>(const BatchCavity<R>*, int, const S*, int,      \
                                                    double*, cudaStream_t);                         \
    template int batch_blocks_per_sm<R, S>(int);

LBM_INSTANTIATE_BATCH(double, double)
LBM_INSTANTIATE_BATCH(float, float)

}  // namespace lbm
