// lbm_batch_kernels.cu -- the global-load batched step kernel and the
// batch's Nusselt kernel (many cavities, one launch per step).  FP32 batches
// of walled cavities run the staged kernel of lbm_step_tma.cu instead.
#include <math.h>

#include "lbm_step.cuh"

namespace lbm {

// ------------------------------------------------------------------ batches

// Resident blocks per SM of the batched step.  Small cavities have many wall
// nodes; the batched kernel runs better with a little more register room for
// their out-of-line path (6 x 128 threads).
#ifndef LBM_BATCH_BLOCKS
#define LBM_BATCH_BLOCKS 6
#endif
template <class R> struct BatchOccupancy { static constexpr int blocks = LBM_BATCH_BLOCKS; };
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
// constants in shared memory; every node runs the same interior / wall
// code as k_step.  Interior tiles and packed wall nodes are separate items,
// so the out-of-line wall path never stalls a warp of interior nodes.
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
