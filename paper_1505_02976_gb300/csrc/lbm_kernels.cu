// lbm_kernels.cu -- the fused step kernel and the small auxiliary kernels.
//
// k_step: one thread per node, pull streaming from the ping buffer, all the
// per-node arithmetic of the step in registers, and one write of the 17
// post-collision planes to the pong buffer.  Wall nodes take the NEES rebuild
// inside the same launch (an out-of-line path that pulls the populations of
// the wall node's fluid neighbour x_f instead of its own).
#include <math.h>

#include "lbm_internal.h"

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

template <class R, class S>
__global__ void k_moments(const __grid_constant__ KConst<R> k, const S* __restrict__ src,
                          double* __restrict__ p, double* __restrict__ ux, double* __restrict__ uy,
                          double* __restrict__ T) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= k.nx) return;
    const State<R> s = node_state_at(k, src, x, y);
    const long long c = (long long)y * k.nx + x;
    p[c] = double(s.p);
    ux[c] = double(s.ux);
    uy[c] = double(s.uy);
    T[c] = double(k.T0) + double(s.th);
}

template <class R, class S>
__global__ void k_get_state(const __grid_constant__ KConst<R> k, const S* __restrict__ src,
                            double* __restrict__ f, double* __restrict__ g, double sT0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= k.nx) return;
    const long long at = (long long)y * k.pitch + x;
    const long long c = (long long)y * k.nx + x;
    const long long N = (long long)k.nx * k.ny;
    f[c] = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
    for (int i = 1; i < 9; ++i) f[i * N + c] = double(load_pop<S, R>(src + (long long)(i - 1) * k.plane + at, k.scale));
#pragma unroll
    for (int i = 0; i < 9; ++i)
        g[i * N + c] = double(load_pop<S, R>(src + (long long)(8 + i) * k.plane + at, k.scale)) + w_of<double>(i) * sT0;
}

template <class R, class S>
__global__ void k_set_state(const __grid_constant__ KConst<R> k, S* __restrict__ dst,
                            const double* __restrict__ f, const double* __restrict__ g, double sT0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= k.nx) return;
    const long long at = (long long)y * k.pitch + x;
    const long long c = (long long)y * k.nx + x;
    const long long N = (long long)k.nx * k.ny;
#pragma unroll
    for (int i = 1; i < 9; ++i) store_pop<S, R>(dst + (long long)(i - 1) * k.plane + at, R(f[i * N + c]), k.scale);
#pragma unroll
    for (int i = 0; i < 9; ++i)
        store_pop<S, R>(dst + (long long)(8 + i) * k.plane + at, R(g[i * N + c] - w_of<double>(i) * sT0), k.scale);
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

template <class R, class S>
__global__ void k_nusselt_local(const __grid_constant__ KConst<R> k, const DiagConst d,
                                const S* __restrict__ src, int side, double* __restrict__ nu) {
    const int n = side <= SE ? k.ny : k.nx;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double t[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        int x, y;
        if (side == SW) { x = m; y = j; }
        else if (side == SE) { x = k.nx - 1 - m; y = j; }
        else if (side == SS) { x = j; y = m; }
        else { x = j; y = k.ny - 1 - m; }
        t[m] = node_T(k, d, src, x, y);
    }
    // derivative from the wall inward, then along +x (W, E) or +y (S, N)
    const double d_in = (-3.0 * t[0] + 4.0 * t[1] - t[2]) * 0.5;
    const double d_axis = (side == SW || side == SS) ? d_in : -d_in;
    nu[j] = -d.L * d_axis / d.dT;
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

__global__ void k_nusselt_mean(const double* __restrict__ nu, int n, double* __restrict__ out) {
    __shared__ double sh[kReduceBlock / 32];
    double acc = 0.0;
    for (int j = threadIdx.x; j < n; j += kReduceBlock) acc += ((j == 0 || j == n - 1) ? 0.5 : 1.0) * nu[j];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] = s / double(n - 1);
}

constexpr int kResBlock = 128;

template <class R, class S>
__global__ void __launch_bounds__(kResBlock)
k_residual(const __grid_constant__ KConst<R> k, const S* __restrict__ src, double* __restrict__ snap,
           double* __restrict__ partial) {
    __shared__ double sh[kResBlock / 32];
    const int x = blockIdx.x * kResBlock + threadIdx.x;
    const int y = blockIdx.y;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (x < k.nx) {
        const State<R> s = node_state_at(k, src, x, y);
        const long long N = (long long)k.nx * k.ny;
        const long long c = (long long)y * k.nx + x;
        const double ux = double(s.ux), uy = double(s.uy), T = double(k.T0) + double(s.th);
        const double dx = ux - snap[c], dy = uy - snap[N + c], dT = T - snap[2 * N + c];
        v[0] = sqrt(dx * dx + dy * dy);
        v[1] = sqrt(ux * ux + uy * uy);
        v[2] = fabs(dT);
        v[3] = fabs(T);
        snap[c] = ux;
        snap[N + c] = uy;
        snap[2 * N + c] = T;
    }
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const double s = block_sum(v[m], sh);
        if (threadIdx.x == 0) partial[4 * b + m] = s;
    }
}

// Per-block sums of sum_{i=1..8} f_i and sum_i g_i over the stored state.
template <class R, class S>
__global__ void __launch_bounds__(kResBlock)
k_totals(const __grid_constant__ KConst<R> k, const S* __restrict__ src, double sT0, double* __restrict__ partial) {
    __shared__ double sh[kResBlock / 32];
    const int x = blockIdx.x * kResBlock + threadIdx.x;
    const int y = blockIdx.y;
    double sf = 0.0, sg = 0.0;
    if (x < k.nx) {
        const long long at = (long long)y * k.pitch + x;
        for (int i = 1; i < 9; ++i) sf += double(load_pop<S, R>(src + (long long)(i - 1) * k.plane + at, k.scale));
        for (int i = 0; i < 9; ++i) sg += double(load_pop<S, R>(src + (long long)(8 + i) * k.plane + at, k.scale));
        sg += sT0;  // sum_i w_i sigma T0
    }
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    const double a = block_sum(sf, sh);
    if (threadIdx.x == 0) partial[4 * b + 0] = a;
    const double c = block_sum(sg, sh);
    if (threadIdx.x == 0) {
        partial[4 * b + 1] = c;
        partial[4 * b + 2] = 0.0;
        partial[4 * b + 3] = 0.0;
    }
}

__global__ void k_reduce4(const double* __restrict__ partial, long long nb, double* __restrict__ out) {
    __shared__ double sh[kReduceBlock / 32];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long b = threadIdx.x; b < nb; b += kReduceBlock)
#pragma unroll
        for (int m = 0; m < 4; ++m) a[m] += partial[4 * b + m];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const double s = block_sum(a[m], sh);
        if (threadIdx.x == 0) out[m] = s;
    }
}

// Stream function up each column x: psi(x, 0) = 0 and
// psi(x, y) = psi(x, y - 1) + (u_x(x, y - 1) + u_x(x, y)) / 2, the trapezoid
// rule for u_x = d psi / dy.  One thread per column; rows are coalesced.
__global__ void k_stream_function(const double* __restrict__ ux, int nx, int ny, double* __restrict__ psi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    double s = 0.0;
    psi[x] = 0.0;
    for (int y = 1; y < ny; ++y) {
        s = s + 0.5 * (ux[(long long)(y - 1) * nx + x] + ux[(long long)y * nx + x]);
        psi[(long long)y * nx + x] = s;
    }
}

// out[0] = min, out[1] = max of v[0 .. n-1] (one block; order-independent).
__global__ void k_minmax(const double* __restrict__ v, long long n, double* __restrict__ out) {
    __shared__ double lo_s[kReduceBlock / 32], hi_s[kReduceBlock / 32];
    double lo = INFINITY, hi = -INFINITY;
    for (long long i = threadIdx.x; i < n; i += kReduceBlock) {
        lo = fmin(lo, v[i]);
        hi = fmax(hi, v[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        lo_s[wid] = lo;
        hi_s[wid] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kReduceBlock / 32; ++i) {
            lo = fmin(lo, lo_s[i]);
            hi = fmax(hi, hi_s[i]);
        }
        out[0] = lo;
        out[1] = hi;
    }
}

template <class R>
__global__ void k_convert(const double* __restrict__ in, R* __restrict__ out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = R(in[i]);
}

// ------------------------------------------------------------------ launchers

template <class R>
cudaError_t launch_convert(const double* in, R* out, long long n, cudaStream_t st) {
    k_convert<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}
template cudaError_t launch_convert<double>(const double*, double*, long long, cudaStream_t);
template cudaError_t launch_convert<float>(const double*, float*, long long, cudaStream_t);

static dim3 row_grid(int nx, int ny, int bx) { return dim3((unsigned)((nx + bx - 1) / bx), (unsigned)ny); }

cudaError_t launch_stream_function(const double* ux, int nx, int ny, double* psi, double* range,
                                   cudaStream_t st) {
    k_stream_function<<<(nx + 127) / 128, 128, 0, st>>>(ux, nx, ny, psi);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_minmax<<<1, kReduceBlock, 0, st>>>(psi, (long long)nx * ny, range);
    return cudaGetLastError();
}

long long residual_blocks(int nx, int ny) {
    return (long long)((nx + kResBlock - 1) / kResBlock) * ny;
}

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

template <class R, class S>
cudaError_t launch_moments(const KConst<R>& k, const S* src, double* p, double* ux, double* uy,
                           double* T, cudaStream_t st) {
    k_moments<R, S><<<row_grid(k.nx, k.ny, 128), 128, 0, st>>>(k, src, p, ux, uy, T);
    return cudaGetLastError();
}

template <class R, class S>
cudaError_t launch_get_state(const KConst<R>& k, const S* src, double* f, double* g, double sT0,
                             cudaStream_t st) {
    k_get_state<R, S><<<row_grid(k.nx, k.ny, 128), 128, 0, st>>>(k, src, f, g, sT0);
    return cudaGetLastError();
}

template <class R, class S>
cudaError_t launch_set_state(const KConst<R>& k, S* dst, const double* f, const double* g,
                             double sT0, cudaStream_t st) {
    k_set_state<R, S><<<row_grid(k.nx, k.ny, 128), 128, 0, st>>>(k, dst, f, g, sT0);
    return cudaGetLastError();
}

template <class R, class S>
cudaError_t launch_nusselt(const KConst<R>& k, const DiagConst& d, const S* src, int side,
                           double* nu_local, double* out, cudaStream_t st) {
    const int n = side <= SE ? k.ny : k.nx;
    k_nusselt_local<R, S><<<(n + 127) / 128, 128, 0, st>>>(k, d, src, side, nu_local);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_nusselt_mean<<<1, kReduceBlock, 0, st>>>(nu_local, n, out);
    return cudaGetLastError();
}

template <class R, class S>
cudaError_t launch_residual(const KConst<R>& k, const S* src, double* snap, double* partial,
                            double* out, cudaStream_t st) {
    k_residual<R, S><<<row_grid(k.nx, k.ny, kResBlock), kResBlock, 0, st>>>(k, src, snap, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce4<<<1, kReduceBlock, 0, st>>>(partial, residual_blocks(k.nx, k.ny), out);
    return cudaGetLastError();
}

template <class R, class S>
cudaError_t launch_totals(const KConst<R>& k, const S* src, double sT0, double* partial, double* out,
                          cudaStream_t st) {
    k_totals<R, S><<<row_grid(k.nx, k.ny, kResBlock), kResBlock, 0, st>>>(k, src, sT0, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce4<<<1, kReduceBlock, 0, st>>>(partial, residual_blocks(k.nx, k.ny), out);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE(R, S)                                                                        \
    template cudaError_t launch_totals<R, S>(const KConst<R>&, const S*, double, double*, double*,  \
                                             cudaStream_t);                                         \
    template cudaError_t launch_step<R, S>(const KConst<R>&, const S*, S*, uint32_t, cudaStream_t);           \
    template cudaError_t launch_init<R, S>(const KConst<R>&, S*, const double*, const double*,      \
                                           const double*, double, cudaStream_t);                    \
    template cudaError_t launch_moments<R, S>(const KConst<R>&, const S*, double*, double*, double*, \
                                              double*, cudaStream_t);                               \
    template cudaError_t launch_get_state<R, S>(const KConst<R>&, const S*, double*, double*,       \
                                                double, cudaStream_t);                              \
    template cudaError_t launch_set_state<R, S>(const KConst<R>&, S*, const double*, const double*, \
                                                double, cudaStream_t);                              \
    template cudaError_t launch_nusselt<R, S>(const KConst<R>&, const DiagConst&, const S*, int,    \
                                              double*, double*, cudaStream_t);                      \
    template cudaError_t launch_residual<R, S>(const KConst<R>&, const S*, double*, double*,        \
                                               double*, cudaStream_t);

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
