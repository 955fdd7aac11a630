// lbm_diag.cu -- kernels off the step's hot path: initial and stored state
// conversion, moments, Nusselt numbers, residual, totals, stream function.
// Reductions are deterministic (fixed-order block sums in FP64).
#include <math.h>

#include "lbm_diag.cuh"

namespace lbm {

// Residual and totals: a grid of at most kResGrid blocks strides over the
// nodes in a fixed order (deterministic; one node per thread up to 16.7 M
// nodes).  FP64 arithmetic is slow on this GPU, so the per-node work and the
// warp sums of the residual run in the lattice's arithmetic and only the
// per-warp results are added in FP64.
constexpr int kResBlock = 256;
constexpr int kResGrid = 65536;

// Block sum of one value per thread: warp sums in R, then the warps' sums
// in FP64 in a fixed order (valid in thread 0).
template <class R>
__device__ __forceinline__ double block_sum_r(R v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = double(v);
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;
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

__global__ void k_nusselt_mean(const double* __restrict__ nu, int n, double* __restrict__ out) {
    __shared__ double sh[kReduceBlock / 32];
    double acc = 0.0;
    for (int j = threadIdx.x; j < n; j += kReduceBlock) acc += ((j == 0 || j == n - 1) ? 0.5 : 1.0) * nu[j];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] = s / double(n - 1);
}

// Per-node terms in the lattice's arithmetic R (the snapshot holds values
// of type R, so the differences are exact up to one rounding); per-thread
// sums in R over the thread's nodes, block and grid sums in FP64.
template <class R, class S>
__global__ void __launch_bounds__(kResBlock)
k_residual(const __grid_constant__ KConst<R> k, const S* __restrict__ src, double* __restrict__ snap,
           double* __restrict__ partial) {
    __shared__ double sh[kResBlock / 32];
    const long long N = (long long)k.nx * k.ny;
    // the snapshot holds values of type R (FP64 conversions are slow here)
    R* sn = reinterpret_cast<R*>(snap);
    R v[4] = {R(0), R(0), R(0), R(0)};
    for (long long c = (long long)blockIdx.x * kResBlock + threadIdx.x; c < N; c += (long long)gridDim.x * kResBlock) {
        const int y = (int)((unsigned long long)c / (unsigned)k.nx), x = (int)(c - (long long)y * k.nx);
        // snapshot loads first: they do not depend on the node's moments
        const R s0 = sn[c], s1 = sn[N + c], s2 = sn[2 * N + c];
        R ux, uy, th;
        node_u_th(k, src, x, y, &ux, &uy, &th);
        const R T = k.T0 + th;
        const R dx = ux - s0, dy = uy - s1, dT = T - s2;
        v[0] += sqrt(dx * dx + dy * dy);
        v[1] += sqrt(ux * ux + uy * uy);
        v[2] += fabs(dT);
        v[3] += fabs(T);
        sn[c] = ux;
        sn[N + c] = uy;
        sn[2 * N + c] = T;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const double s = block_sum_r(v[m], sh);
        if (threadIdx.x == 0) partial[4 * blockIdx.x + m] = s;
    }
}

// Per-block sums of sum_{i=1..8} f_i and sum_i g_i over the stored state.
// Per node: the sums of its populations in R; per thread and above: FP64.
template <class R, class S>
__global__ void __launch_bounds__(kResBlock)
k_totals(const __grid_constant__ KConst<R> k, const S* __restrict__ src, double sT0, double* __restrict__ partial) {
    __shared__ double sh[kResBlock / 32];
    const long long N = (long long)k.nx * k.ny;
    double sf = 0.0, sg = 0.0;
    for (long long c = (long long)blockIdx.x * kResBlock + threadIdx.x; c < N; c += (long long)gridDim.x * kResBlock) {
        const int y = (int)(c / k.nx), x = (int)(c - (long long)y * k.nx);
        const long long at = (long long)y * k.pitch + x;
        R nf = R(0), ng = R(0);
        for (int i = 1; i < 9; ++i) nf += load_pop<S, R>(src + (long long)(i - 1) * k.plane + at, k.scale);
        for (int i = 0; i < 9; ++i) ng += load_pop<S, R>(src + (long long)(8 + i) * k.plane + at, k.scale);
        sf += double(nf);
        sg += double(ng) + sT0;  // sum_i w_i sigma T0 of the stored deviations
    }
    const double a = block_sum(sf, sh);
    if (threadIdx.x == 0) partial[4 * blockIdx.x + 0] = a;
    const double b = block_sum(sg, sh);
    if (threadIdx.x == 0) {
        partial[4 * blockIdx.x + 1] = b;
        partial[4 * blockIdx.x + 2] = 0.0;
        partial[4 * blockIdx.x + 3] = 0.0;
    }
}

constexpr int kReduce4Block = 1024;

__global__ void __launch_bounds__(kReduce4Block) k_reduce4(const double* __restrict__ partial, long long nb,
                                                          double* __restrict__ out) {
    __shared__ double sh[kReduce4Block / 32];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long b = threadIdx.x; b < nb; b += kReduce4Block)
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

cudaError_t launch_stream_function(const double* ux, int nx, int ny, double* psi, double* range,
                                   cudaStream_t st) {
    k_stream_function<<<(nx + 127) / 128, 128, 0, st>>>(ux, nx, ny, psi);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_minmax<<<1, kReduceBlock, 0, st>>>(psi, (long long)nx * ny, range);
    return cudaGetLastError();
}

long long residual_blocks(int nx, int ny) {
    const long long b = ((long long)nx * ny + kResBlock - 1) / kResBlock;
    return b < kResGrid ? b : kResGrid;
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
    k_residual<R, S><<<(unsigned)residual_blocks(k.nx, k.ny), kResBlock, 0, st>>>(k, src, snap, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce4<<<1, kReduce4Block, 0, st>>>(partial, residual_blocks(k.nx, k.ny), out);
    return cudaGetLastError();
}

template <class R, class S>
cudaError_t launch_totals(const KConst<R>& k, const S* src, double sT0, double* partial, double* out,
                          cudaStream_t st) {
    k_totals<R, S><<<(unsigned)residual_blocks(k.nx, k.ny), kResBlock, 0, st>>>(k, src, sT0, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce4<<<1, kReduce4Block, 0, st>>>(partial, residual_blocks(k.nx, k.ny), out);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE_DIAG(R, S)                                                                        \
    template cudaError_t launch_totals<R, S>(const KConst<R>&, const S*, double, double*, double*,  \
                                             cudaStream_t);                                         \
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

LBM_INSTANTIATE_DIAG(double, double)
LBM_INSTANTIATE_DIAG(float, float)
LBM_INSTANTIATE_DIAG(float, __half)

}  // namespace lbm
