// lbm_adjoint.cu -- discrete adjoint of the fused step (lbm_adjoint).
//
// Loss: the mean Nusselt number on one wall after n steps (Eq. Eq:AvNuss),
// as a function of the porosity field and of the Dirichlet wall
// temperatures.  The step maps the post-collision state s_n to s_{n+1};
// node x of s_{n+1} depends on the 17 populations it pulls from its source
// node (x itself, or x_f for a wall node), on T(x_ff) for adiabatic walls,
// on the porosity at the source and at x, and on the Dirichlet T_b.  The
// adjoint runs the steps backwards:
//   k_adj_pass,   per node, the transposed Jacobian of its update applied to
//   k_adj_combine: lambda_{n+1}(x), from directional derivatives of the very
//                 same per-node code (node_update_generic) evaluated in dual
//                 numbers, giving the adjoints of the pulled values and the
//                 porosity / wall-temperature contributions.  The update
//                 depends on its 17 pulled values only through the BGK term
//                 (1 - 1/tau) in and through nine linear moment sums M in
//                 (Sec. 3.1-3.3: sum g, c g, sum f, c f, c c f), so
//                 J = diag(1 - 1/tau) + D M and J^T l = diag(1 - 1/tau) l +
//                 M^T D^T l: nine derivatives along directions d_k with
//                 M d_k = e_k give D^T l (plus up to two for the porosity
//                 and wall temperature), one thread per (node, pass);
//   k_adj_gather: the transpose of pull streaming: each stored value
//                 collects the adjoints of every node that pulled it (its
//                 downstream neighbour, the wall nodes whose x_f or x_ff it
//                 feeds), deterministically, without atomics.
// States are recomputed from checkpoints kept every ceil(sqrt(n)) steps.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lbm_handle.h"
#include "lbm_host.h"
#include "lbm_internal.h"

namespace lbm {

constexpr int kAdjBlock = 128;

template <class R>
__device__ __forceinline__ long long at_of(const KConst<R>& k, int x, int y) { return (long long)y * k.pitch + x; }

// Directions d_k in the space of the 17 pulled values (f_1..f_8, h_0..h_8)
// with M d_k = e_k for the moment sums k = 0 sum h, 1 sum_x c_x h,
// 2 sum c_y h, 3 sum f, 4 sum c_x f, 5 sum c_y f, 6 sum c_x^2 f,
// 7 sum c_y^2 f, 8 sum c_x c_y f (M: row k holds the weights of sum k).
__device__ __forceinline__ float moment_dir(int k, int q) {
    if (q >= 8) {
        const int i = q - 8;
        if (k == 0) return i == 0 ? 1.f : 0.f;
        if (k == 1) return i == 1 ? 0.5f : (i == 3 ? -0.5f : 0.f);
        if (k == 2) return i == 2 ? 0.5f : (i == 4 ? -0.5f : 0.f);
        return 0.f;
    }
    const int i = q + 1;
    const bool axis13 = i == 1 || i == 3, axis24 = i == 2 || i == 4, diag = i >= 5;
    switch (k) {
    case 3: return axis13 || axis24 ? 0.5f : -0.25f;            // sum f
    case 4: return i == 1 ? 0.5f : (i == 3 ? -0.5f : 0.f);      // sum c_x f
    case 5: return i == 2 ? 0.5f : (i == 4 ? -0.5f : 0.f);      // sum c_y f
    case 6: return axis24 ? -0.5f : (diag ? 0.25f : 0.f);       // sum c_x^2 f
    case 7: return axis13 ? -0.5f : (diag ? 0.25f : 0.f);       // sum c_y^2 f
    case 8: return diag ? ((i == 5 || i == 7) ? 0.25f : -0.25f) : 0.f;  // sum c_x c_y f
    default: return 0.f;
    }
}

// Weight of pulled value q in moment sum k (row k of M).
__device__ __forceinline__ float moment_weight(int k, int q) {
    if (q >= 8) {
        const int i = q - 8;
        return k == 0 ? 1.f : (k == 1 ? float(cx_of(i)) : (k == 2 ? float(cy_of(i)) : 0.f));
    }
    const int i = q + 1;
    const float cx = float(cx_of(i)), cy = float(cy_of(i));
    switch (k) {
    case 3: return 1.f;
    case 4: return cx;
    case 5: return cy;
    case 6: return cx * cx;
    case 7: return cy * cy;
    case 8: return cx * cy;
    default: return 0.f;
    }
}

// Passes of the local transposed Jacobian: 0..8 the moment directions d_k,
// 9 porosity at the source node, 10 porosity at the node (wall nodes only),
// 11 T(x_ff) (adiabatic walls), 12 the Dirichlet T_b.
constexpr int kAdjPasses = 13;

// One pass per thread (blockIdx.z = pass j): the directional derivative of
// node (x, y)'s update along its direction, dotted with lambda_{n+1}(x).
// D[j][x]: for j < 9 (D^T l)_j = l . J d_j - l . (diag(1 - 1/tau) d_j);
// otherwise l . (dout / d input j), 0 where the input does not exist.
template <class R, class S>
__global__ void __launch_bounds__(kAdjBlock)
k_adj_pass(const __grid_constant__ KConst<R> k, const S* __restrict__ state, const R* __restrict__ lam,
           R* __restrict__ D) {
    const int x = blockIdx.x * kAdjBlock + threadIdx.x;
    const int y = blockIdx.y;
    const int j = blockIdx.z;
    if (x >= k.nx) return;
    const long long a = at_of(k, x, y);
    const WallInfo w = classify(k, x, y);
    const bool field = k.eps_field != nullptr;
    const bool used = j < 9 || (j == 9 && field) || (j == 10 && field && w.wall) ||
                      (j == 11 && w.wall && w.tside < 0) || (j == 12 && w.wall && w.tside >= 0);
    if (!used) {
        D[j * k.plane + a] = R(0);
        return;
    }
    const int xs = w.wall ? w.xs : x, ys = w.wall ? w.ys : y;
    Pops<R> P;
    pull(k, state, xs, ys, P);
    R thff = R(0);
    if (w.wall && w.tside < 0) thff = (pull_hsum<R, R, S>(k, state, w.xff, w.yff) + R(0.5) * k.Q) * k.inv_sigma;
    const R thb = (w.wall && w.tside >= 0) ? k.T_bc[w.tside] - k.T0 : R(0);
    const R eps_s = node_eps(k, xs, ys), eps_x = node_eps(k, x, y);
    Dual<R> din[17], dout[17];
#pragma unroll
    for (int i = 1; i < 9; ++i) din[i - 1] = Dual<R>(P.f[i], j < 9 ? R(moment_dir(j, i - 1)) : R(0));
#pragma unroll
    for (int i = 0; i < 9; ++i) din[8 + i] = Dual<R>(P.h[i], j < 9 ? R(moment_dir(j, 8 + i)) : R(0));
    const Dual<R> des(eps_s, j == 9 ? R(1) : R(0));
    // an interior node's own porosity is its source porosity
    const Dual<R> dex = w.wall ? Dual<R>(eps_x, j == 10 ? R(1) : R(0)) : des;
    const Dual<R> dff(thff, j == 11 ? R(1) : R(0));
    const Dual<R> dtb(thb, j == 12 ? R(1) : R(0));
    node_update_generic(k, w, din, des, dex, dff, dtb, row_ay(k, ys), row_ay(k, y), dout);
    R acc = R(0);
#pragma unroll
    for (int q = 0; q < 17; ++q) {
        const R l = lam[q * k.plane + a];
        acc += dout[q].d * l;
        if (j < 9) acc -= (q < 8 ? k.omf : k.omT) * l * R(moment_dir(j, q));
    }
    D[j * k.plane + a] = acc;
}

// V = J^T l = diag(1 - 1/tau) l + M^T D^T l per node, the x_ff adjoint, and
// the porosity / wall-temperature gradient contributions.
template <class R>
__global__ void __launch_bounds__(kAdjBlock)
k_adj_combine(const __grid_constant__ KConst<R> k, const R* __restrict__ lam, const R* __restrict__ D,
              R* __restrict__ V, R* __restrict__ Vff, double* __restrict__ g_eps, double* __restrict__ g_epsf,
              double* __restrict__ g_tb) {
    const int x = blockIdx.x * kAdjBlock + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= k.nx) return;
    const long long a = at_of(k, x, y);
    R dtl[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) dtl[m] = D[m * k.plane + a];
#pragma unroll
    for (int q = 0; q < 17; ++q) {
        R v = (q < 8 ? k.omf : k.omT) * lam[q * k.plane + a];
#pragma unroll
        for (int m = 0; m < 9; ++m) v += R(moment_weight(m, q)) * dtl[m];
        V[q * k.plane + a] = v;
    }
    Vff[a] = D[11 * k.plane + a];
    const long long c = (long long)y * k.nx + x;
    const R v_es = D[9 * k.plane + a];
    if (!classify(k, x, y).wall) {
        g_eps[c] += double(v_es);
    } else {
        g_eps[c] += double(D[10 * k.plane + a]);
        g_epsf[c] += double(v_es);
        g_tb[c] += double(D[12 * k.plane + a]);
    }
}

// Does some wall node b satisfy (x_f or x_ff of b) == s?  Checked only near
// the walls (sources of both lie at most two nodes inside).
template <class R>
__device__ __forceinline__ bool near_wall(const KConst<R>& k, int sx, int sy) {
    return (k.bc[SW] != BC_PERIODIC && (sx <= 2 || sx >= k.nx - 3)) ||
           (k.bc[SS] != BC_PERIODIC && (sy <= 2 || sy >= k.ny - 3));
}

// Transpose of pull streaming: lambda_n(y, q) = sum of V_q over the nodes that
// pulled value (y, q) during step n -> n+1.
template <class R>
__global__ void __launch_bounds__(kAdjBlock)
k_adj_gather(const __grid_constant__ KConst<R> k, const R* __restrict__ V, const R* __restrict__ Vff,
             R* __restrict__ lam_prev) {
    const int x = blockIdx.x * kAdjBlock + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= k.nx) return;
    const bool px = k.bc[SW] == BC_PERIODIC, py = k.bc[SS] == BC_PERIODIC;
#pragma unroll 1
    for (int q = 0; q < 17; ++q) {
        const int i = q < 8 ? q + 1 : q - 8;
        int sx = x + cx_of(i), sy = y + cy_of(i);  // the node that pulls (x, y) along c_i
        R acc = R(0);
        if (px) sx = (sx + k.nx) % k.nx;
        if (py) sy = (sy + k.ny) % k.ny;
        if (sx >= 0 && sx < k.nx && sy >= 0 && sy < k.ny) {
            const WallInfo ws = classify(k, sx, sy);
            if (!ws.wall) acc += V[q * k.plane + at_of(k, sx, sy)];
            if (near_wall(k, sx, sy)) {
                for (int d = 1; d < 9; ++d) {
                    for (int m = 1; m <= 2; ++m) {
                        if (m == 2 && q < 8) continue;  // x_ff feeds only T
                        const int bx = sx - m * cx_of(d), by = sy - m * cy_of(d);
                        if (bx < 0 || bx >= k.nx || by < 0 || by >= k.ny) continue;
                        const WallInfo wb = classify(k, bx, by);
                        if (!wb.wall) continue;
                        if (m == 1 && wb.xs == sx && wb.ys == sy) acc += V[q * k.plane + at_of(k, bx, by)];
                        if (m == 2 && wb.tside < 0 && wb.xff == sx && wb.yff == sy)
                            acc += Vff[at_of(k, bx, by)] * k.inv_sigma;
                    }
                }
            }
        }
        lam_prev[q * k.plane + at_of(k, x, y)] = acc;
    }
}

// Seed: lambda_n(y, q) = dL/dT(s) / sigma for the thermal planes, where s is
// the interior node that pulls (y, q) (T = T0 + (sum h + Q/2)/sigma).
template <class R>
__global__ void k_adj_seed(const __grid_constant__ KConst<R> k, const double* __restrict__ dLdT, R* __restrict__ lam) {
    const int x = blockIdx.x * kAdjBlock + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= k.nx) return;
    const bool px = k.bc[SW] == BC_PERIODIC, py = k.bc[SS] == BC_PERIODIC;
    for (int q = 0; q < 17; ++q) {
        R v = R(0);
        if (q >= 8) {
            const int i = q - 8;
            int sx = x + cx_of(i), sy = y + cy_of(i);
            if (px) sx = (sx + k.nx) % k.nx;
            if (py) sy = (sy + k.ny) % k.ny;
            if (sx >= 0 && sx < k.nx && sy >= 0 && sy < k.ny && !classify(k, sx, sy).wall)
                v = R(dLdT[(long long)sy * k.nx + sx] * double(k.inv_sigma));
        }
        lam[q * k.plane + at_of(k, x, y)] = v;
    }
}

// D: scratch of kAdjPasses planes.
template <class R, class S>
cudaError_t launch_adj_local(const KConst<R>& k, const S* state, const R* lam, R* D, R* V, R* Vff, double* g_eps,
                             double* g_epsf, double* g_tb, cudaStream_t st) {
    const unsigned bx = (unsigned)((k.nx + kAdjBlock - 1) / kAdjBlock);
    k_adj_pass<R, S><<<dim3(bx, (unsigned)k.ny, kAdjPasses), kAdjBlock, 0, st>>>(k, state, lam, D);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adj_combine<R><<<dim3(bx, (unsigned)k.ny), kAdjBlock, 0, st>>>(k, lam, D, V, Vff, g_eps, g_epsf, g_tb);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_adj_gather(const KConst<R>& k, const R* V, const R* Vff, R* lam_prev, cudaStream_t st) {
    const dim3 grid((unsigned)((k.nx + kAdjBlock - 1) / kAdjBlock), (unsigned)k.ny);
    k_adj_gather<R><<<grid, kAdjBlock, 0, st>>>(k, V, Vff, lam_prev);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_adj_seed(const KConst<R>& k, const double* dLdT, R* lam, cudaStream_t st) {
    const dim3 grid((unsigned)((k.nx + kAdjBlock - 1) / kAdjBlock), (unsigned)k.ny);
    k_adj_seed<R><<<grid, kAdjBlock, 0, st>>>(k, dLdT, lam);
    return cudaGetLastError();
}

}  // namespace lbm

// ------------------------------------------------------------------- host

namespace {

// Host mirror of the wall classification (Sec. 3.4 readings).
struct HostWall {
    bool wall;
    int xs, ys, xff, yff, tside;
};

HostWall host_classify(const lbm_params& p, int x, int y) {
    HostWall w{};
    const bool onW = x == 0 && p.bc[0] != LBM_BC_PERIODIC;
    const bool onE = x == p.nx - 1 && p.bc[1] != LBM_BC_PERIODIC;
    const bool onS = y == 0 && p.bc[2] != LBM_BC_PERIODIC;
    const bool onN = y == p.ny - 1 && p.bc[3] != LBM_BC_PERIODIC;
    w.wall = onW || onE || onS || onN;
    const int dx = onW ? 1 : (onE ? -1 : 0), dy = onS ? 1 : (onN ? -1 : 0);
    w.xs = x + dx;
    w.ys = y + dy;
    w.xff = x + 2 * dx;
    w.yff = y + 2 * dy;
    const int xsd = onW ? 0 : (onE ? 1 : -1), ysd = onS ? 2 : (onN ? 3 : -1);
    w.tside = -1;
    if (xsd >= 0 && p.bc[xsd] == LBM_BC_DIRICHLET) w.tside = xsd;
    else if (ysd >= 0 && p.bc[ysd] == LBM_BC_DIRICHLET) w.tside = ysd;
    return w;
}

}  // namespace

namespace {

template <class R, class S>
lbm_status run_adjoint(lbm_handle* h, const lbm::KConst<R>& k, int64_t n, int64_t seg_len, int side, double* loss,
                       double* dloss_deps, double* dloss_dTbc) {
    cudaStream_t st = h->stream;
    const lbm_params& p = h->prm;
    const size_t N = (size_t)p.nx * p.ny;
    const int64_t K = seg_len > 0 ? seg_len : (int64_t)ceil(sqrt((double)n));
    const int64_t nseg = (n + K - 1) / K;
    const size_t sb = h->L.buf_bytes;                               // one state
    const size_t lam_bytes = 17 * (size_t)k.plane * sizeof(R);    // one adjoint state
    std::vector<void*> allocs;
    auto fail_free = [&](lbm_status s, const std::string& m) {
        for (void* a : allocs) cudaFreeAsync(a, st);
        cudaStreamSynchronize(st);
        return lbm_handle_fail(h, s, m);
    };
    auto alloc = [&](size_t bytes) -> void* {
        void* a = nullptr;
        if (cudaMallocAsync(&a, bytes, st) != cudaSuccess) return nullptr;
        allocs.push_back(a);
        return a;
    };
    char* ckpt = (char*)alloc(sb * (size_t)nseg);
    char* segs = (char*)alloc(sb * (size_t)K);
    R* lam0 = (R*)alloc(lam_bytes);
    R* lam1 = (R*)alloc(lam_bytes);
    R* V = (R*)alloc(lam_bytes);
    R* Vff = (R*)alloc((size_t)k.plane * sizeof(R));
    R* Dp = (R*)alloc((size_t)lbm::kAdjPasses * k.plane * sizeof(R));  // per-pass products
    double* g = (double*)alloc(4 * N * sizeof(double));  // g_eps, g_epsf, g_tb, dL/dT
    if (!ckpt || !segs || !lam0 || !lam1 || !V || !Vff || !Dp || !g)
        return fail_free(LBM_ERR_OOM, "adjoint buffers (checkpoints grow as sqrt(n))");
    double *g_eps = g, *g_epsf = g + N, *g_tb = g + 2 * N, *dLdT = g + 3 * N;
    if (cudaMemsetAsync(g, 0, 3 * N * sizeof(double), st) != cudaSuccess) return fail_free(LBM_ERR_CUDA, "memset");

    // forward, keeping a checkpoint at the start of every segment
    const int64_t step0 = h->steps;
    for (int64_t t = 0; t < n; ++t) {
        if (t % K == 0)
            if (cudaMemcpyAsync(ckpt + sb * (size_t)(t / K), h->buf(h->cur), sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return fail_free(LBM_ERR_CUDA, "checkpoint copy");
        cudaError_t e = lbm::launch_step(k, (const S*)h->buf(h->cur), (S*)h->buf(1 - h->cur), (uint32_t)(step0 + t), st);
        if (e != cudaSuccess) return fail_free(LBM_ERR_CUDA, std::string("step kernel: ") + cudaGetErrorString(e));
        h->cur = 1 - h->cur;
        ++h->steps;
        ++h->launches;
    }
    // loss
    cudaError_t e = lbm::launch_nusselt(k, h->diag, (const S*)h->buf(h->cur), side, h->nu(), h->out(), st);
    if (e != cudaSuccess) return fail_free(LBM_ERR_CUDA, "nusselt kernels");
    if (cudaMemcpyAsync(loss, h->out(), sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return fail_free(LBM_ERR_CUDA, "loss copy");

    // seed: dL/dT per node, wall nodes resolved onto interior nodes
    std::vector<double> dT(N, 0.0);
    double dTbc[4] = {0, 0, 0, 0};
    const int nw = side <= 1 ? p.ny : p.nx;
    for (int j = 0; j < nw; ++j) {
        const double wj = (j == 0 || j == nw - 1) ? 0.5 : 1.0;
        const double sgn = (side == 0 || side == 2) ? 1.0 : -1.0;  // d_axis = sgn * d_inward
        const double base = -h->d.L / h->d.dT * sgn * wj / double(nw - 1);
        const double coef[3] = {-1.5 * base, 2.0 * base, -0.5 * base};
        for (int m = 0; m < 3; ++m) {
            int x, y;
            if (side == 0) { x = m; y = j; }
            else if (side == 1) { x = p.nx - 1 - m; y = j; }
            else if (side == 2) { x = j; y = m; }
            else { x = j; y = p.ny - 1 - m; }
            const HostWall w = host_classify(p, x, y);
            if (!w.wall) dT[(size_t)y * p.nx + x] += coef[m];
            else if (w.tside >= 0) dTbc[w.tside] += coef[m];
            else {
                dT[(size_t)w.ys * p.nx + w.xs] += coef[m] * 4.0 / 3.0;
                dT[(size_t)w.yff * p.nx + w.xff] -= coef[m] / 3.0;
            }
        }
    }
    if (cudaMemcpyAsync(dLdT, dT.data(), N * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail_free(LBM_ERR_CUDA, "seed copy");
    e = lbm::launch_adj_seed(k, dLdT, lam0, st);
    if (e != cudaSuccess) return fail_free(LBM_ERR_CUDA, "seed kernel");
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail_free(LBM_ERR_CUDA, "seed");  // dT reused below

    // backward over the segments, recomputing each from its checkpoint
    R* lc = lam0;
    R* ln = lam1;
    for (int64_t sgi = nseg - 1; sgi >= 0; --sgi) {
        const int64_t t0 = sgi * K, len = std::min<int64_t>(K, n - t0);
        if (cudaMemcpyAsync(segs, ckpt + sb * (size_t)sgi, sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return fail_free(LBM_ERR_CUDA, "checkpoint restore");
        for (int64_t t = 1; t < len; ++t) {
            e = lbm::launch_step(k, (const S*)(segs + sb * (size_t)(t - 1)), (S*)(segs + sb * (size_t)t),
                                 (uint32_t)(step0 + t0 + t - 1), st);
            if (e != cudaSuccess) return fail_free(LBM_ERR_CUDA, "recompute step");
        }
        for (int64_t t = len - 1; t >= 0; --t) {
            e = lbm::launch_adj_local(k, (const S*)(segs + sb * (size_t)t), lc, Dp, V, Vff, g_eps, g_epsf, g_tb, st);
            if (e == cudaSuccess) e = lbm::launch_adj_gather(k, V, Vff, ln, st);
            if (e != cudaSuccess) return fail_free(LBM_ERR_CUDA, std::string("adjoint kernels: ") + cudaGetErrorString(e));
            std::swap(lc, ln);
        }
    }
    // gradients
    std::vector<double> hg(3 * N);
    if (cudaMemcpyAsync(hg.data(), g, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail_free(LBM_ERR_CUDA, "gradient copy");
    std::vector<double> ge(hg.begin(), hg.begin() + N);
    for (int y = 0; y < p.ny; ++y)
        for (int x = 0; x < p.nx; ++x) {
            const HostWall w = host_classify(p, x, y);
            if (!w.wall) continue;
            const size_t c = (size_t)y * p.nx + x;
            ge[(size_t)w.ys * p.nx + w.xs] += hg[N + c];
            if (w.tside >= 0) dTbc[w.tside] += hg[2 * N + c];
        }
    if (dloss_deps) memcpy(dloss_deps, ge.data(), N * sizeof(double));
    if (dloss_dTbc) memcpy(dloss_dTbc, dTbc, sizeof(dTbc));
    for (void* a : allocs) cudaFreeAsync(a, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return lbm_handle_fail(h, LBM_ERR_CUDA, "adjoint cleanup");
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_adjoint(lbm_handle* h, int64_t n_steps, int64_t segment, int side, double* loss,
                                  double* dloss_deps, double* dloss_dTbc) {
    const lbm_host::NvtxRange range("lbm_adjoint");
    if (!h) return LBM_ERR_ARG;
    if (n_steps < 1 || segment < 0 || side < 0 || side > 3 || !loss)
        return lbm_handle_fail(h, LBM_ERR_ARG, "bad step count, segment, side or null loss");
    if (h->prm.precision == LBM_F16)
        return lbm_handle_fail(h, LBM_ERR_ARG, "the adjoint runs on FP64 or FP32 storage");
    if (h->moments_kind())
        return lbm_handle_fail(h, LBM_ERR_ARG, "the adjoint runs on population storage, not on a moment state");
    if (h->nonfinite) return lbm_handle_fail(h, LBM_ERR_NONFINITE, "non-finite velocity or temperature");
    const bool field = h->prm.precision == LBM_F64 ? h->k64.eps_field != nullptr : h->k32.eps_field != nullptr;
    if (dloss_deps && !field)
        return lbm_handle_fail(h, LBM_ERR_ARG, "a porosity gradient needs a porosity field (lbm_set_fields)");
    if ((side <= 1 ? h->prm.nx : h->prm.ny) < 3)
        return lbm_handle_fail(h, LBM_ERR_ARG, "the one-sided difference needs 3 nodes");
    if (h->prm.precision == LBM_F64)
        return run_adjoint<double, double>(h, h->k64, n_steps, segment, side, loss, dloss_deps, dloss_dTbc);
    return run_adjoint<float, float>(h, h->k32, n_steps, segment, side, loss, dloss_deps, dloss_dTbc);
}
