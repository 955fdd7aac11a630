// lbm_moment.cu -- the step at tau_f = tau_T = 1 on a moment state.
//
// At unit relaxation times the BGK collision discards the non-equilibrium
// part: f* = f^eq + F_i and g* = g^eq + P_i + Q_i (Eqs. LBEeq, TEqColli),
// so the post-collision populations of a node are a function of nine
// numbers, (p, u, S, T, grad T), the very state the step computes after
// streaming (Sec. 3.1-3.3).  A wall node at tau = 1 is the same function of
// its boundary state (p(x_f), u_b, S(x_f), T_b, grad T_b) of Sec. 3.4: the
// extrapolated non-equilibrium part is multiplied by 1 - 1/tau = 0.
//
// The lattice therefore stores those nine moments (36 bytes per node in
// FP32 instead of 68) and each step
//   1. expands the moments of every node (and a one-node halo) into its
//      17 post-collision populations, in shared memory,
//   2. pulls the 17 populations of each node from its neighbours there,
//   3. computes the new moments (fast_moments), and the boundary state of the
//      wall nodes from their x_f, x_ff neighbours, and stores them.
// A block owns a band of up to 126 columns and a segment of rows; it marches
// up its rows keeping the expansions of three rows in a shared ring, so every
// node is expanded once per band it borders (2 halo columns per band, 2 halo
// rows per segment).
#include <math.h>

#include "lbm_internal.h"

namespace lbm {

constexpr int kMBlock = 128;           // threads = expansion columns of a band
constexpr int kMBand = kMBlock - 2;    // output columns of a band, at most
// Expanded rows kept in shared memory: rows y - 1, y, y + 1 while row y is
// updated, and a barrier after the update frees the slot of row y - 1.  (A
// fourth slot would save that barrier but costs two resident blocks per SM,
// which measured slower.)
constexpr int kMRing = 3;
constexpr int kMaxDevices = 64;
template <class R> struct MomentOccupancy { static constexpr int blocks = 8; };
template <> struct MomentOccupancy<double> { static constexpr int blocks = 2; };

// State of a node from its stored moments; F is recomputed from (u, T) as in
// fast_moments (and, for a wall node, as in wall_state).
template <class R>
__device__ __forceinline__ FastState<R> state_from_moments(const KConst<R>& k, const R* m, int y) {
    FastState<R> s;
    s.p = m[MP];
    s.ux = m[MUX];
    s.uy = m[MUY];
    s.Sxx = m[MSXX];
    s.Syy = m[MSYY];
    s.Sxy = m[MSXY];
    s.th = m[MTH];
    s.gx = m[MGX];
    s.gy = m[MGY];
    s.T = k.T0 + s.th;
    s.uu = s.ux * s.ux + s.uy * s.uy;
    const R drag = k.e_nuK + k.e_FK * sqrt(s.uu);
    const R Gy = k.gbeta * s.th + row_ay(k, y);
    s.Fx = k.eps * k.ax - drag * s.ux;
    s.Fy = k.eps * Gy - drag * s.uy;
    s.uF = s.ux * s.Fx + s.uy * s.Fy;
    s.ep = k.eps * s.p;
    return s;
}

// Plane strides are 32-bit (9 planes of ny * pitch < 2^31 elements).
template <class R>
__device__ __forceinline__ void store_moments(const KConst<R>& k, R* dst, long long at, const FastState<R>& s) {
    R* d = dst + at;
    const int pl = k.plane32;
    d[MP * pl] = s.p;
    d[MUX * pl] = s.ux;
    d[MUY * pl] = s.uy;
    d[MSXX * pl] = s.Sxx;
    d[MSYY * pl] = s.Syy;
    d[MSXY * pl] = s.Sxy;
    d[MTH * pl] = s.th;
    d[MGX * pl] = s.gx;
    d[MGY * pl] = s.gy;
}

// Boundary state of wall node (x, y) from the new moments of x_f and the new
// temperature of x_ff (read back from dst, written earlier in this launch by
// this block), Sec. 3.4 as in wall_state.
template <class R>
__device__ __forceinline__ void wall_moments(const KConst<R>& k, R* dst, int x, int y) {
    const WallInfo w = classify(k, x, y);
    const long long af = (long long)w.ys * k.pitch + w.xs;
    R m[kMPlanes];
#pragma unroll
    for (int q = 0; q < kMPlanes; ++q) m[q] = dst[q * k.plane + af];
    m[MUX] = k.u_bc[w.uside][0];
    m[MUY] = k.u_bc[w.uside][1];
    if (w.tside >= 0) {
        m[MTH] = k.T_bc[w.tside] - k.T0;
    } else {
        // Eq. (TNEESApGra): T_b = (4 T(x_f) - T(x_ff)) / 3, zero normal gradient
        const R thff = dst[MTH * k.plane + (long long)w.yff * k.pitch + w.xff];
        m[MTH] = (R(4) * m[MTH] - thff) * (R(1) / R(3));
        if (w.fixgx) m[MGX] = R(0);
        if (w.fixgy) m[MGY] = R(0);
    }
    const long long at = (long long)y * k.pitch + x;
#pragma unroll
    for (int q = 0; q < kMPlanes; ++q) dst[q * k.plane + at] = m[q];
    if (!isfinite(m[MTH] + m[MP])) atomicOr(k.flag, 1);
}

// Band b of nb (columns [x0, x1)) and segment s of ns (rows [y0, y1)): the
// columns and rows are split as evenly as integer division allows.
struct Tile {
    int x0, x1, y0, y1;
};

__device__ __forceinline__ Tile tile_of(int nx, int ny) {
    Tile t;
    t.x0 = (int)((long long)blockIdx.x * nx / gridDim.x);
    t.x1 = (int)((long long)(blockIdx.x + 1) * nx / gridDim.x);
    t.y0 = (int)((long long)blockIdx.y * ny / gridDim.y);
    t.y1 = (int)((long long)(blockIdx.y + 1) * ny / gridDim.y);
    return t;
}

// One step from the moments in src to the moments in dst.  SOURCES = false:
// src is the state lbm_set_fields writes, whose populations are the
// equilibria alone (no F_i, P_i, Q_i).
template <class R, bool EPS_FIELD, bool SOURCES>
__global__ void __launch_bounds__(kMBlock, MomentOccupancy<R>::blocks)
k_step_m(const __grid_constant__ KConst<R> k, const R* __restrict__ src, R* dst) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* ring = reinterpret_cast<R*>(smem_raw);  // [kMRing][17][kMBlock]
    const int tid = threadIdx.x;
    const Tile t = tile_of(k.nx, k.ny);
    const bool perx = k.bc[SW] == BC_PERIODIC, pery = k.bc[SS] == BC_PERIODIC;

    // expansion column of this thread: x0 - 1 + tid, needed up to x1
    int xe = t.x0 - 1 + tid;
    bool xe_ok = xe <= t.x1;
    if (xe < 0 || xe >= k.nx) {
        if (perx) xe = xe < 0 ? xe + k.nx : xe - k.nx;
        else xe_ok = false;
    }
    // output column of this thread
    const int x = t.x0 - 1 + tid;
    const bool out_col = tid >= 1 && x < t.x1;

    // row r of the lattice as stored (periodic wrap), or -1 if it does not exist
    auto row_of = [&](int r) {
        if (r >= 0 && r < k.ny) return r;
        if (!pery) return -1;
        return r < 0 ? r + k.ny : r - k.ny;
    };
    // the moments of this thread's expansion node in row r (issued early so
    // that the loads are in flight while the previous row is processed)
    auto load_row = [&](int r, R* m) {
        r = row_of(r);
        if (r < 0 || !xe_ok) return;
        const R* s = src + ((long long)r * k.pitch + xe);
#pragma unroll
        for (int q = 0; q < kMPlanes; ++q) m[q] = s[q * k.plane32];
    };
    auto expand = [&](int r, int slot, const R* m) {
        r = row_of(r);
        if (r < 0 || !xe_ok) return;
        R fo[9], ho[9];
        if constexpr (EPS_FIELD) {
            KConst<R> kc = k;
            apply_eps(kc, node_eps(k, xe, r));
            fast_collide<R, true, SOURCES>(kc, state_from_moments(kc, m, r), nullptr, nullptr, fo, ho);
        } else {
            fast_collide<R, true, SOURCES>(k, state_from_moments(k, m, r), nullptr, nullptr, fo, ho);
        }
        R* sl = ring + slot * (NPLANES * kMBlock);
#pragma unroll
        for (int i = 1; i < 9; ++i) sl[(i - 1) * kMBlock + tid] = fo[i];
#pragma unroll
        for (int i = 0; i < 9; ++i) sl[(8 + i) * kMBlock + tid] = ho[i];
    };

    // interior node (x, y): pull from the ring (slots of rows y-1, y, y+1)
    auto update = [&](int y, int sm, int s0, int sp) {
        const R* rm = ring + sm * (NPLANES * kMBlock);
        const R* r0 = ring + s0 * (NPLANES * kMBlock);
        const R* rp = ring + sp * (NPLANES * kMBlock);
        R f[9], h[9];
        // f_i(x) = f_i*(x - c_i); c: 1 (+1,0) 2 (0,+1) 3 (-1,0) 4 (0,-1)
        // 5 (+1,+1) 6 (-1,+1) 7 (-1,-1) 8 (+1,-1)
        f[1] = r0[0 * kMBlock + tid - 1];
        f[2] = rm[1 * kMBlock + tid];
        f[3] = r0[2 * kMBlock + tid + 1];
        f[4] = rp[3 * kMBlock + tid];
        f[5] = rm[4 * kMBlock + tid - 1];
        f[6] = rm[5 * kMBlock + tid + 1];
        f[7] = rp[6 * kMBlock + tid + 1];
        f[8] = rp[7 * kMBlock + tid - 1];
        h[0] = r0[8 * kMBlock + tid];
        h[1] = r0[9 * kMBlock + tid - 1];
        h[2] = rm[10 * kMBlock + tid];
        h[3] = r0[11 * kMBlock + tid + 1];
        h[4] = rp[12 * kMBlock + tid];
        h[5] = rm[13 * kMBlock + tid - 1];
        h[6] = rm[14 * kMBlock + tid + 1];
        h[7] = rp[15 * kMBlock + tid + 1];
        h[8] = rp[16 * kMBlock + tid - 1];
        const long long at = (long long)y * k.pitch + x;
        if constexpr (EPS_FIELD) {
            KConst<R> kc = k;
            apply_eps(kc, node_eps(k, x, y));
            store_moments(k, dst, at, fast_moments(kc, f, h, y));
        } else {
            store_moments(k, dst, at, fast_moments(k, f, h, y));
        }
    };

    const bool wallS = !pery && t.y0 == 0;             // this segment holds the S wall row
    const bool wallN = !pery && t.y1 == k.ny;          // ... the N wall row
    const bool wallWE = !perx && (t.x0 == 0 || t.x1 == k.nx);
    int sm = 0, s0 = 1, sp = 2;
    R mnext[kMPlanes];
    load_row(t.y0 - 1, mnext);
    expand(t.y0 - 1, sm, mnext);
    load_row(t.y0, mnext);
    expand(t.y0, s0, mnext);
    load_row(t.y0 + 1, mnext);
    for (int y = t.y0; y < t.y1; ++y) {
        R mcur[kMPlanes];
#pragma unroll
        for (int q = 0; q < kMPlanes; ++q) mcur[q] = mnext[q];
        if (y + 2 <= t.y1) load_row(y + 2, mnext);
        expand(y + 1, sp, mcur);
        __syncthreads();
        const bool wall_row = (wallS && y == 0) || (wallN && y == k.ny - 1);
        if (!wall_row) {
            if (out_col && !is_wall_x(k, x)) update(y, sm, s0, sp);
            if (wallWE) {
                __syncthreads();  // x_f, x_ff of the W/E wall nodes are in this row
                if (out_col && is_wall_x(k, x)) wall_moments(k, dst, x, y);
            }
        } else if (y == k.ny - 1) {
            __syncthreads();  // rows ny-2, ny-3 are complete
            if (out_col) wall_moments(k, dst, x, y);
        }
        if (wallS && y == 2) {
            __syncthreads();  // rows 1 and 2 are complete: the S wall row
            if (out_col) wall_moments(k, dst, x, 0);
        }
        __syncthreads();  // the ring slot of row y - 1 is free
        const int tmp = sm;
        sm = s0;
        s0 = sp;
        sp = tmp;
    }
}

// Expansion of the moment state into the post-collision populations (the
// state the population kernels and the diagnostics read).
template <class R, bool SOURCES>
__global__ void k_expand_m(const __grid_constant__ KConst<R> k, const R* __restrict__ src, R* __restrict__ dst) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= k.nx) return;
    const long long at = (long long)y * k.pitch + x;
    R m[kMPlanes];
#pragma unroll
    for (int q = 0; q < kMPlanes; ++q) m[q] = src[q * k.plane + at];
    KConst<R> kc = k;
    if (k.eps_field) apply_eps(kc, node_eps(k, x, y));
    R fo[9], ho[9];
    fast_collide<R, true, SOURCES>(kc, state_from_moments(kc, m, y), nullptr, nullptr, fo, ho);
#pragma unroll
    for (int i = 1; i < 9; ++i) dst[(i - 1) * k.plane + at] = fo[i];
#pragma unroll
    for (int i = 0; i < 9; ++i) dst[(8 + i) * k.plane + at] = ho[i];
}

// The state lbm_set_fields defines: p = 0, S = 0, grad T = 0 with the given
// u and T (Sec. 3 initial state, as k_init).
template <class R>
__global__ void k_init_m(const __grid_constant__ KConst<R> k, R* __restrict__ dst, const double* __restrict__ T,
                         const double* __restrict__ ux, const double* __restrict__ uy, double T_init) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= k.nx) return;
    const long long c = (long long)y * k.nx + x;
    const long long at = (long long)y * k.pitch + x;
    R m[kMPlanes];
#pragma unroll
    for (int q = 0; q < kMPlanes; ++q) m[q] = R(0);
    m[MUX] = ux ? R(ux[c]) : R(0);
    m[MUY] = uy ? R(uy[c]) : R(0);
    m[MTH] = R((T ? T[c] : T_init) - double(k.T0));
#pragma unroll
    for (int q = 0; q < kMPlanes; ++q) dst[q * k.plane + at] = m[q];
}

// ------------------------------------------------------------------ launchers

template <class R>
size_t moment_smem_bytes() {
    return (size_t)kMRing * NPLANES * kMBlock * sizeof(R);
}

// The ring exceeds the default 48 KB of dynamic shared memory in FP64.
template <class R, bool E, bool S>
cudaError_t allow_smem() {
    // once per device (the attribute belongs to the function on the current device)
    static bool done[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < kMaxDevices && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_step_m<R, E, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)moment_smem_bytes<R>());
    if (e == cudaSuccess && dev < kMaxDevices) done[dev] = true;
    return e;
}

template <class R, bool E, bool S>
cudaError_t launch_m(const KConst<R>& k, const R* src, R* dst, dim3 grid, cudaStream_t st) {
    const size_t smem = moment_smem_bytes<R>();
    cudaError_t e = allow_smem<R, E, S>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kMBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step_m<R, E, S>, k, src, dst);
}

template <class R>
dim3 moment_grid(const KConst<R>& k, int segments) {
    const int nb = (k.nx + kMBand - 1) / kMBand;
    int ns = segments > 0 ? segments : 1;
    if (ns > k.ny / 3) ns = k.ny / 3 > 0 ? k.ny / 3 : 1;  // segments keep >= 3 rows
    return dim3((unsigned)nb, (unsigned)ns);
}

template <class R>
int moment_segments_default(const KConst<R>& k) {
    // about three waves of resident blocks (measured at 2048^2: one wave of
    // long segments 45.9 GLUPS, three waves 48.3, six 46.2), rows per
    // segment >= 3 (moment_grid clamps)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    if (allow_smem<R, false, true>() == cudaSuccess)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_m<R, false, true>, kMBlock,
                                                      moment_smem_bytes<R>());
    if (per_sm < 1) per_sm = 1;
    const int nb = (k.nx + kMBand - 1) / kMBand;
    int ns = 3 * (sms * per_sm) / nb;
    return ns < 1 ? 1 : ns;
}

template <class R>
cudaError_t launch_step_m(const KConst<R>& k, const R* src, R* dst, bool sources, int segments, cudaStream_t st) {
    const dim3 grid = moment_grid(k, segments);
    if (k.eps_field)
        return sources ? launch_m<R, true, true>(k, src, dst, grid, st) : launch_m<R, true, false>(k, src, dst, grid, st);
    return sources ? launch_m<R, false, true>(k, src, dst, grid, st) : launch_m<R, false, false>(k, src, dst, grid, st);
}

template <class R>
cudaError_t launch_expand_m(const KConst<R>& k, const R* src, R* dst, bool sources, cudaStream_t st) {
    const dim3 grid((unsigned)((k.nx + 127) / 128), (unsigned)k.ny);
    if (sources) k_expand_m<R, true><<<grid, 128, 0, st>>>(k, src, dst);
    else k_expand_m<R, false><<<grid, 128, 0, st>>>(k, src, dst);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_init_m(const KConst<R>& k, R* dst, const double* T, const double* ux, const double* uy,
                          double T_init, cudaStream_t st) {
    const dim3 grid((unsigned)((k.nx + 127) / 128), (unsigned)k.ny);
    k_init_m<R><<<grid, 128, 0, st>>>(k, dst, T, ux, uy, T_init);
    return cudaGetLastError();
}

#define LBM_MOMENT_INSTANTIATE(R)                                                                          \
    template cudaError_t launch_step_m<R>(const KConst<R>&, const R*, R*, bool, int, cudaStream_t);          \
    template cudaError_t launch_expand_m<R>(const KConst<R>&, const R*, R*, bool, cudaStream_t);              \
    template cudaError_t launch_init_m<R>(const KConst<R>&, R*, const double*, const double*, const double*, \
                                          double, cudaStream_t);                                            \
    template int moment_segments_default<R>(const KConst<R>&);

LBM_MOMENT_INSTANTIATE(float)
LBM_MOMENT_INSTANTIATE(double)

}  // namespace lbm
