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
//      17 post-collision populations,
//   2. pulls the 17 populations of each node from its neighbours,
//   3. computes the new moments (fast_moments), and the boundary state of the
//      wall nodes from their x_f, x_ff neighbours, and stores them.
// Each warp owns a strip of up to 30 columns (32 lanes: the strip and one
// halo column on each side) and a segment of rows, and marches up the
// segment: lane L expands its column's node of row y + 1 once, keeps in
// registers only the values still to be pulled (the six moving up, the five
// moving along x and staying, the six moving down), and takes its x
// neighbours' values by warp shuffles (12 per node).  No shared memory and
// no block barrier: the x_f and x_ff neighbours of a wall node always lie in
// the same strip (strips are at least 3 columns wide, segments at least 3
// rows tall); a W or E wall node takes their new moments from their lanes by
// shuffles, an S or N wall row reads them back from the output after a warp
// barrier.
// Every node is expanded once per strip and segment it borders (2 halo
// columns per 30, 2 halo rows per segment).
#include <math.h>

#include <algorithm>

#include "lbm_internal.h"

#ifndef LBM_MOMENT_WAVES
#define LBM_MOMENT_WAVES 2
#endif

namespace lbm {

constexpr int kMBlock = 128;     // threads per block: four independent warps
constexpr int kMStrip = 30;      // output columns of a strip, at most (32 lanes with the halo)
#ifndef LBM_MOMENT_BLOCKS
#define LBM_MOMENT_BLOCKS 5
#endif
template <class R> struct MomentOccupancy { static constexpr int blocks = LBM_MOMENT_BLOCKS; };
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

// Boundary state of wall node (x, y) from m, the new moments of its x_f node,
// and thff, the new temperature of its x_ff node (Sec. 3.4, as wall_state).
template <class R>
__device__ __forceinline__ void wall_store(const KConst<R>& k, R* dst, int x, int y, R* m, R thff) {
    const WallInfo w = classify(k, x, y);
    m[MUX] = k.u_bc[w.uside][0];
    m[MUY] = k.u_bc[w.uside][1];
    if (w.tside >= 0) {
        m[MTH] = k.T_bc[w.tside] - k.T0;
    } else {
        // Eq. (TNEESApGra): T_b = (4 T(x_f) - T(x_ff)) / 3, zero normal gradient
        m[MTH] = (R(4) * m[MTH] - thff) * (R(1) / R(3));
        if (w.fixgx) m[MGX] = R(0);
        if (w.fixgy) m[MGY] = R(0);
    }
    const long long at = (long long)y * k.pitch + x;
#pragma unroll
    for (int q = 0; q < kMPlanes; ++q) dst[q * k.plane + at] = m[q];
    if (!isfinite(m[MTH] + m[MP])) atomicOr(k.flag, 1);
}

// Boundary state of an S or N wall node (x, y), its x_f and x_ff neighbours
// read back from dst (written earlier in this launch by this warp).
template <class R>
__device__ __forceinline__ void wall_moments(const KConst<R>& k, R* dst, int x, int y) {
    const WallInfo w = classify(k, x, y);
    const long long af = (long long)w.ys * k.pitch + w.xs;
    R m[kMPlanes];
#pragma unroll
    for (int q = 0; q < kMPlanes; ++q) m[q] = dst[q * k.plane + af];
    const R thff = dst[MTH * k.plane + (long long)w.yff * k.pitch + w.xff];
    wall_store(k, dst, x, y, m, thff);
}

// Values of an expanded node that later rows pull: moving up (f2, f5, f6,
// h2, h5, h6; pulled by row y + 1), along x or resting (f1, f3, h0, h1, h3;
// pulled by row y) and moving down (f4, f7, f8, h4, h7, h8; pulled by row
// y - 1).
template <class R>
struct Expanded {
    R up[6], hz[5], dn[6];
};

// The moments of this lane's expansion node in row r (periodic wrap), or
// nothing when that row or column does not exist.
template <class R>
__device__ __forceinline__ void load_moments(const KConst<R>& k, const R* __restrict__ src, int r, int xe, bool ok,
                                             R* m) {
    if (!ok) return;
    const R* s = src + ((long long)r * k.pitch + xe);
#pragma unroll
    for (int q = 0; q < kMPlanes; ++q) m[q] = s[q * k.plane32];
}

template <class R, bool EPS_FIELD, bool SOURCES>
__device__ __forceinline__ Expanded<R> expand_node(const KConst<R>& k, const R* m, int xe, int r, bool ok) {
    Expanded<R> e;
    if (!ok) return e;
    R fo[9], ho[9];
    if constexpr (EPS_FIELD) {
        KConst<R> kc = k;
        apply_eps(kc, node_eps(k, xe, r));
        fast_collide<R, true, SOURCES>(kc, state_from_moments(kc, m, r), nullptr, nullptr, fo, ho);
    } else {
        fast_collide<R, true, SOURCES>(k, state_from_moments(k, m, r), nullptr, nullptr, fo, ho);
    }
    e.up[0] = fo[2]; e.up[1] = fo[5]; e.up[2] = fo[6];
    e.up[3] = ho[2]; e.up[4] = ho[5]; e.up[5] = ho[6];
    e.hz[0] = fo[1]; e.hz[1] = fo[3]; e.hz[2] = ho[0]; e.hz[3] = ho[1]; e.hz[4] = ho[3];
    e.dn[0] = fo[4]; e.dn[1] = fo[7]; e.dn[2] = fo[8];
    e.dn[3] = ho[4]; e.dn[4] = ho[7]; e.dn[5] = ho[8];
    return e;
}

// One step from the moments in src to the moments in dst.  SOURCES = false:
// src is the state lbm_set_fields writes, whose populations are the
// equilibria alone (no F_i, P_i, Q_i).  Warp g of the grid takes strip
// g % nstrips and segment g / nstrips; strips and segments split the columns
// and rows as evenly as integer division allows.
template <class R, bool EPS_FIELD, bool SOURCES>
__global__ void __launch_bounds__(kMBlock, MomentOccupancy<R>::blocks)
k_step_m(const __grid_constant__ KConst<R> k, const R* __restrict__ src, R* dst, int nstrips, int nseg) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * (kMBlock / 32) + (threadIdx.x >> 5);
    if (g >= nstrips * nseg) return;  // a whole warp leaves together
    const int strip = g % nstrips, seg = g / nstrips;
    const int xa = (int)((long long)strip * k.nx / nstrips), xb = (int)((long long)(strip + 1) * k.nx / nstrips);
    const int y0 = (int)((long long)seg * k.ny / nseg), y1 = (int)((long long)(seg + 1) * k.ny / nseg);
    const bool perx = k.bc[SW] == BC_PERIODIC, pery = k.bc[SS] == BC_PERIODIC;

    // expansion column of this lane: xa - 1 + lane, needed up to xb
    int xe = xa - 1 + lane;
    bool xe_ok = xe <= xb;
    if (xe < 0 || xe >= k.nx) {
        if (perx) xe = xe < 0 ? xe + k.nx : xe - k.nx;
        else xe_ok = false;
    }
    // output column of this lane
    const int x = xa - 1 + lane;
    const bool out_col = lane >= 1 && x < xb;
    const bool wall_col = out_col && is_wall_x(k, x);

    // row r of the lattice as stored (periodic wrap), or -1 if it does not exist
    auto row_of = [&](int r) {
        if (r >= 0 && r < k.ny) return r;
        if (!pery) return -1;
        return r < 0 ? r + k.ny : r - k.ny;
    };
    const bool wallS = !pery && y0 == 0;        // this segment holds the S wall row
    const bool wallN = !pery && y1 == k.ny;     // ... the N wall row
    const bool wallWE = !perx && (xa == 0 || xb == k.nx);

    R mn[kMPlanes];
    int r = row_of(y0 - 1);
    load_moments(k, src, r, xe, xe_ok && r >= 0, mn);
    Expanded<R> em = expand_node<R, EPS_FIELD, SOURCES>(k, mn, xe, r, xe_ok && r >= 0);  // row y - 1
    r = row_of(y0);
    load_moments(k, src, r, xe, xe_ok && r >= 0, mn);
    Expanded<R> e0 = expand_node<R, EPS_FIELD, SOURCES>(k, mn, xe, r, xe_ok && r >= 0);  // row y
    int rn = row_of(y0 + 1);
    load_moments(k, src, rn, xe, xe_ok && rn >= 0, mn);  // row y + 1, expanded in the loop
    for (int y = y0; y < y1; ++y) {
        R mc[kMPlanes];
#pragma unroll
        for (int q = 0; q < kMPlanes; ++q) mc[q] = mn[q];
        const int rc = rn;
        rn = row_of(y + 2);
        if (y + 2 <= y1) load_moments(k, src, rn, xe, xe_ok && rn >= 0, mn);
        const Expanded<R> ep = expand_node<R, EPS_FIELD, SOURCES>(k, mc, xe, rc, xe_ok && rc >= 0);  // row y + 1
        // pulls of node (x, y): f_i(x) = f_i*(x - c_i); c: 1 (+1,0) 2 (0,+1)
        // 3 (-1,0) 4 (0,-1) 5 (+1,+1) 6 (-1,+1) 7 (-1,-1) 8 (+1,-1)
        R f[9], h[9];
        f[1] = __shfl_up_sync(0xffffffffu, e0.hz[0], 1);
        f[2] = em.up[0];
        f[3] = __shfl_down_sync(0xffffffffu, e0.hz[1], 1);
        f[4] = ep.dn[0];
        f[5] = __shfl_up_sync(0xffffffffu, em.up[1], 1);
        f[6] = __shfl_down_sync(0xffffffffu, em.up[2], 1);
        f[7] = __shfl_down_sync(0xffffffffu, ep.dn[1], 1);
        f[8] = __shfl_up_sync(0xffffffffu, ep.dn[2], 1);
        h[0] = e0.hz[2];
        h[1] = __shfl_up_sync(0xffffffffu, e0.hz[3], 1);
        h[2] = em.up[3];
        h[3] = __shfl_down_sync(0xffffffffu, e0.hz[4], 1);
        h[4] = ep.dn[3];
        h[5] = __shfl_up_sync(0xffffffffu, em.up[4], 1);
        h[6] = __shfl_down_sync(0xffffffffu, em.up[5], 1);
        h[7] = __shfl_down_sync(0xffffffffu, ep.dn[4], 1);
        h[8] = __shfl_up_sync(0xffffffffu, ep.dn[5], 1);
        const bool wall_row = (wallS && y == 0) || (wallN && y == k.ny - 1);
        if (!wall_row) {
            FastState<R> s = {};
            if (out_col && !wall_col) {
                const long long at = (long long)y * k.pitch + x;
                if constexpr (EPS_FIELD) {
                    KConst<R> kc = k;
                    apply_eps(kc, node_eps(k, x, y));
                    s = fast_moments(kc, f, h, y);
                } else {
                    s = fast_moments(k, f, h, y);
                }
                store_moments(k, dst, at, s);
            }
            if (wallWE) {
                // x_f and x_ff of a W or E wall node are the nodes one and two
                // columns inward in this row and strip: their new moments come
                // from those lanes' registers (a read back from dst would hold
                // the whole warp on a memory round trip every row)
                const int in = x == 0 ? 1 : -1;
                const int lf = wall_col ? lane + in : lane, lff = wall_col ? lane + 2 * in : lane;
                R mf[kMPlanes];
                mf[MP] = __shfl_sync(0xffffffffu, s.p, lf);
                mf[MUX] = __shfl_sync(0xffffffffu, s.ux, lf);
                mf[MUY] = __shfl_sync(0xffffffffu, s.uy, lf);
                mf[MSXX] = __shfl_sync(0xffffffffu, s.Sxx, lf);
                mf[MSYY] = __shfl_sync(0xffffffffu, s.Syy, lf);
                mf[MSXY] = __shfl_sync(0xffffffffu, s.Sxy, lf);
                mf[MTH] = __shfl_sync(0xffffffffu, s.th, lf);
                mf[MGX] = __shfl_sync(0xffffffffu, s.gx, lf);
                mf[MGY] = __shfl_sync(0xffffffffu, s.gy, lf);
                const R thff = __shfl_sync(0xffffffffu, s.th, lff);
                if (wall_col) wall_store(k, dst, x, y, mf, thff);
            }
        } else if (y == k.ny - 1) {
            __syncwarp();  // rows ny-2, ny-3 of this strip are complete
            if (out_col) wall_moments(k, dst, x, y);
        }
        if (wallS && y == 2) {
            __syncwarp();  // rows 1 and 2 of this strip are complete: the S wall row
            if (out_col) wall_moments(k, dst, x, 0);
        }
        em = e0;
        e0 = ep;
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

// Strips of at most kMStrip columns (split evenly; at least 3 columns each
// for nx >= 4) and `segments` segments of at least 3 rows.
template <class R>
void moment_shape(const KConst<R>& k, int segments, int* nstrips, int* nseg) {
    *nstrips = (k.nx + kMStrip - 1) / kMStrip;
    int ns = segments > 0 ? segments : 1;
    if (ns > k.ny / 3) ns = k.ny / 3 > 0 ? k.ny / 3 : 1;
    *nseg = ns;
}

template <class R, bool E, bool S>
cudaError_t launch_m(const KConst<R>& k, const R* src, R* dst, int nstrips, int nseg, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    const long long warps = (long long)nstrips * nseg;
    cfg.gridDim = dim3((unsigned)((warps + kMBlock / 32 - 1) / (kMBlock / 32)));
    cfg.blockDim = dim3(kMBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step_m<R, E, S>, k, src, dst, nstrips, nseg);
}

template <class R>
int moment_segments_default(const KConst<R>& k) {
    // two waves of resident warps (segments of >= 3 rows; moment_shape clamps):
    // at 2048^2 one and two waves measure alike (52-58 GLUPS from box to
    // box), 1.2 waves 44.2 (the tail of a partial wave)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_m<R, false, true>, kMBlock, 0);
    if (per_sm < 1) per_sm = 1;
    const int nstrips = (k.nx + kMStrip - 1) / kMStrip;
    const long long warps = (long long)sms * per_sm * (kMBlock / 32);
    const long long ns = (LBM_MOMENT_WAVES * warps) / nstrips;
    return ns < 1 ? 1 : (int)std::min<long long>(ns, 1 << 20);
}

template <class R>
cudaError_t launch_step_m(const KConst<R>& k, const R* src, R* dst, bool sources, int segments, cudaStream_t st) {
    int nstrips = 0, nseg = 0;
    moment_shape(k, segments, &nstrips, &nseg);
    if (k.eps_field)
        return sources ? launch_m<R, true, true>(k, src, dst, nstrips, nseg, st)
                       : launch_m<R, true, false>(k, src, dst, nstrips, nseg, st);
    return sources ? launch_m<R, false, true>(k, src, dst, nstrips, nseg, st)
                   : launch_m<R, false, false>(k, src, dst, nstrips, nseg, st);
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
