// lbm_device.cuh -- per-node arithmetic of the modified LBGK step (device side).
//
// One node of one time step, in the order the paper defines it:
//   pull-stream f_i, g_i from x - c_i                      (Eq. LBEeq, streaming of Sec. 3.2)
//   T from sigma T = sum g + Q/2                            (Sec. 3.2)
//   G = g beta (T - T0) j + a; v; u from the quadratic solve (Sec. 3.1)
//   F = -eps nu/K u - eps F_eps/sqrt(K) |u| u + eps G        (Eq. ForceEq)
//   p from sum_{i!=0} f_i, F_0 and s_0                       (Sec. 3.1, Appendix A)
//   S from the non-equilibrium second moment                 (Eq. ShearEqCom)
//   grad T from the 2x2 system M grad T = N                  (Eqs. TeEqCom-MatrN)
//   collide f and g                                          (Eqs. LBEeq, TEqColli)
// Wall nodes are rebuilt by non-equilibrium extrapolation from x_f (Sec. 3.4).
//
// The tensor contractions are expanded in closed form for D2Q9 (c_s^2 = 1/3):
//   s_i  = w_i [3 cu + 4.5 cu^2/eps - 1.5 |u|^2/eps]
//   r_i  = 1.5 w_i A [cx^2 Sxx + 2 cx cy Sxy + cy^2 Syy - (Sxx + Syy)/3]
//   F_i  = w_i rho0 (1 - 1/2tau_f) [3 cF + 9 cu cF/eps - 3 u.F/eps]
//   P_i  = w_i (1 - 1/2tau_T) [3 c.(T F + eps p grad T/rho0) + 3 (1/eps - 1/sigma) cu (u.grad T)]
//   Q_i  = w_i (1 - 1/2tau_T) (1 + 3 cu/sigma) Q
// and the moments the local schemes need use the closed-form equilibrium
// moments (Appendix A, Eq. EqZEqu; Sec. 3.2, Eq. MeOtEq):
//   sum c c f^{e(0)} = eps p I + rho0 u u / eps,  sum c g^{e(0)} = T u.
//
// Storage: flow populations f_1..f_8 as they are (f_0 is never read: p uses
// sum_{i!=0} f_i, u uses sum c_i f_i, S uses sum c c (f - f^{e(0)})), thermal
// populations as deviations h_i = g_i - w_i sigma T0 from the rest state.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_half.cuh"

namespace lbm {

// D2Q9 in the paper's order (Sec. 3.1).
__host__ __device__ constexpr int cx_of(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
// Weight of the diagonal directions, 1/36.  In FP32, 1/9 and 4/9 round to
// exactly 4 and 16 times the rounded 1/36, so the nine rounded weights would
// sum to 36 fl(1/36) = 1 + 7.45e-9: every step would scale the zeroth
// moments (T - T0, and the pressure) by that factor, a bias that builds up
// to ~1e-4 of the temperature over 1e5 steps.  The FP32 value is therefore
// one unit in the last place below fl(1/36) (2^-29 smaller), which makes the
// FP32 weights sum to exactly 1; the second moment moves by 1.5e-8 relative
// (a constant change of the viscosity of that size, which does not build up).
template <class R>
__host__ __device__ constexpr R w_diag() { return R(1) / R(36); }
template <>
__host__ __device__ constexpr float w_diag<float>() { return 0x1.c71c7p-6f; }

template <class R>
__host__ __device__ constexpr R w_of(int i) {
    return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : w_diag<R>());
}

enum : int { BC_PERIODIC = 0, BC_DIRICHLET = 1, BC_ADIABATIC = 2 };
enum : int { SW = 0, SE = 1, SS = 2, SN = 3 };

// Constants of one run in the compute type R (filled on the host).
template <class R>
struct KConst {
    int nx, ny, pitch;     // pitch: elements per stored row
    int bc[4];
    long long plane;       // elements per stored plane (ny * pitch)
    R rho0, eps, inv_eps, sigma, inv_sigma;
    R omf, omT;            // 1 - 1/tau
    R tau_f, kf, kT;       // kf, kT = 1 - 1/(2 tau)
    R A, B, T0, gbeta, ax, ay, Q;
    R e_nuK, e_FK;         // eps nu / K, eps F_eps / sqrt(K)
    R c0, c0sq, c1;
    R p_pref;              // c_s^2 / (eps (1 - w_0)) = 3 / (5 eps)
    R invD;                // 1 / (c_s^2 rho0 (A - tau_f))
    R a_const;             // c_s^2 sigma (B - tau_T)
    R bcoef;               // (1/eps - 1/sigma) / 2
    R sT0;                 // sigma T0
    R T_bc[4];
    R u_bc[4][2];
    float scale;           // FP16 storage: stored value = population / scale
    float inv_scale;       // 1 / scale (a power of two)
    int* flag;             // non-finite flag (device)
    int plane32;           // plane stride as a 32-bit offset (17 planes < 2^31 elements)
    // porosity field (nullptr: uniform eps).  With a field, K follows the
    // Kozeny-Carman form of the Ergun permeability, K(eps) = K_ref r(eps) with
    // r(eps) = [eps^3 / (1 - eps)^2] / [eps_ref^3 / (1 - eps_ref)^2].
    const R* eps_field;    // [ny][nx]
    R kc_inv_ref;          // (1 - eps_ref)^2 / eps_ref^3
    R nu_over_Kref;        // nu / K_ref
    R inv_sqrt_Kref;       // 1 / sqrt(K_ref)
    R p_pref_eps;          // c_s^2 / (1 - w_0)
    int da_inf, forch;
    const R* ay_row;       // extra external acceleration a_y per row, or nullptr
    // constants of the interior fast path (see interior_update)
    R inv_rho0, half_eps_ax, half_eps, p_uF, p_uu;
    R fA_ep, fA_uu, fA_tr, fA_uF, f_cu2, f_ScS, f_cucF, f_cu, f_cF;
    R h_sig, h_uu, h_pT, h_kQ, h_cu2, h_u3, h_ug, h_uQ, h_g, h_W;
    R h0_sig, h0_uu, h0_pT, h0_kQ;
    // nodes at the end of a staged step's sweep whose stores ask L2 to keep
    // them (evict-last hint): the next step reads those rows first (0: none)
    long long l2_hot;
};

// Population storage conversion.
template <class S, class R>
__device__ __forceinline__ R load_pop(const S* p, float) { return R(*p); }
template <>
__device__ __forceinline__ float load_pop<__half, float>(const __half* p, float scale) {
    return __half2float(*p) * scale;
}
template <class S, class R>
__device__ __forceinline__ void store_pop(S* p, R v, float) { *p = S(v); }
template <>
__device__ __forceinline__ void store_pop<__half, float>(__half* p, float v, float scale) {
    *p = __float2half_rn(v / scale);
}

// Store of the 17 post-collision values of one node; FP16 storage rounds
// stochastically (dither != nullptr) or to nearest (lbm_half.cuh).
// evict_last (FP32 storage): the stores carry an L2 evict-last policy.
template <class S, class R>
__device__ __forceinline__ void store_planes(S* __restrict__ d, long long pl, const R* fo, const R* ho,
                                             float inv_scale, Dither* dither, bool evict_last = false) {
    if constexpr (std::is_same<S, __half>::value) {
        store_planes_half<R>(d, pl, fo, ho, inv_scale, dither);
    } else {
        if constexpr (std::is_same<S, float>::value) {
            if (evict_last) {
                uint64_t pol;
                asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
#pragma unroll
                for (int i = 1; i < 9; ++i)
                    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(d + (i - 1) * pl),
                                 "f"(float(fo[i])), "l"(pol) : "memory");
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(d + (8 + i) * pl),
                                 "f"(float(ho[i])), "l"(pol) : "memory");
                return;
            }
        }
#pragma unroll
        for (int i = 1; i < 9; ++i) d[(i - 1) * pl] = S(fo[i]);
#pragma unroll
        for (int i = 0; i < 9; ++i) d[(8 + i) * pl] = S(ho[i]);
    }
}

// Plane k of the stored state: k = 0..7 hold f_1..f_8, k = 8..16 hold h_0..h_8.
constexpr int NPLANES = 17;

template <class R>
struct Pops {
    R f[9];  // f[0] unused
    R h[9];
};

// Role of node (x, y): interior, or a wall node with its NEES neighbours.
struct WallInfo {
    int wall;       // 0 interior
    int xs, ys;     // node whose post-streaming state is used (x itself, or x_f)
    int xff, yff;   // x_ff for the Neumann extrapolation
    int tside;      // side whose Dirichlet T applies, -1: adiabatic
    int uside;      // side whose wall velocity applies
    int fixgx, fixgy;
};

template <class R>
__device__ __forceinline__ WallInfo classify(const KConst<R>& k, int x, int y) {
    WallInfo w;
    const bool onW = x == 0 && k.bc[SW] != BC_PERIODIC;
    const bool onE = x == k.nx - 1 && k.bc[SE] != BC_PERIODIC;
    const bool onS = y == 0 && k.bc[SS] != BC_PERIODIC;
    const bool onN = y == k.ny - 1 && k.bc[SN] != BC_PERIODIC;
    w.wall = onW || onE || onS || onN;
    const int dx = onW ? 1 : (onE ? -1 : 0);
    const int dy = onS ? 1 : (onN ? -1 : 0);
    w.xs = x + dx;
    w.ys = y + dy;
    w.xff = x + 2 * dx;
    w.yff = y + 2 * dy;
    const int xsd = onW ? SW : (onE ? SE : -1);
    const int ysd = onS ? SS : (onN ? SN : -1);
    w.tside = -1;
    if (xsd >= 0 && k.bc[xsd] == BC_DIRICHLET) w.tside = xsd;
    else if (ysd >= 0 && k.bc[ysd] == BC_DIRICHLET) w.tside = ysd;
    w.uside = xsd >= 0 ? xsd : (ysd >= 0 ? ysd : 0);
    w.fixgx = xsd >= 0;
    w.fixgy = ysd >= 0;
    return w;
}

template <class R>
__device__ __forceinline__ bool is_wall(const KConst<R>& k, int x, int y) {
    return (x == 0 && k.bc[SW] != BC_PERIODIC) || (x == k.nx - 1 && k.bc[SE] != BC_PERIODIC) ||
           (y == 0 && k.bc[SS] != BC_PERIODIC) || (y == k.ny - 1 && k.bc[SN] != BC_PERIODIC);
}

// Column x is a W or E wall column.
template <class R>
__device__ __forceinline__ bool is_wall_x(const KConst<R>& k, int x) {
    return (x == 0 && k.bc[SW] != BC_PERIODIC) || (x == k.nx - 1 && k.bc[SE] != BC_PERIODIC);
}

// Post-streaming populations of node (x, y): f_i and g_i pulled from x - c_i.
template <class R, class S>
__device__ __forceinline__ void pull(const KConst<R>& k, const S* __restrict__ src, int x, int y,
                                     Pops<R>& P) {
    const int xm = x == 0 ? k.nx - 1 : x - 1;
    const int xp = x == k.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? k.ny - 1 : y - 1;
    const int yp = y == k.ny - 1 ? 0 : y + 1;
    const long long r0 = (long long)y * k.pitch, rm = (long long)ym * k.pitch,
                    rp = (long long)yp * k.pitch;
    // source of direction i is x - c_i
    const long long at[9] = {r0 + x, r0 + xm, rm + x, r0 + xp, rp + x,
                             rm + xm, rm + xp, rp + xp, rp + xm};
    const float sc = k.scale;
#pragma unroll
    for (int i = 1; i < 9; ++i) P.f[i] = load_pop<S, R>(src + (long long)(i - 1) * k.plane + at[i], sc);
#pragma unroll
    for (int i = 0; i < 9; ++i) P.h[i] = load_pop<S, R>(src + (long long)(8 + i) * k.plane + at[i], sc);
    P.f[0] = R(0);
}

// Sum of the thermal deviations pulled into (x, y), accumulated in Acc (for T alone).
template <class Acc, class R, class S>
__device__ __forceinline__ Acc pull_hsum(const KConst<R>& k, const S* __restrict__ src, int x, int y) {
    const int xm = x == 0 ? k.nx - 1 : x - 1;
    const int xp = x == k.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? k.ny - 1 : y - 1;
    const int yp = y == k.ny - 1 ? 0 : y + 1;
    const long long r0 = (long long)y * k.pitch, rm = (long long)ym * k.pitch,
                    rp = (long long)yp * k.pitch;
    const long long at[9] = {r0 + x, r0 + xm, rm + x, r0 + xp, rp + x,
                             rm + xm, rm + xp, rp + xp, rp + xm};
    Acc s = Acc(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) s += Acc(load_pop<S, R>(src + (long long)(8 + i) * k.plane + at[i], k.scale));
    return s;
}

// ------------------------------------------------------------ dual numbers
// Forward-mode derivatives: a value and one tangent.  The generic per-node
// functions below are templates over the value type V (R, or Dual<R> for
// the adjoint), so the adjoint differentiates exactly the code that runs.
template <class R>
struct Dual {
    R v, d;
    __host__ __device__ Dual() : v(R(0)), d(R(0)) {}
    __host__ __device__ Dual(R v_) : v(v_), d(R(0)) {}
    __host__ __device__ Dual(R v_, R d_) : v(v_), d(d_) {}
};
template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, Dual<R> b) { return {a.v + b.v, a.d + b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, Dual<R> b) { return {a.v - b.v, a.d - b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, Dual<R> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, Dual<R> b) {
    const R q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a) { return {-a.v, -a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, R b) { return {a.v + b, a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator+(R a, Dual<R> b) { return {a + b.v, b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, R b) { return {a.v - b, a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(R a, Dual<R> b) { return {a - b.v, -b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, R b) { return {a.v * b, a.d * b}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(R a, Dual<R> b) { return {a * b.v, a * b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, R b) { return {a.v / b, a.d / b}; }
template <class R> __device__ __forceinline__ Dual<R> operator/(R a, Dual<R> b) {
    const R q = a / b.v;
    return {q, -q * b.d / b.v};
}

template <class R> __device__ __forceinline__ R val(R x) { return x; }
template <class R> __device__ __forceinline__ R val(Dual<R> x) { return x.v; }

// Square root of an argument that is never zero.
template <class R> __device__ __forceinline__ R vsqrt(R x) { return sqrt(x); }
template <class R> __device__ __forceinline__ Dual<R> vsqrt(Dual<R> x) {
    const R r = sqrt(x.v);
    return {r, x.d / (R(2) * r)};
}
// Euclidean norm from its square.  Where the vector is zero the norm is not
// differentiable, but it only enters multiplied by the vector itself
// (abs(v) v in the quadratic solve, abs(u) u in the Forchheimer drag), whose
// derivative there is zero: the tangent is set to 0.
template <class R> __device__ __forceinline__ R vnorm(R sq) { return sqrt(sq); }
template <class R> __device__ __forceinline__ Dual<R> vnorm(Dual<R> sq) {
    const R r = sqrt(sq.v);
    return {r, r > R(0) ? sq.d / (R(2) * r) : R(0)};
}

// Porosity-dependent constants of one node, and the y-component of the
// external acceleration a at its row.
template <class V>
struct CellC {
    V eps, inv_eps, e_nuK, e_FK, c0, c0sq, c1, p_pref, bcoef, ay;
};

// a_y at row y: the uniform a_y plus the optional per-row profile.
template <class R>
__device__ __forceinline__ R row_ay(const KConst<R>& k, int y) {
    return k.ay_row ? k.ay + k.ay_row[y] : k.ay;
}

template <class R>
__device__ __forceinline__ R node_eps(const KConst<R>& k, int x, int y) {
    return k.eps_field ? k.eps_field[(long long)y * k.nx + x] : k.eps;
}

// Constants at porosity eps: the run's own constants for a uniform porosity,
// else from the Kozeny-Carman permeability K(eps) and the Ergun F_eps(eps)
// (Sec. 2): e_nuK = eps nu/K, e_FK = eps F_eps/sqrt(K), c0 = (1 + e_nuK/2)/2,
// c1 = e_FK/2 (Sec. 3.1).
template <class R, class V>
__device__ __forceinline__ CellC<V> cell_consts(const KConst<R>& k, V eps) {
    CellC<V> c;
    if (!k.eps_field) {
        c.eps = V(k.eps);
        c.inv_eps = V(k.inv_eps);
        c.e_nuK = V(k.e_nuK);
        c.e_FK = V(k.e_FK);
        c.c0 = V(k.c0);
        c.c0sq = V(k.c0sq);
        c.c1 = V(k.c1);
        c.p_pref = V(k.p_pref);
        c.bcoef = V(k.bcoef);
        c.ay = V(k.ay);
        return c;
    }
    c.eps = eps;
    c.inv_eps = R(1) / eps;
    if (k.da_inf) {
        c.e_nuK = V(R(0));
        c.e_FK = V(R(0));
    } else {
        const V om = R(1) - eps;
        const V ratio = eps * eps * eps / (om * om) * k.kc_inv_ref;  // K / K_ref
        c.e_nuK = eps * k.nu_over_Kref / ratio;
        if (k.forch) {
            const V Feps = R(1.75) / vsqrt(R(150) * eps * eps * eps);
            c.e_FK = eps * Feps * k.inv_sqrt_Kref / vsqrt(ratio);
        } else {
            c.e_FK = V(R(0));
        }
    }
    c.c0 = R(0.5) + R(0.25) * c.e_nuK;
    c.c0sq = c.c0 * c.c0;
    c.c1 = R(0.5) * c.e_FK;
    c.p_pref = k.p_pref_eps * c.inv_eps;
    c.bcoef = R(0.5) * (c.inv_eps - k.inv_sigma);
    c.ay = V(k.ay);
    return c;
}

template <class V>
struct State {
    V th;               // T - T0
    V ux, uy, Fx, Fy;   // velocity, total force
    V p;
    V Sxx, Sxy, Syy;    // shear rate
    V gx, gy;           // grad T
};

// Moments of one node from its post-streaming populations (f[1..8], h[0..8]).
template <class R, class V>
__device__ __forceinline__ State<V> node_moments(const KConst<R>& k, const CellC<V>& c, const V* f,
                                                 const V* h) {
    State<V> s;
    // sigma T = sum g + Q/2, with sum g = sum h + sigma T0
    const V sh = h[0] + h[1] + h[2] + h[3] + h[4] + h[5] + h[6] + h[7] + h[8];
    s.th = (sh + R(0.5) * k.Q) * k.inv_sigma;
    const V T = k.T0 + s.th;
    // flow moments
    const V sf = f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    const V mx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const V my = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
    const V d58 = f[5] + f[6] + f[7] + f[8];
    const V Pxx = f[1] + f[3] + d58;
    const V Pyy = f[2] + f[4] + d58;
    const V Pxy = (f[5] + f[7]) - (f[6] + f[8]);
    // buoyancy, temporary velocity, quadratic solve
    const R Gx = k.ax;
    const V Gy = k.gbeta * s.th + c.ay;
    const V vx = mx * k.inv_rho0 + R(0.5) * c.eps * Gx;
    const V vy = my * k.inv_rho0 + R(0.5) * c.eps * Gy;
    const V vmag = vnorm(vx * vx + vy * vy);
    const V den = c.c0 + vsqrt(c.c0sq + c.c1 * vmag);
    s.ux = vx / den;
    s.uy = vy / den;
    const V uu = s.ux * s.ux + s.uy * s.uy;
    const V umag = vnorm(uu);
    const V drag = c.e_nuK + c.e_FK * umag;
    s.Fx = c.eps * Gx - drag * s.ux;
    s.Fy = c.eps * Gy - drag * s.uy;
    const V uF = s.ux * s.Fx + s.uy * s.Fy;
    // p = c_s^2/(eps (1-w0)) [sum_{i!=0} f + tau_f F_0 + rho0 s_0],
    // F_0 = -3 w0 rho0 kf u.F/eps, s_0 = -1.5 w0 |u|^2/eps, w0 = 4/9
    const V F0 = -(R(4) / R(3)) * k.rho0 * k.kf * uF * c.inv_eps;
    const V s0 = -(R(2) / R(3)) * uu * c.inv_eps;
    s.p = c.p_pref * (sf + k.tau_f * F0 + k.rho0 * s0);
    // S = [Pi - eps p I - rho0 u u/eps + (rho0/2)(uF + Fu)/eps] / (c_s^2 rho0 (A - tau_f))
    const V re = k.rho0 * c.inv_eps;
    const V ep = c.eps * s.p;
    s.Sxx = (Pxx - ep - re * s.ux * s.ux + re * s.ux * s.Fx) * k.invD;
    s.Syy = (Pyy - ep - re * s.uy * s.uy + re * s.uy * s.Fy) * k.invD;
    s.Sxy = (Pxy - re * s.ux * s.uy + R(0.5) * re * (s.ux * s.Fy + s.Fx * s.uy)) * k.invD;
    // N = sum c (g - g^{e(0)}) + (T F + u Q/sigma)/2 with sum c g^{e(0)} = T u
    const V nx_ = (h[1] - h[3]) + (h[5] - h[6]) + (h[8] - h[7]);
    const V ny_ = (h[2] - h[4]) + (h[5] - h[8]) + (h[6] - h[7]);
    const R qs = R(0.5) * k.Q * k.inv_sigma;
    const V Nx = nx_ - T * s.ux + R(0.5) * T * s.Fx + qs * s.ux;
    const V Ny = ny_ - T * s.uy + R(0.5) * T * s.Fy + qs * s.uy;
    // M = a I - b u u^T, a = -eps p/(2 rho0) + c_s^2 sigma (B - tau_T),
    // b = (1/eps - 1/sigma)/2; M^{-1} N = (N + b u (u.N)/(a - b|u|^2)) / a
    const V a = k.a_const - R(0.5) * ep * k.inv_rho0;
    const V uN = s.ux * Nx + s.uy * Ny;
    const V t = c.bcoef * uN / (a - c.bcoef * uu);
    const V ia = R(1) / a;
    s.gx = (Nx + t * s.ux) * ia;
    s.gy = (Ny + t * s.uy) * ia;
    return s;
}

// Equilibria and source terms of one state, direction by direction.
template <class V>
struct EqTerms {
    V fe[9];   // f^eq_i, i = 1..8 (index 0 unused)
    V Fi[9];   // forcing term F_i, i = 1..8
    V he[9];   // g^eq_i - w_i sigma T0
    V PQ[9];   // P_i + Q_i
};

template <class R, class V>
__device__ __forceinline__ void eq_terms(const KConst<R>& k, const CellC<V>& c, const State<V>& s,
                                         EqTerms<V>& e) {
    const V T = k.T0 + s.th;
    const V uu = s.ux * s.ux + s.uy * s.uy;
    const V ie = c.inv_eps;
    const V flow_c = R(3) * c.eps * s.p - R(1.5) * k.rho0 * uu * ie - R(0.5) * k.rho0 * k.A * (s.Sxx + s.Syy);
    const V uF = s.ux * s.Fx + s.uy * s.Fy;
    const V force_c = -R(3) * uF * ie;
    const V pT = R(3) * T * c.eps * s.p * k.inv_rho0;   // 3 T eps p / rho0
    const V ug = s.ux * s.gx + s.uy * s.gy;
    const V Wx = T * s.Fx + c.eps * s.p * s.gx * k.inv_rho0;
    const V Wy = T * s.Fy + c.eps * s.p * s.gy * k.inv_rho0;
    const V therm_c = k.sigma * s.th - R(1.5) * T * uu * ie;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R cx = R(cx_of(i)), cy = R(cy_of(i));
        const R w = w_of<R>(i);
        const V cu = cx * s.ux + cy * s.uy;
        const V cF = cx * s.Fx + cy * s.Fy;
        if (i > 0) {
            const V ScS = cx * cx * s.Sxx + R(2) * cx * cy * s.Sxy + cy * cy * s.Syy;
            e.fe[i] = w * (flow_c + k.rho0 * (R(3) * cu + R(4.5) * cu * cu * ie) + R(1.5) * k.rho0 * k.A * ScS);
            e.Fi[i] = w * k.rho0 * k.kf * (R(3) * cF + R(9) * cu * cF * ie + force_c);
        } else {
            e.fe[0] = V(R(0));
            e.Fi[0] = V(R(0));
        }
        const V cg = cx * s.gx + cy * s.gy;
        // varpi_0 = -5/9 = -(1 - w0); varpi_i = w_i otherwise
        const V pv = (i == 0) ? -(R(5) / R(9)) * pT : w * pT;
        e.he[i] = w * (therm_c + T * (R(3) * cu + R(4.5) * cu * cu * ie) + k.sigma * k.B * cg) + pv;
        const V cW = cx * Wx + cy * Wy;
        e.PQ[i] = w * k.kT * (R(3) * cW + R(6) * c.bcoef * cu * ug + (R(1) + R(3) * cu * k.inv_sigma) * k.Q);
    }
}

// Boundary state of a wall node (Sec. 3.4): u_b, T_b, p(x_f), S(x_f),
// grad T_b, and F at (u_b, T_b) with the wall node's own porosity (cb).
// thff is T(x_ff) - T0 (adiabatic walls), thb the Dirichlet T_b - T0.
template <class R, class V>
__device__ __forceinline__ State<V> wall_state(const KConst<R>& k, const CellC<V>& cb, const WallInfo& w,
                                               const State<V>& sf, V thff, V thb) {
    State<V> b = sf;
    b.ux = V(k.u_bc[w.uside][0]);
    b.uy = V(k.u_bc[w.uside][1]);
    if (w.tside >= 0) {
        b.th = thb;
    } else {
        // Eq. (TNEESApGra) with zero normal gradient
        if (w.fixgx) b.gx = V(R(0));
        if (w.fixgy) b.gy = V(R(0));
        b.th = (R(4) * sf.th - thff) * (R(1) / R(3));
    }
    const V umag = vnorm(b.ux * b.ux + b.uy * b.uy);
    const V drag = cb.e_nuK + cb.e_FK * umag;
    b.Fx = cb.eps * k.ax - drag * b.ux;
    b.Fy = cb.eps * (k.gbeta * b.th + cb.ay) - drag * b.uy;
    return b;
}

// out[i-1] += a_f f^eq_i + b_f F_i (i = 1..8) and out[8+i] += a_g h^eq_i +
// b_g (P_i + Q_i) (i = 0..8): the equilibria and sources of one state
// accumulated straight into the outputs, so no per-direction array stays
// live (the wall path then fits the step kernel's register budget).
template <class R, class V>
__device__ __forceinline__ void eq_accumulate(const KConst<R>& k, const CellC<V>& c, const State<V>& s, R a_f,
                                              R b_f, R a_g, R b_g, V* out) {
    const V T = k.T0 + s.th;
    const V uu = s.ux * s.ux + s.uy * s.uy;
    const V ie = c.inv_eps;
    const V flow_c = R(3) * c.eps * s.p - R(1.5) * k.rho0 * uu * ie - R(0.5) * k.rho0 * k.A * (s.Sxx + s.Syy);
    const V uF = s.ux * s.Fx + s.uy * s.Fy;
    const V force_c = -R(3) * uF * ie;
    const V pT = R(3) * T * c.eps * s.p * k.inv_rho0;
    const V ug = s.ux * s.gx + s.uy * s.gy;
    const V Wx = T * s.Fx + c.eps * s.p * s.gx * k.inv_rho0;
    const V Wy = T * s.Fy + c.eps * s.p * s.gy * k.inv_rho0;
    const V therm_c = k.sigma * s.th - R(1.5) * T * uu * ie;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R cx = R(cx_of(i)), cy = R(cy_of(i));
        const R w = w_of<R>(i);
        const V cu = cx * s.ux + cy * s.uy;
        if (i > 0) {
            const V cF = cx * s.Fx + cy * s.Fy;
            const V ScS = cx * cx * s.Sxx + R(2) * cx * cy * s.Sxy + cy * cy * s.Syy;
            const V fe = w * (flow_c + k.rho0 * (R(3) * cu + R(4.5) * cu * cu * ie) + R(1.5) * k.rho0 * k.A * ScS);
            const V Fi = w * k.rho0 * k.kf * (R(3) * cF + R(9) * cu * cF * ie + force_c);
            out[i - 1] = out[i - 1] + a_f * fe + b_f * Fi;
        }
        const V cg = cx * s.gx + cy * s.gy;
        const V pv = (i == 0) ? -(R(5) / R(9)) * pT : w * pT;
        const V he = w * (therm_c + T * (R(3) * cu + R(4.5) * cu * cu * ie) + k.sigma * k.B * cg) + pv;
        const V cW = cx * Wx + cy * Wy;
        const V PQ = w * k.kT * (R(3) * cW + R(6) * c.bcoef * cu * ug + (R(1) + R(3) * cu * k.inv_sigma) * k.Q);
        out[8 + i] = out[8 + i] + a_g * he + b_g * PQ;
    }
}

// The whole update of one node in the generic form: inputs are the 17
// populations pulled at the source node (the node itself, or x_f for a wall
// node), the porosity at the source and at the node, T(x_ff) - T0, the
// Dirichlet T_b - T0 and a_y at the rows of the source and of the node;
// outputs the 17 post-collision values.  Interior nodes:
// BGK collision (Eqs. LBEeq, TEqColli),
//   f* = (1 - 1/tau) f + f^eq/tau + F_i.
// Wall nodes: NEES rebuild (Eqs. NEESVel, TNEESAp) and collision with the
// boundary equilibrium,
//   f* = (1 - 1/tau)[f(x_f) - f^eq(x_f)] + f^eq(x_b) + F_i(x_b).
template <class R, class V>
__device__ __forceinline__ void node_update_generic(const KConst<R>& k, const WallInfo& w, const V* in,
                                                    V eps_s, V eps_x, V thff, V thb, R ay_s, R ay_x, V* out) {
    V f[9], h[9];
    f[0] = V(R(0));
#pragma unroll
    for (int i = 1; i < 9; ++i) f[i] = in[i - 1];
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = in[8 + i];
    CellC<V> cs = cell_consts(k, eps_s);
    cs.ay = V(ay_s);
    const State<V> s = node_moments(k, cs, f, h);
#pragma unroll
    for (int q = 0; q < 8; ++q) out[q] = k.omf * in[q];
#pragma unroll
    for (int q = 8; q < 17; ++q) out[q] = k.omT * in[q];
    if (!w.wall) {
        eq_accumulate(k, cs, s, R(1) - k.omf, R(1), R(1) - k.omT, R(1), out);
        return;
    }
    eq_accumulate(k, cs, s, -k.omf, R(0), -k.omT, R(0), out);
    CellC<V> cb = cell_consts(k, eps_x);
    cb.ay = V(ay_x);
    const State<V> b = wall_state(k, cb, w, s, thff, thb);
    eq_accumulate(k, cb, b, R(1), R(1), R(1), R(1), out);
}

// Fast-path constants of a node with its own porosity (porosity field).
template <class R>
__device__ __forceinline__ void apply_eps(KConst<R>& k, R eps) {
    const CellC<R> c = cell_consts(k, eps);
    const R itf = R(1) - k.omf, itT = R(1) - k.omT;
    k.eps = eps;
    k.inv_eps = c.inv_eps;
    k.e_nuK = c.e_nuK;
    k.e_FK = c.e_FK;
    k.c0 = c.c0;
    k.c0sq = c.c0sq;
    k.c1 = c.c1;
    k.p_pref = c.p_pref;
    k.bcoef = c.bcoef;
    k.half_eps = R(0.5) * eps;
    k.half_eps_ax = R(0.5) * eps * k.ax;
    k.p_uF = c.p_pref * (R(4) / R(3)) * k.rho0 * k.kf * k.tau_f * c.inv_eps;
    k.p_uu = c.p_pref * (R(2) / R(3)) * k.rho0 * c.inv_eps;
    k.fA_uu = R(1.5) * itf * k.rho0 * c.inv_eps;
    k.fA_uF = R(3) * k.rho0 * k.kf * c.inv_eps;
    k.f_cu2 = R(4.5) * itf * k.rho0 * c.inv_eps;
    k.f_cucF = R(9) * k.rho0 * k.kf * c.inv_eps;
    k.h_uu = itT * R(1.5) * c.inv_eps;
    k.h_cu2 = itT * R(4.5) * c.inv_eps;
    k.h_ug = R(6) * k.kT * c.bcoef;
    k.h0_uu = itT * (R(4) / R(9)) * R(1.5) * c.inv_eps;
}

// Macroscopic state of a node in the fast path: the moments the step
// computes after streaming (Sec. 3.1-3.3) plus the derived quantities the
// collision uses.
template <class R>
struct FastState {
    R th, T, ux, uy, uu, Fx, Fy, uF, p, ep, Sxx, Syy, Sxy, gx, gy;
};

// Planes of the moment state (tau = 1 storage): p, u, S, T - T0, grad T.
enum MomentPlane { MP = 0, MUX, MUY, MSXX, MSYY, MSXY, MTH, MGX, MGY };
constexpr int kMPlanes = 9;

// Moments of an interior node from its pulled populations (f[1..8], h[0..8]),
// in the fast path's arrangement of node_moments.
template <class R>
__device__ __forceinline__ FastState<R> fast_moments(const KConst<R>& k, const R* f, const R* h, int y) {
    FastState<R> s;
    const R sh = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
    s.th = (sh + R(0.5) * k.Q) * k.inv_sigma;
    s.T = k.T0 + s.th;
    const R a13 = f[1] + f[3], a24 = f[2] + f[4], d58 = (f[5] + f[7]) + (f[6] + f[8]);
    const R sf = a13 + a24 + d58;
    const R mx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
    const R my = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
    const R Pxx = a13 + d58, Pyy = a24 + d58;
    const R Pxy = (f[5] + f[7]) - (f[6] + f[8]);
    const R Gy = k.gbeta * s.th + row_ay(k, y);
    const R vx = mx * k.inv_rho0 + k.half_eps_ax;
    const R vy = my * k.inv_rho0 + k.half_eps * Gy;
    const R vmag = sqrt(vx * vx + vy * vy);
    const R iden = R(1) / (k.c0 + sqrt(k.c0sq + k.c1 * vmag));
    s.ux = vx * iden;
    s.uy = vy * iden;
    if (!isfinite(s.th + s.ux + s.uy)) atomicOr(k.flag, 1);
    s.uu = s.ux * s.ux + s.uy * s.uy;
    // |u| = |v| / (c0 + sqrt(c0^2 + c1 |v|)): no second square root
    const R drag = k.e_nuK + k.e_FK * (vmag * iden);
    s.Fx = k.eps * k.ax - drag * s.ux;
    s.Fy = k.eps * Gy - drag * s.uy;
    s.uF = s.ux * s.Fx + s.uy * s.Fy;
    const R p = k.p_pref * sf - k.p_uF * s.uF - k.p_uu * s.uu;
    s.p = p;
    s.ep = k.eps * p;
    const R re = k.rho0 * k.inv_eps;
    s.Sxx = (Pxx - s.ep + re * s.ux * (s.Fx - s.ux)) * k.invD;
    s.Syy = (Pyy - s.ep + re * s.uy * (s.Fy - s.uy)) * k.invD;
    s.Sxy = (Pxy + re * (R(0.5) * (s.ux * s.Fy + s.Fx * s.uy) - s.ux * s.uy)) * k.invD;
    const R hx = (h[1] - h[3]) + (h[5] - h[7]) + (h[8] - h[6]);
    const R hy = (h[2] - h[4]) + (h[5] - h[7]) + (h[6] - h[8]);
    const R qs = R(0.5) * k.Q * k.inv_sigma;
    const R Nx = hx + s.T * (R(0.5) * s.Fx - s.ux) + qs * s.ux;
    const R Ny = hy + s.T * (R(0.5) * s.Fy - s.uy) + qs * s.uy;
    const R a = k.a_const - R(0.5) * s.ep * k.inv_rho0;
    const R d = a - k.bcoef * s.uu;
    // one reciprocal for 1/a = d r and 1/d = a r, r = 1/(a d)
    const R r = R(1) / (a * d);
    const R t = k.bcoef * (s.ux * Nx + s.uy * Ny) * (a * r);
    const R ia = d * r;
    s.gx = (Nx + t * s.ux) * ia;
    s.gy = (Ny + t * s.uy) * ia;
    return s;
}

// Collision of one node from its state: h_i* = (1 - 1/tau) h_i +
// [h_i^eq/tau + source_i], the bracket split into the parts even and odd
// under c_i -> -c_i so that each pair of opposite directions shares one
// evaluation.  TAU1: tau_f = tau_T = 1, where the first term vanishes and
// f, h are not read.  SOURCES = false drops the force and heat-source terms
// (F_i, P_i, Q_i) and keeps the equilibria alone.  wscale (TAU1 only)
// multiplies every output: the FP16 storage scale folded into the weights.
template <class R, bool TAU1, bool SOURCES = true>
__device__ __forceinline__ void fast_collide(const KConst<R>& k, const FastState<R>& s, const R* f,
                                             const R* h, R* fo, R* ho, R wscale = R(1)) {
    const R uF = SOURCES ? s.uF : R(0);
    const R Fx = SOURCES ? s.Fx : R(0), Fy = SOURCES ? s.Fy : R(0);
    const R kQ = SOURCES ? k.h_kQ : R(0), uQ = SOURCES ? k.h_uQ : R(0), k0Q = SOURCES ? k.h0_kQ : R(0);
    const R T = s.T, ep = s.ep, uu = s.uu, ux = s.ux, uy = s.uy, gx = s.gx, gy = s.gy;
    const R EF0 = k.fA_ep * ep - k.fA_uu * uu - k.fA_tr * (s.Sxx + s.Syy) - k.fA_uF * uF;
    const R EH0 = k.h_sig * s.th - k.h_uu * T * uu + k.h_pT * T * ep + kQ;
    const R Kc = k.h_cu2 * T;
    const R Ku = k.h_u3 * T + (SOURCES ? k.h_ug * (ux * gx + uy * gy) : R(0)) + uQ;
    const R epr = ep * k.inv_rho0;
    const R Wx = SOURCES ? T * Fx + epr * gx : R(0), Wy = SOURCES ? T * Fy + epr * gy : R(0);
    auto pair = [&](int i, int j, R w, R cu, R cF, R ScS, R cg, R cW) {
        const R evF = EF0 + k.f_cu2 * cu * cu + k.f_ScS * ScS + k.f_cucF * cu * cF;
        const R odF = k.f_cu * cu + k.f_cF * cF;
        const R evH = EH0 + Kc * cu * cu;
        const R odH = Ku * cu + k.h_g * cg + k.h_W * cW;
        if (TAU1) {
            fo[i] = w * (evF + odF);
            fo[j] = w * (evF - odF);
            ho[i] = w * (evH + odH);
            ho[j] = w * (evH - odH);
        } else {
            fo[i] = k.omf * f[i] + w * (evF + odF);
            fo[j] = k.omf * f[j] + w * (evF - odF);
            ho[i] = k.omT * h[i] + w * (evH + odH);
            ho[j] = k.omT * h[j] + w * (evH - odH);
        }
    };
    const R w1 = wscale * (R(1) / R(9)), w5 = wscale * w_diag<R>();
    pair(1, 3, w1, ux, Fx, s.Sxx, gx, Wx);
    pair(2, 4, w1, uy, Fy, s.Syy, gy, Wy);
    pair(5, 7, w5, ux + uy, Fx + Fy, s.Sxx + s.Syy + R(2) * s.Sxy, gx + gy, Wx + Wy);
    pair(6, 8, w5, uy - ux, Fy - Fx, s.Sxx + s.Syy - R(2) * s.Sxy, gy - gx, Wy - Wx);
    const R c0 = k.h0_sig * s.th - k.h0_uu * T * uu - k.h0_pT * T * ep + k0Q;
    ho[0] = TAU1 ? wscale * c0 : k.omT * h[0] + c0;
}

// Interior node of one step, fast path.  Same arithmetic as node_moments +
// eq_terms + BGK collision, rearranged for the GPU: the nine pull sources are
// 32-bit offsets from the node (periodic wrap by per-thread deltas), plane
// strides are uniform across the launch; then fast_moments and fast_collide.
// TAU1: tau_f = tau_T = 1 (no (1 - 1/tau) terms; FP16 storage then takes its
// scale in the collision weights).
template <class R, class S, bool TAU1 = false>
__device__ __forceinline__ void interior_update(const KConst<R>& k, const S* __restrict__ src,
                                                S* __restrict__ dst, int x, int y, uint32_t step) {
    const int dxm = x == 0 ? k.nx - 1 : -1;
    const int dxp = x == k.nx - 1 ? 1 - k.nx : 1;
    const int dym = y == 0 ? (k.ny - 1) * k.pitch : -k.pitch;
    const int dyp = y == k.ny - 1 ? (1 - k.ny) * k.pitch : k.pitch;
    const int o[9] = {0, dxm, dym, dxp, dyp, dxm + dym, dxp + dym, dxp + dyp, dxm + dyp};
    const int pl = k.plane32;
    const int at = y * k.pitch + x;
    const S* __restrict__ c = src + at;
    const float sc = k.scale;
    R f[9], h[9];
#pragma unroll
    for (int i = 1; i < 9; ++i) f[i] = load_pop<S, R>(c + ((i - 1) * pl + o[i]), sc);
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = load_pop<S, R>(c + ((8 + i) * pl + o[i]), sc);
    const FastState<R> s = fast_moments(k, f, h, y);
    R fo[9], ho[9];
    constexpr bool prescale = TAU1 && std::is_same<S, __half>::value;
    if constexpr (TAU1) fast_collide<R, true>(k, s, f, h, fo, ho, prescale ? R(k.inv_scale) : R(1));
    else fast_collide<R, false>(k, s, f, h, fo, ho);
    Dither dither((uint32_t)at, step);
    store_planes<S, R>(dst + at, pl, fo, ho, prescale ? 1.0f : k.inv_scale, &dither);
}

}  // namespace lbm
