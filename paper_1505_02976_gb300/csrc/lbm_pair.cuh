// lbm_pair.cuh -- the interior update at tau_f = tau_T = 1 written once for
// one node (lane type float) or two nodes at a time (lane type float2, the
// packed FP32 instructions: one instruction applies the same operation to
// both nodes).
//
// Same moments, quadratic solve, force, pressure, shear rate, temperature
// gradient and collision as fast_moments / fast_collide (lbm_device.cuh,
// Secs. 3.1-3.3, Eqs. EQFIN-Eq:Tforce), with every arithmetic operation
// spelled out (add, multiply, fused multiply-add).  Each packed operation
// rounds per lane as the scalar one does, but the compiler may fuse a packed
// multiply into the add or subtraction that consumes it (one rounding where
// the scalar code has two), so the results agree with fast_moments /
// fast_collide to FP32 rounding, not bit for bit.  Used by the FP16-storage
// staged step on its pairs of interior nodes.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// ---------------------------------------------------------------- lane ops
__device__ __forceinline__ float lbc(float, float c) { return c; }
__device__ __forceinline__ float2 lbc(float2, float c) { return make_float2(c, c); }
// The packed operations are PTX with round-to-nearest and flush-to-zero
// (the scalar arithmetic of this build runs with -ftz=true).
__device__ __forceinline__ unsigned long long lbits(float2 a) { return *reinterpret_cast<unsigned long long*>(&a); }
__device__ __forceinline__ float2 lfrom(unsigned long long u) { return *reinterpret_cast<float2*>(&u); }
__device__ __forceinline__ float ladd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 ladd(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(lbits(a)), "l"(lbits(b)));
    return lfrom(r);
}
__device__ __forceinline__ float lsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float2 lsub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(lbits(a)), "l"(lbits(b)));
    return lfrom(r);
}
__device__ __forceinline__ float lmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 lmul(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(lbits(a)), "l"(lbits(b)));
    return lfrom(r);
}
// a * b + c, one rounding
__device__ __forceinline__ float lfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 lfma(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(lbits(a)), "l"(lbits(b)), "l"(lbits(c)));
    return lfrom(r);
}
__device__ __forceinline__ float lsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ float2 lsqrt(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
__device__ __forceinline__ float lrcp(float a) { return 1.0f / a; }
__device__ __forceinline__ float2 lrcp(float2 a) { return make_float2(1.0f / a.x, 1.0f / a.y); }
__device__ __forceinline__ float lsum(float a) { return a; }
__device__ __forceinline__ float lsum(float2 a) { return a.x + a.y; }

template <class L>
struct LaneState {
    L th, T, ux, uy, uu, Fx, Fy, uF, ep, Sxx, Syy, Sxy, gx, gy;
};

// Moments of interior nodes from their pulled populations (f[1..8],
// h[0..8]), the arrangement of fast_moments with explicit operations.
template <class L>
__device__ __forceinline__ LaneState<L> lane_moments(const KConst<float>& k, const L* f, const L* h, int y) {
    const L z = lbc(L(), 0.f);
    LaneState<L> s;
    const L sh = ladd(ladd(ladd(ladd(h[0], h[1]), ladd(h[2], h[3])), ladd(ladd(h[4], h[5]), ladd(h[6], h[7]))), h[8]);
    s.th = lmul(ladd(sh, lbc(z, 0.5f * k.Q)), lbc(z, k.inv_sigma));
    s.T = ladd(lbc(z, k.T0), s.th);
    const L a13 = ladd(f[1], f[3]), a24 = ladd(f[2], f[4]);
    const L s57 = ladd(f[5], f[7]), s68 = ladd(f[6], f[8]);
    const L d58 = ladd(s57, s68);
    const L sf = ladd(ladd(a13, a24), d58);
    const L d57 = lsub(f[5], f[7]);
    const L mx = ladd(ladd(lsub(f[1], f[3]), d57), lsub(f[8], f[6]));
    const L my = ladd(ladd(lsub(f[2], f[4]), d57), lsub(f[6], f[8]));
    const L Pxx = ladd(a13, d58), Pyy = ladd(a24, d58);
    const L Pxy = lsub(s57, s68);
    const L Gy = lfma(lbc(z, k.gbeta), s.th, lbc(z, row_ay(k, y)));
    const L vx = lfma(mx, lbc(z, k.inv_rho0), lbc(z, k.half_eps_ax));
    const L vy = lfma(my, lbc(z, k.inv_rho0), lmul(lbc(z, k.half_eps), Gy));
    const L vmag = lsqrt(lfma(vx, vx, lmul(vy, vy)));
    const L iden = lrcp(ladd(lbc(z, k.c0), lsqrt(lfma(lbc(z, k.c1), vmag, lbc(z, k.c0sq)))));
    s.ux = lmul(vx, iden);
    s.uy = lmul(vy, iden);
    if (!isfinite(lsum(ladd(ladd(s.th, s.ux), s.uy)))) atomicOr(k.flag, 1);
    s.uu = lfma(s.ux, s.ux, lmul(s.uy, s.uy));
    // |u| = |v| / (c0 + sqrt(c0^2 + c1 |v|)): no second square root
    const L drag = lfma(lbc(z, k.e_FK), lmul(vmag, iden), lbc(z, k.e_nuK));
    s.Fx = lsub(lbc(z, k.eps * k.ax), lmul(drag, s.ux));
    s.Fy = lsub(lmul(lbc(z, k.eps), Gy), lmul(drag, s.uy));
    s.uF = lfma(s.ux, s.Fx, lmul(s.uy, s.Fy));
    const L p = lsub(lmul(lbc(z, k.p_pref), sf), lfma(lbc(z, k.p_uF), s.uF, lmul(lbc(z, k.p_uu), s.uu)));
    s.ep = lmul(lbc(z, k.eps), p);
    const L re = lbc(z, k.rho0 * k.inv_eps);
    const L invD = lbc(z, k.invD);
    s.Sxx = lmul(lfma(lmul(re, s.ux), lsub(s.Fx, s.ux), lsub(Pxx, s.ep)), invD);
    s.Syy = lmul(lfma(lmul(re, s.uy), lsub(s.Fy, s.uy), lsub(Pyy, s.ep)), invD);
    const L sym = lsub(lmul(lbc(z, 0.5f), lfma(s.ux, s.Fy, lmul(s.Fx, s.uy))), lmul(s.ux, s.uy));
    s.Sxy = lmul(lfma(re, sym, Pxy), invD);
    const L d57h = lsub(h[5], h[7]);
    const L hx = ladd(ladd(lsub(h[1], h[3]), d57h), lsub(h[8], h[6]));
    const L hy = ladd(ladd(lsub(h[2], h[4]), d57h), lsub(h[6], h[8]));
    const L qs = lbc(z, 0.5f * k.Q * k.inv_sigma);
    const L half = lbc(z, 0.5f);
    const L Nx = lfma(s.T, lfma(half, s.Fx, lsub(z, s.ux)), lfma(qs, s.ux, hx));
    const L Ny = lfma(s.T, lfma(half, s.Fy, lsub(z, s.uy)), lfma(qs, s.uy, hy));
    const L a = lfma(lbc(z, -0.5f * k.inv_rho0), s.ep, lbc(z, k.a_const));
    const L d = lfma(lbc(z, -k.bcoef), s.uu, a);
    // one reciprocal for 1/a = d r and 1/d = a r, r = 1/(a d)
    const L r = lrcp(lmul(a, d));
    const L t = lmul(lmul(lbc(z, k.bcoef), lfma(s.ux, Nx, lmul(s.uy, Ny))), lmul(a, r));
    const L ia = lmul(d, r);
    s.gx = lmul(lfma(t, s.ux, Nx), ia);
    s.gy = lmul(lfma(t, s.uy, Ny), ia);
    return s;
}

// Collision at tau_f = tau_T = 1 (f* = f^eq + F_i, g* = g^eq + P_i + Q_i),
// every output multiplied by wscale (the FP16 storage scale folded into the
// weights); the bracket of each pair of opposite directions is split into
// its even and odd parts as in fast_collide.
template <class L>
__device__ __forceinline__ void lane_collide(const KConst<float>& k, const LaneState<L>& s, L* fo, L* ho,
                                             float wscale) {
    const L z = lbc(L(), 0.f);
    const L T = s.T, ep = s.ep, uu = s.uu, ux = s.ux, uy = s.uy, gx = s.gx, gy = s.gy;
    // EF0 = fA_ep ep - fA_uu uu - fA_tr (Sxx + Syy) - fA_uF uF
    const L EF0 = lfma(lbc(z, k.fA_ep), ep,
                       lfma(lbc(z, -k.fA_uu), uu, lfma(lbc(z, -k.fA_tr), ladd(s.Sxx, s.Syy),
                                                       lmul(lbc(z, -k.fA_uF), s.uF))));
    // EH0 = h_sig th - h_uu T uu + h_pT T ep + h_kQ
    const L EH0 = lfma(lbc(z, k.h_sig), s.th,
                       lfma(T, lfma(lbc(z, k.h_pT), ep, lmul(lbc(z, -k.h_uu), uu)), lbc(z, k.h_kQ)));
    const L Kc = lmul(lbc(z, k.h_cu2), T);
    const L Ku = lfma(lbc(z, k.h_u3), T, lfma(lbc(z, k.h_ug), lfma(ux, gx, lmul(uy, gy)), lbc(z, k.h_uQ)));
    const L epr = lmul(ep, lbc(z, k.inv_rho0));
    const L Wx = lfma(T, s.Fx, lmul(epr, gx)), Wy = lfma(T, s.Fy, lmul(epr, gy));
    auto pair = [&](int i, int j, const L& w, const L& cu, const L& cF, const L& ScS, const L& cg, const L& cW) {
        const L cu2 = lmul(cu, cu);
        const L evF = lfma(lbc(z, k.f_cu2), cu2, lfma(lbc(z, k.f_ScS), ScS, lfma(lmul(lbc(z, k.f_cucF), cu), cF, EF0)));
        const L odF = lfma(lbc(z, k.f_cu), cu, lmul(lbc(z, k.f_cF), cF));
        const L evH = lfma(Kc, cu2, EH0);
        const L odH = lfma(Ku, cu, lfma(lbc(z, k.h_g), cg, lmul(lbc(z, k.h_W), cW)));
        fo[i] = lmul(w, ladd(evF, odF));
        fo[j] = lmul(w, lsub(evF, odF));
        ho[i] = lmul(w, ladd(evH, odH));
        ho[j] = lmul(w, lsub(evH, odH));
    };
    const L w1 = lbc(z, wscale * (1.0f / 9.0f)), w5 = lbc(z, wscale * w_diag<float>());
    const L two = lbc(z, 2.f);
    const L Sd = ladd(s.Sxx, s.Syy);
    pair(1, 3, w1, ux, s.Fx, s.Sxx, gx, Wx);
    pair(2, 4, w1, uy, s.Fy, s.Syy, gy, Wy);
    pair(5, 7, w5, ladd(ux, uy), ladd(s.Fx, s.Fy), lfma(two, s.Sxy, Sd), ladd(gx, gy), ladd(Wx, Wy));
    pair(6, 8, w5, lsub(uy, ux), lsub(s.Fy, s.Fx), lfma(lbc(z, -2.f), s.Sxy, Sd), lsub(gy, gx), lsub(Wy, Wx));
    // c0 = h0_sig th - h0_uu T uu - h0_pT T ep + h0_kQ
    const L c0 = lfma(lbc(z, k.h0_sig), s.th,
                      lfma(T, lfma(lbc(z, -k.h0_pT), ep, lmul(lbc(z, -k.h0_uu), uu)), lbc(z, k.h0_kQ)));
    ho[0] = lmul(lbc(z, wscale), c0);
}

}  // namespace lbm
