// lbm_host.h -- host-side helpers shared by the C ABI entry points:
// parameter derivation and checks, workspace layout, kernel constants.
#pragma once

#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbm_host {

constexpr double kCs2 = 1.0 / 3.0;
constexpr double kW0 = 4.0 / 9.0;
constexpr int NPLANES_HOST = lbm::NPLANES;

struct Derived {
    double L, T0, dT, U, gbeta, nu, nu_e, alpha_e, A, B, K, Feps, Q;
};

inline bool isnan_(double v) { return v != v; }

// Lattice constants from the problem statement (Sec. 2, Sec. 4, Eq. EQA&B,
// Eq. Therdiff, Appendix A): see the table in include/lbm.h.
inline lbm_status derive(const lbm_params* p, Derived* d, std::string* why) {
    d->L = isnan_(p->L) ? double(p->nx - 1) : p->L;
    d->T0 = isnan_(p->T0) ? 0.5 * (p->Th + p->Tc) : p->T0;
    d->dT = p->Th - p->Tc;
    d->U = p->Ma * sqrt(kCs2);
    d->gbeta = isnan_(p->gbeta) ? d->U * d->U / (d->dT * d->L) : p->gbeta;
    if (!isnan_(p->nu)) d->nu = p->nu;
    else if (!isnan_(p->A)) d->nu = kCs2 * (p->tau_f - p->A - 0.5) / p->J;
    else d->nu = d->U * d->L * sqrt(p->Pr / p->Ra);
    d->nu_e = p->J * d->nu;
    if (!isnan_(p->alpha_e)) d->alpha_e = p->alpha_e;
    else if (!isnan_(p->B)) d->alpha_e = p->sigma * kCs2 * (p->tau_T - p->B - 0.5);
    else d->alpha_e = d->nu / p->Pr;
    d->A = isnan_(p->A) ? p->tau_f - 0.5 - d->nu_e / kCs2 : p->A;
    d->B = isnan_(p->B) ? p->tau_T - 0.5 - d->alpha_e / (p->sigma * kCs2) : p->B;
    d->K = p->da_infinite ? INFINITY : (isnan_(p->K) ? p->Da * d->L * d->L : p->K);
    d->Feps = p->forchheimer ? 1.75 / sqrt(150.0 * p->eps * p->eps * p->eps) : 0.0;
    d->Q = isnan_(p->Q) ? p->Ra_I * d->alpha_e * d->dT / (p->Ra * d->L * d->L) : p->Q;
    auto bad = [&](const char* m) {
        if (why) *why = m;
        return LBM_ERR_PARAM_RANGE;
    };
    if (!(p->eps > 0.0 && p->eps <= 1.0)) return bad("porosity eps must lie in (0, 1]");
    if (!(p->tau_f > 0.5 && p->tau_T > 0.5)) return bad("relaxation times must exceed 1/2");
    if (!(d->A < p->tau_f - 0.5)) return bad("A must be below tau_f - 1/2 (positive viscosity)");
    if (!(d->B < p->tau_T - 0.5)) return bad("B must be below tau_T - 1/2 (positive diffusivity)");
    if (!(p->sigma > 0.0 && p->rho0 > 0.0)) return bad("sigma and rho0 must be positive");
    if (!(isfinite(d->gbeta) && isfinite(d->nu) && isfinite(d->alpha_e) && isfinite(d->T0) &&
          isfinite(d->Q)))
        return bad("derived constants are not finite (check Ra, Ra_I, Pr, Ma, Th - Tc)");
    return LBM_OK;
}

inline lbm_status check_shape(const lbm_params* p, std::string* why) {
    for (int s = 0; s < 4; ++s)
        if (p->bc[s] < 0 || p->bc[s] > 2) { *why = "unknown boundary kind"; return LBM_ERR_ARG; }
    if ((p->bc[0] == LBM_BC_PERIODIC) != (p->bc[1] == LBM_BC_PERIODIC) ||
        (p->bc[2] == LBM_BC_PERIODIC) != (p->bc[3] == LBM_BC_PERIODIC)) {
        *why = "a periodic side needs a periodic opposite side";
        return LBM_ERR_ARG;
    }
    if (p->nx < 1 || p->ny < 1 || p->ny > 65535 || p->nx > (1 << 24)) {
        *why = "lattice size out of range (1 <= nx, 1 <= ny <= 65535)";
        return LBM_ERR_ARG;
    }
    if ((p->bc[0] != LBM_BC_PERIODIC && p->nx < 4) || (p->bc[2] != LBM_BC_PERIODIC && p->ny < 4)) {
        *why = "a walled direction needs at least 4 nodes";
        return LBM_ERR_ARG;
    }
    if ((double)NPLANES_HOST * (double)((size_t)p->nx + 128) * (double)p->ny >= 2147483647.0) {
        *why = "lattice too large for 32-bit plane offsets (17 nx ny < 2^31)";
        return LBM_ERR_ARG;
    }
    if (p->precision < LBM_F64 || p->precision > LBM_F16 || p->moment_state < 0 || p->moment_state > 1) {
        *why = "unknown precision or state kind";
        return LBM_ERR_ARG;
    }
    if (p->moment_state && !(p->tau_f == 1.0 && p->tau_T == 1.0 && p->precision != LBM_F16)) {
        *why = "moment storage needs tau_f = tau_T = 1 and FP32 or FP64";
        return LBM_ERR_ARG;
    }
    return LBM_OK;
}

inline size_t elem_size(int precision) {
    return precision == LBM_F64 ? 8 : (precision == LBM_F32 ? 4 : 2);
}

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// NVTX range over one entry point (visible to Nsight tools; a no-op
// otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Guard words: kGuardBytes of kGuardByte after every region of a workspace,
// written at creation and compared on request (lbm_check_guards), so that a
// kernel writing past the end of any region is detected.
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
constexpr int kMaxGuards = 32;

struct Layout {
    int pitch;
    size_t plane_elems, buf_bytes;
    size_t off_buf[2], off_fields, off_snap, off_nu, off_partial, off_eps, off_ay, off_out, off_flag, total;
    size_t off_mom[2], mom_bytes;  // moment state: two 9-plane buffers; off_buf[0] = off_buf[1] = expansion
    size_t guard[kMaxGuards];      // offsets of the guard words
    int n_guards;
};

inline Layout layout(const lbm_params* p) {
    Layout L;
    const size_t es = elem_size(p->precision);
    const size_t row = ((size_t)p->nx * es + 127) / 128 * 128;  // 128-byte rows
    L.pitch = int(row / es);
    L.plane_elems = (size_t)L.pitch * p->ny;
    L.buf_bytes = align256(L.plane_elems * es * lbm::NPLANES);
    const size_t N = (size_t)p->nx * p->ny;
    size_t o = 0;
    L.n_guards = 0;
    // each region is followed by a guard word
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        L.guard[L.n_guards++] = o;
        o += kGuardBytes;
        return at;
    };
    L.off_buf[0] = take(L.buf_bytes);
    if (p->moment_state) {
        L.off_buf[1] = L.off_buf[0];
        L.mom_bytes = align256(L.plane_elems * es * lbm::kMPlanes);
        L.off_mom[0] = take(L.mom_bytes);
        L.off_mom[1] = take(L.mom_bytes);
    } else {
        L.off_buf[1] = take(L.buf_bytes);
        L.mom_bytes = 0;
        L.off_mom[0] = L.off_mom[1] = 0;
    }
    L.off_fields = take(4 * N * sizeof(double));
    L.off_snap = take(3 * N * sizeof(double));
    L.off_nu = take((size_t)(p->nx > p->ny ? p->nx : p->ny) * sizeof(double));
    L.off_partial = take((size_t)lbm::residual_blocks(p->nx, p->ny) * 4 * sizeof(double));
    L.off_eps = take(N * sizeof(double));
    L.off_ay = take((size_t)p->ny * sizeof(double));
    L.off_out = take(256);
    L.off_flag = take(256);
    L.total = o;
    return L;
}

template <class R>
inline lbm::KConst<R> make_kconst(const lbm_params* p, const Derived& d, const Layout& L, int* flag) {
    lbm::KConst<R> k;
    memset(&k, 0, sizeof(k));
    k.nx = p->nx;
    k.ny = p->ny;
    k.pitch = L.pitch;
    for (int s = 0; s < 4; ++s) k.bc[s] = p->bc[s];
    k.plane = (long long)L.plane_elems;
    const double eps = p->eps;
    const double nuK = isinf(d.K) ? 0.0 : d.nu / d.K;
    const double FK = isinf(d.K) ? 0.0 : d.Feps / sqrt(d.K);
    const double c0 = 0.5 * (1.0 + eps * 0.5 * nuK);
    const double c1 = eps * 0.5 * FK;
    k.rho0 = R(p->rho0);
    k.eps = R(eps);
    k.inv_eps = R(1.0 / eps);
    k.sigma = R(p->sigma);
    k.inv_sigma = R(1.0 / p->sigma);
    k.omf = R(1.0 - 1.0 / p->tau_f);
    k.omT = R(1.0 - 1.0 / p->tau_T);
    k.tau_f = R(p->tau_f);
    k.kf = R(1.0 - 0.5 / p->tau_f);
    k.kT = R(1.0 - 0.5 / p->tau_T);
    k.A = R(d.A);
    k.B = R(d.B);
    k.T0 = R(d.T0);
    k.gbeta = R(d.gbeta);
    k.ax = R(p->ax);
    k.ay = R(p->ay);
    k.Q = R(d.Q);
    k.e_nuK = R(eps * nuK);
    k.e_FK = R(eps * FK);
    k.c0 = R(c0);
    k.c0sq = R(c0 * c0);
    k.c1 = R(c1);
    k.p_pref = R(kCs2 / (eps * (1.0 - kW0)));
    k.invD = R(1.0 / (kCs2 * p->rho0 * (d.A - p->tau_f)));
    k.a_const = R(kCs2 * p->sigma * (d.B - p->tau_T));
    k.bcoef = R(0.5 * (1.0 / eps - 1.0 / p->sigma));
    k.sT0 = R(p->sigma * d.T0);
    for (int s = 0; s < 4; ++s) {
        k.T_bc[s] = R(p->T_bc[s]);
        k.u_bc[s][0] = R(p->u_bc[s][0]);
        k.u_bc[s][1] = R(p->u_bc[s][1]);
    }
    k.scale = p->precision == LBM_F16 ? ldexpf(1.0f, -10) : 1.0f;
    k.inv_scale = 1.0f / k.scale;
    k.flag = flag;
    k.plane32 = (int)L.plane_elems;
    // interior fast path: h* = (1 - 1/tau) h + [h^eq / tau + source], split
    // into parts even and odd in c_i (lbm_device.cuh, interior_update)
    const double rho0 = p->rho0, ie = 1.0 / eps, itf = 1.0 / p->tau_f, itT = 1.0 / p->tau_T;
    const double kf = 1.0 - 0.5 / p->tau_f, kT = 1.0 - 0.5 / p->tau_T;
    const double bc = 0.5 * (1.0 / eps - 1.0 / p->sigma);
    k.inv_rho0 = R(1.0 / rho0);
    k.half_eps_ax = R(0.5 * eps * p->ax);
    k.half_eps = R(0.5 * eps);
    k.p_uF = R(kCs2 / (eps * (1.0 - kW0)) * (4.0 / 3.0) * rho0 * kf * p->tau_f * ie);
    k.p_uu = R(kCs2 / (eps * (1.0 - kW0)) * (2.0 / 3.0) * rho0 * ie);
    k.fA_ep = R(3.0 * itf);
    k.fA_uu = R(1.5 * itf * rho0 * ie);
    k.fA_tr = R(0.5 * itf * rho0 * d.A);
    k.fA_uF = R(3.0 * rho0 * kf * ie);
    k.f_cu2 = R(4.5 * itf * rho0 * ie);
    k.f_ScS = R(1.5 * itf * rho0 * d.A);
    k.f_cucF = R(9.0 * rho0 * kf * ie);
    k.f_cu = R(3.0 * rho0 * itf);
    k.f_cF = R(3.0 * rho0 * kf);
    k.h_sig = R(itT * p->sigma);
    k.h_uu = R(itT * 1.5 * ie);
    k.h_pT = R(itT * 3.0 / rho0);
    k.h_kQ = R(kT * d.Q);
    k.h_cu2 = R(itT * 4.5 * ie);
    k.h_u3 = R(3.0 * itT);
    k.h_ug = R(6.0 * kT * bc);
    k.h_uQ = R(3.0 * kT * d.Q / p->sigma);
    k.h_g = R(itT * p->sigma * d.B);
    k.h_W = R(3.0 * kT);
    k.h0_sig = R(itT * kW0 * p->sigma);
    k.h0_uu = R(itT * kW0 * 1.5 * ie);
    k.h0_pT = R(itT * (5.0 / 3.0) / rho0);
    k.h0_kQ = R(kW0 * kT * d.Q);
    // porosity field support (the field pointer is set by lbm_set_fields)
    k.eps_field = nullptr;
    k.kc_inv_ref = R(eps < 1.0 ? (1.0 - eps) * (1.0 - eps) / (eps * eps * eps) : 0.0);
    k.nu_over_Kref = R(nuK);
    k.inv_sqrt_Kref = R(isinf(d.K) ? 0.0 : 1.0 / sqrt(d.K));
    k.p_pref_eps = R(kCs2 / (1.0 - kW0));
    k.da_inf = p->da_infinite ? 1 : 0;
    k.forch = p->forchheimer ? 1 : 0;
    k.ay_row = nullptr;
    return k;
}


}  // namespace lbm_host
