// lbm_api.cu -- the C ABI declared in include/lbm.h: parameter derivation,
// workspace layout, launches and error handling.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>
#include <new>
#include <type_traits>
#include <string>

#include "../../include/lbm.h"
#include "lbm_handle.h"
#include "lbm_host.h"
#include "lbm_internal.h"

namespace {

using namespace lbm_host;

thread_local std::string g_create_error;

}  // namespace


namespace {

lbm_status fail(lbm_handle* h, lbm_status s, const std::string& m) {
    if (h) h->err = m;
    else g_create_error = m;
    return s;
}

}  // namespace

lbm_status lbm_handle_fail(lbm_handle* h, lbm_status s, const std::string& m) { return fail(h, s, m); }

namespace {

lbm_status cuda_fail(lbm_handle* h, cudaError_t e, const char* what) {
    return fail(h, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(h, call, what)                                   \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, (what)); \
    } while (0)

// Dispatch on the storage precision.
template <class F>
cudaError_t dispatch(lbm_handle* h, F&& fn) {
    switch (h->prm.precision) {
    case LBM_F64: return fn(h->k64, (double*)nullptr);
    case LBM_F32: return fn(h->k32, (float*)nullptr);
    default: return fn(h->k32, (__half*)nullptr);
    }
}

lbm_status copy_in(lbm_handle* h, double* dst, const double* src, int on_device) {
    const size_t bytes = h->N() * sizeof(double);
    LBM_CUDA(h, cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                h->stream), "copy of an input field");
    return LBM_OK;
}

// Where a kernel reads an input field from: a host field in page-locked
// memory is read in place through its device mapping (on this machine the
// GPU reads host memory over the coherent chip-to-chip link, with no staging
// copy); any other host field is copied into the staging area `stage` first,
// and device fields are copied there too.  The caller synchronises before
// returning, so the host array need not outlive the call.
lbm_status field_source(lbm_handle* h, double* stage, const double* src, int on_device, const double** out) {
    if (!on_device) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, src) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer) {
            *out = (const double*)a.devicePointer;
            return LBM_OK;
        }
        (void)cudaGetLastError();  // an unregistered pointer is not an error here
    }
    lbm_status s = copy_in(h, stage, src, on_device);
    if (s != LBM_OK) return s;
    *out = stage;
    return LBM_OK;
}

// Moment state: bring the expansion buffer up to date with the moments (a
// no-op with population storage, or when nothing changed since the last one).
lbm_status ensure_pops(lbm_handle* h) {
    if (!h->moments_kind() || h->pops_valid) return LBM_OK;
    cudaError_t e = h->prm.precision == LBM_F64
                        ? lbm::launch_expand_m(h->k64, (const double*)h->mom(h->mcur), (double*)h->buf(0),
                                               h->msources, h->stream)
                        : lbm::launch_expand_m(h->k32, (const float*)h->mom(h->mcur), (float*)h->buf(0),
                                               h->msources, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "moment expansion");
    h->pops_valid = true;
    return LBM_OK;
}

#define LBM_POPS(h)                                  \
    do {                                             \
        lbm_status s_ = ensure_pops(h);              \
        if (s_ != LBM_OK) return s_;                 \
    } while (0)

// Nodes at the end of a staged step's sweep whose stores ask L2 to keep them
// (evict-last hint; the next step, sweeping the other way, reads those rows
// first).  Where a step writes at most four L2s, every store: the kept rows
// outweigh the halo re-reads the copies then lose from L2 (FP32 2048^2,
// 2.2 L2s: 48.75 vs 48.20 GLUPS, the last half L2 only 48.55).  Larger
// lattices keep only the last half L2 of the sweep (FP32 8192^2: every
// store 49.03 vs 49.46, half an L2 49.40; FP16 8192^2: 90.04 vs 89.89).
// 0 for FP64 (no staged kernel) or if the L2 size is unknown; the hint
// changes no value.
long long l2_hot_nodes(const lbm_params* p) {
    if (p->precision == LBM_F64) return 0;
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    const long long per_node = lbm::NPLANES * (p->precision == LBM_F16 ? 2LL : 4LL);
    const long long nodes = (long long)p->nx * p->ny;
    if (nodes * per_node <= 4LL * l2) return nodes;
    return (long long)l2 / 2 / per_node;
}

lbm_status reset_snapshot(lbm_handle* h) {
    LBM_POPS(h);
    cudaError_t e = dispatch(h, [&](auto& k, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_residual(k, (const S*)h->buf(h->cur), h->snap(), h->partial(), h->out(), h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "residual snapshot");
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_params_default(lbm_params* p) {
    if (!p) return LBM_ERR_ARG;
    memset(p, 0, sizeof(*p));
    p->nx = p->ny = 32;
    p->bc[0] = LBM_BC_DIRICHLET;
    p->bc[1] = LBM_BC_DIRICHLET;
    p->bc[2] = LBM_BC_ADIABATIC;
    p->bc[3] = LBM_BC_ADIABATIC;
    p->forchheimer = 1;
    p->da_infinite = 0;
    p->precision = LBM_F32;
    p->Ra = 1e3; p->Pr = 1.0; p->Da = 1e-2; p->J = 1.0; p->eps = 0.6; p->sigma = 1.0; p->Ma = 0.1;
    p->tau_f = 1.0; p->tau_T = 1.0;
    p->Th = 1.0; p->Tc = 0.0; p->T_init = 0.5; p->rho0 = 1.0; p->Q = 0.0; p->ax = 0.0; p->ay = 0.0;
    p->L = p->nu = p->alpha_e = p->gbeta = p->A = p->B = p->K = p->T0 = NAN;
    p->Ra_I = 0.0;
    p->T_bc[0] = 1.0; p->T_bc[1] = 0.0; p->T_bc[2] = 1.0; p->T_bc[3] = 0.0;
    return LBM_OK;
}

lbm_status lbm_derived(const lbm_params* p, double out[13]) {
    if (!p || !out) return LBM_ERR_ARG;
    Derived d;
    std::string why;
    lbm_status s = derive(p, &d, &why);
    const double v[13] = {d.L, d.T0, d.dT, d.U, d.gbeta, d.nu, d.nu_e, d.alpha_e, d.A, d.B, d.K, d.Feps, d.Q};
    memcpy(out, v, sizeof(v));
    return s;
}

lbm_status lbm_workspace_size(const lbm_params* p, size_t* bytes) {
    if (!p || !bytes) return LBM_ERR_ARG;
    std::string why;
    lbm_status s = check_shape(p, &why);
    if (s != LBM_OK) return fail(nullptr, s, why);
    *bytes = layout(p).total;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_params* p, void* stream, void* workspace, size_t workspace_bytes,
                      lbm_handle** out) {
    if (!p || !out) return fail(nullptr, LBM_ERR_ARG, "null argument");
    *out = nullptr;
    std::string why;
    lbm_status s = check_shape(p, &why);
    if (s != LBM_OK) return fail(nullptr, s, why);
    Derived d;
    s = derive(p, &d, &why);
    if (s != LBM_OK) return fail(nullptr, s, why);
    const Layout L = layout(p);
    if (workspace && (workspace_bytes < L.total || ((uintptr_t)workspace & 255)))
        return fail(nullptr, LBM_ERR_OOM, "workspace too small or not 256-byte aligned");
    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    h->prm = *p;
    h->d = d;
    h->L = L;
    h->stream = (cudaStream_t)stream;
    h->owns_ws = workspace == nullptr;
    h->ws = (char*)workspace;
    if (h->owns_ws) {
        cudaError_t e = cudaMalloc((void**)&h->ws, L.total);
        if (e != cudaSuccess) {
            delete h;
            return fail(nullptr, LBM_ERR_OOM, std::string("cudaMalloc of the workspace: ") + cudaGetErrorString(e));
        }
    }
    h->cur = 0;
    h->steps = h->launches = 0;
    h->nonfinite = false;
    h->timeout = false;
    h->mcur = 0;
    h->msources = false;
    h->pops_valid = false;
    h->k64 = make_kconst<double>(p, d, L, h->flag());
    h->k32 = make_kconst<float>(p, d, L, h->flag());
    h->k32.l2_hot = l2_hot_nodes(p);
    h->tma = h->tma_ready = false;
    h->tma_rows = 0;
    if (p->precision != LBM_F64 && !p->moment_state && lbm::tma_step_supported(h->k32)) {
        if (p->precision == LBM_F32)
            h->tma_ready = lbm::make_step_tensor_map(h->k32, (const float*)h->buf(0), &h->tmap[0]) &&
                           lbm::make_step_tensor_map(h->k32, (const float*)h->buf(1), &h->tmap[1]);
        else
            h->tma_ready = lbm::make_step_tensor_map(h->k32, (const __half*)h->buf(0), &h->tmap[0]) &&
                           lbm::make_step_tensor_map(h->k32, (const __half*)h->buf(1), &h->tmap[1]);
        h->tma = h->tma_ready;
        h->tma_rows = lbm::tma_rows_default(h->k32);
    }
    h->msegments = 1;
    if (p->moment_state)
        h->msegments = p->precision == LBM_F64 ? lbm::moment_segments_default(h->k64)
                                               : lbm::moment_segments_default(h->k32);
    h->diag.T0 = d.T0;
    h->diag.inv_sigma = 1.0 / p->sigma;
    h->diag.Q = d.Q;
    h->diag.L = d.L;
    h->diag.dT = d.dT;
    for (int q = 0; q < 4; ++q) h->diag.T_bc[q] = p->T_bc[q];
    s = LBM_OK;
    for (int g = 0; g < L.n_guards && s == LBM_OK; ++g) {
        const cudaError_t e = cudaMemsetAsync(h->ws + L.guard[g], kGuardByte, kGuardBytes, h->stream);
        if (e != cudaSuccess) s = cuda_fail(h, e, "guard words");
    }
    if (s == LBM_OK) s = lbm_set_fields(h, nullptr, nullptr, nullptr, nullptr, 1);
    if (s != LBM_OK) {
        g_create_error = h->err;
        lbm_destroy(h);
        return s;
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_check_guards(lbm_handle* h) {
    if (!h) return LBM_ERR_ARG;
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "stream synchronise");
    unsigned char w[kGuardBytes];
    for (int g = 0; g < h->L.n_guards; ++g) {
        LBM_CUDA(h, cudaMemcpy(w, h->ws + h->L.guard[g], kGuardBytes, cudaMemcpyDeviceToHost), "guard read");
        for (size_t b = 0; b < kGuardBytes; ++b)
            if (w[b] != kGuardByte)
                return fail(h, LBM_ERR_GUARD,
                            "guard word after workspace region " + std::to_string(g) + " overwritten at byte " +
                                std::to_string(b));
    }
    return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    if (h->owns_ws && h->ws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ws);
    }
    delete h;
}

const char* lbm_last_error(const lbm_handle* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

lbm_status lbm_set_fields(lbm_handle* h, const double* T, const double* ux, const double* uy,
                          const double* eps_field, int on_device) {
    const NvtxRange range("lbm_set_fields");
    if (!h) return LBM_ERR_ARG;
    double* F = h->fields();
    const size_t N = h->N();
    if (eps_field) {
        if (!(h->prm.eps < 1.0))
            return fail(h, LBM_ERR_PARAM_RANGE, "a porosity field needs a reference eps below 1");
        if (!on_device)
            for (size_t i = 0; i < N; ++i)
                if (!(eps_field[i] > 0.0 && eps_field[i] < 1.0))
                    return fail(h, LBM_ERR_PARAM_RANGE, "porosity field values must lie in (0, 1)");
        const double* deps = nullptr;
        lbm_status s0 = field_source(h, F + 3 * N, eps_field, on_device, &deps);
        if (s0 != LBM_OK) return s0;
        char* area = h->ws + h->L.off_eps;
        cudaError_t e = h->prm.precision == LBM_F64
                            ? lbm::launch_convert<double>(deps, (double*)area, (long long)N, h->stream)
                            : lbm::launch_convert<float>(deps, (float*)area, (long long)N, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "porosity field");
        h->k64.eps_field = (const double*)area;
        h->k32.eps_field = (const float*)area;
    } else {
        h->k64.eps_field = nullptr;
        h->k32.eps_field = nullptr;
    }
    const double* dT = nullptr;
    const double* dux = nullptr;
    const double* duy = nullptr;
    lbm_status s;
    if (T && (s = field_source(h, F, T, on_device, &dT)) != LBM_OK) return s;
    if (ux && (s = field_source(h, F + N, ux, on_device, &dux)) != LBM_OK) return s;
    if (uy && (s = field_source(h, F + 2 * N, uy, on_device, &duy)) != LBM_OK) return s;
    h->cur = 0;
    cudaError_t e;
    if (h->moments_kind()) {
        h->mcur = 0;
        h->msources = false;
        h->pops_valid = false;
        e = h->prm.precision == LBM_F64
                ? lbm::launch_init_m(h->k64, (double*)h->mom(0), dT, dux, duy, h->prm.T_init, h->stream)
                : lbm::launch_init_m(h->k32, (float*)h->mom(0), dT, dux, duy, h->prm.T_init, h->stream);
    } else {
        e = dispatch(h, [&](auto& k, auto* tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            return lbm::launch_init(k, (S*)h->buf(0), dT, dux, duy, h->prm.T_init, h->stream);
        });
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "init kernel");
    LBM_CUDA(h, cudaMemsetAsync(h->flag(), 0, sizeof(int), h->stream), "flag reset");
    if ((s = reset_snapshot(h)) != LBM_OK) return s;
    if (!on_device) LBM_CUDA(h, cudaStreamSynchronize(h->stream), "set_fields");
    h->steps = 0;
    h->nonfinite = false;
    h->timeout = false;
    return LBM_OK;
}

lbm_status lbm_step(lbm_handle* h, int64_t n) {
    const NvtxRange range("lbm_step");
    if (!h || n < 0) return h ? fail(h, LBM_ERR_ARG, "negative step count") : LBM_ERR_ARG;
    if (h->timeout) return fail(h, LBM_ERR_TIMEOUT, "a bounded wait of the TMA step gave up");
    if (h->nonfinite) return fail(h, LBM_ERR_NONFINITE, "non-finite velocity or temperature");
    if (h->moments_kind()) {
        for (int64_t i = 0; i < n; ++i) {
            const int src = h->mcur, dst = 1 - h->mcur;
            cudaError_t e = h->prm.precision == LBM_F64
                                ? lbm::launch_step_m(h->k64, (const double*)h->mom(src), (double*)h->mom(dst),
                                                     h->msources, h->msegments, h->stream)
                                : lbm::launch_step_m(h->k32, (const float*)h->mom(src), (float*)h->mom(dst),
                                                     h->msources, h->msegments, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "moment step kernel");
            h->mcur = dst;
            h->msources = true;
            h->pops_valid = false;
            ++h->steps;
            ++h->launches;
        }
        return LBM_OK;
    }
    for (int64_t i = 0; i < n; ++i) {
        const int src = h->cur, dst = 1 - h->cur;
        if (h->tma) {
            const uint32_t step = (uint32_t)h->steps;
            cudaError_t e = h->prm.precision == LBM_F32
                                ? lbm::launch_step_tma(h->k32, h->tmap[src], (const float*)h->buf(src),
                                                       (float*)h->buf(dst), h->tma_rows, step, h->stream)
                                : lbm::launch_step_tma(h->k32, h->tmap[src], (const __half*)h->buf(src),
                                                       (__half*)h->buf(dst), h->tma_rows, step, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "step kernel (TMA)");
            h->cur = dst;
            ++h->steps;
            ++h->launches;
            continue;
        }
        cudaError_t e = dispatch(h, [&](auto& k, auto* tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            return lbm::launch_step(k, (const S*)h->buf(src), (S*)h->buf(dst), (uint32_t)h->steps, h->stream);
        });
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
        h->cur = dst;
        ++h->steps;
        ++h->launches;
    }
    return LBM_OK;
}

lbm_status lbm_set_step_staging(lbm_handle* h, int32_t staged) {
    if (!h) return LBM_ERR_ARG;
    if (staged && !h->tma_ready)
        return fail(h, LBM_ERR_ARG, "staged rows need FP32 or FP16 populations on a lattice walled on all sides");
    h->tma = staged != 0;
    return LBM_OK;
}

int32_t lbm_step_staged(const lbm_handle* h) { return h && h->tma ? 1 : 0; }

lbm_status lbm_set_moment_segments(lbm_handle* h, int32_t segments) {
    if (!h) return LBM_ERR_ARG;
    if (!h->moments_kind() || segments < 0) return fail(h, LBM_ERR_ARG, "not a moment-state handle, or segments < 0");
    if (segments == 0)
        segments = h->prm.precision == LBM_F64 ? lbm::moment_segments_default(h->k64)
                                               : lbm::moment_segments_default(h->k32);
    h->msegments = segments;
    return LBM_OK;
}

lbm_status lbm_sync(lbm_handle* h) {
    if (!h) return LBM_ERR_ARG;
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "stream synchronise");
    int flag = 0;
    LBM_CUDA(h, cudaMemcpy(&flag, h->flag(), sizeof(int), cudaMemcpyDeviceToHost), "flag read");
    if (flag & 2) h->timeout = true;
    if (flag & 1) h->nonfinite = true;
    if (h->timeout) return fail(h, LBM_ERR_TIMEOUT, "a bounded wait of the TMA step gave up");
    if (h->nonfinite) return fail(h, LBM_ERR_NONFINITE, "non-finite velocity or temperature");
    return LBM_OK;
}

lbm_status lbm_wait_selftest(lbm_handle* h) {
    if (!h) return LBM_ERR_ARG;
    cudaError_t e = lbm::launch_wait_selftest(h->flag(), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "wait self-test kernel");
    ++h->launches;
    return LBM_OK;
}

lbm_status lbm_moments(lbm_handle* h, double* p, double* ux, double* uy, double* T, int on_device) {
    const NvtxRange range("lbm_moments");
    if (!h) return LBM_ERR_ARG;
    LBM_POPS(h);
    double* F = h->fields();
    const size_t N = h->N();
    cudaError_t e = dispatch(h, [&](auto& k, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_moments(k, (const S*)h->buf(h->cur), F, F + N, F + 2 * N, F + 3 * N, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    double* outs[4] = {p, ux, uy, T};
    for (int q = 0; q < 4; ++q)
        if (outs[q])
            LBM_CUDA(h, cudaMemcpyAsync(outs[q], F + q * N, N * sizeof(double),
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream),
                     "copy of a moment field");
    if (!on_device) LBM_CUDA(h, cudaStreamSynchronize(h->stream), "moments");
    return LBM_OK;
}

lbm_status lbm_stream_function(lbm_handle* h, double* psi, int on_device, double range[2]) {
    if (!h) return LBM_ERR_ARG;
    LBM_POPS(h);
    double* F = h->fields();
    const size_t N = h->N();
    cudaError_t e = dispatch(h, [&](auto& k, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_moments(k, (const S*)h->buf(h->cur), F, F + N, F + 2 * N, F + 3 * N, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    // psi overwrites the pressure plane of the staging area
    e = lbm::launch_stream_function(F + N, h->prm.nx, h->prm.ny, F, h->out(), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream function kernels");
    if (psi)
        LBM_CUDA(h, cudaMemcpyAsync(psi, F, N * sizeof(double),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream),
                 "copy of the stream function");
    if (range)
        LBM_CUDA(h, cudaMemcpyAsync(range, h->out(), 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                 "copy of the stream function range");
    if (!on_device || range) LBM_CUDA(h, cudaStreamSynchronize(h->stream), "stream function");
    return LBM_OK;
}

lbm_status lbm_nusselt(lbm_handle* h, int side, double* nu_mean, double* nu_local) {
    const NvtxRange range("lbm_nusselt");
    if (!h) return LBM_ERR_ARG;
    if (side < 0 || side > 3 || !nu_mean) return fail(h, LBM_ERR_ARG, "bad side or null output");
    const int n = side <= 1 ? h->prm.ny : h->prm.nx;
    const int across = side <= 1 ? h->prm.nx : h->prm.ny;
    if (across < 3) return fail(h, LBM_ERR_ARG, "the one-sided difference needs 3 nodes");
    LBM_POPS(h);
    cudaError_t e = dispatch(h, [&](auto& k, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_nusselt(k, h->diag, (const S*)h->buf(h->cur), side, h->nu(), h->out(), h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "nusselt kernels");
    LBM_CUDA(h, cudaMemcpyAsync(nu_mean, h->out(), sizeof(double), cudaMemcpyDeviceToHost, h->stream), "nusselt copy");
    if (nu_local)
        LBM_CUDA(h, cudaMemcpyAsync(nu_local, h->nu(), n * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                 "nusselt copy");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "nusselt");
    return LBM_OK;
}

lbm_status lbm_residual(lbm_handle* h, double* res_u, double* res_T) {
    const NvtxRange range("lbm_residual");
    if (!h || !res_u || !res_T) return h ? fail(h, LBM_ERR_ARG, "null output") : LBM_ERR_ARG;
    lbm_status s = reset_snapshot(h);
    if (s != LBM_OK) return s;
    double v[4];
    LBM_CUDA(h, cudaMemcpyAsync(v, h->out(), sizeof(v), cudaMemcpyDeviceToHost, h->stream), "residual copy");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "residual");
    *res_u = v[0] / v[1];
    *res_T = v[2] / v[3];
    return LBM_OK;
}

lbm_status lbm_get_state(lbm_handle* h, double* f, double* g, int on_device) {
    if (!h || !f || !g) return h ? fail(h, LBM_ERR_ARG, "null output") : LBM_ERR_ARG;
    LBM_POPS(h);
    const size_t bytes = 9 * h->N() * sizeof(double);
    double* df = f;
    double* dg = g;
    double* tmp = nullptr;
    if (!on_device) {
        LBM_CUDA(h, cudaMallocAsync((void**)&tmp, 2 * bytes, h->stream), "state staging");
        df = tmp;
        dg = tmp + 9 * h->N();
    }
    cudaError_t e = dispatch(h, [&](auto& k, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_get_state(k, (const S*)h->buf(h->cur), df, dg, h->prm.sigma * h->d.T0, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "get_state kernel");
    if (!on_device) {
        LBM_CUDA(h, cudaMemcpyAsync(f, df, bytes, cudaMemcpyDeviceToHost, h->stream), "state copy");
        LBM_CUDA(h, cudaMemcpyAsync(g, dg, bytes, cudaMemcpyDeviceToHost, h->stream), "state copy");
        LBM_CUDA(h, cudaFreeAsync(tmp, h->stream), "state staging");
        LBM_CUDA(h, cudaStreamSynchronize(h->stream), "get_state");
    }
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_handle* h, const double* f, const double* g, int on_device) {
    if (!h || !f || !g) return h ? fail(h, LBM_ERR_ARG, "null input") : LBM_ERR_ARG;
    if (h->moments_kind())
        return fail(h, LBM_ERR_ARG, "set_state needs population storage (a moment state holds no arbitrary populations)");
    const size_t bytes = 9 * h->N() * sizeof(double);
    const double* df = f;
    const double* dg = g;
    double* tmp = nullptr;
    if (!on_device) {
        LBM_CUDA(h, cudaMallocAsync((void**)&tmp, 2 * bytes, h->stream), "state staging");
        LBM_CUDA(h, cudaMemcpyAsync(tmp, f, bytes, cudaMemcpyHostToDevice, h->stream), "state copy");
        LBM_CUDA(h, cudaMemcpyAsync(tmp + 9 * h->N(), g, bytes, cudaMemcpyHostToDevice, h->stream), "state copy");
        df = tmp;
        dg = tmp + 9 * h->N();
    }
    cudaError_t e = dispatch(h, [&](auto& k, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_set_state(k, (S*)h->buf(h->cur), df, dg, h->prm.sigma * h->d.T0, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state kernel");
    LBM_CUDA(h, cudaMemsetAsync(h->flag(), 0, sizeof(int), h->stream), "flag reset");
    if (!on_device) {
        LBM_CUDA(h, cudaFreeAsync(tmp, h->stream), "state staging");
        LBM_CUDA(h, cudaStreamSynchronize(h->stream), "set_state");
    }
    h->nonfinite = false;
    h->timeout = false;
    return LBM_OK;
}

lbm_status lbm_set_force_profile(lbm_handle* h, const double* ay) {
    if (!h) return LBM_ERR_ARG;
    if (!ay) {
        h->k64.ay_row = nullptr;
        h->k32.ay_row = nullptr;
        h->pops_valid = false;
        return LBM_OK;
    }
    const int ny = h->prm.ny;
    h->pops_valid = false;
    char* area = h->ws + h->L.off_ay;
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "stream synchronise");
    if (h->prm.precision == LBM_F64) {
        LBM_CUDA(h, cudaMemcpy(area, ay, ny * sizeof(double), cudaMemcpyHostToDevice), "force profile");
        h->k64.ay_row = (const double*)area;
    } else {
        std::vector<float> v(ay, ay + ny);
        LBM_CUDA(h, cudaMemcpy(area, v.data(), ny * sizeof(float), cudaMemcpyHostToDevice), "force profile");
        h->k32.ay_row = (const float*)area;
    }
    return LBM_OK;
}

lbm_status lbm_totals(lbm_handle* h, double* sum_f, double* sum_g) {
    if (!h || !sum_f || !sum_g) return h ? fail(h, LBM_ERR_ARG, "null output") : LBM_ERR_ARG;
    LBM_POPS(h);
    cudaError_t e = dispatch(h, [&](auto& k, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_totals(k, (const S*)h->buf(h->cur), h->prm.sigma * h->d.T0, h->partial(), h->out(),
                                  h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "totals kernels");
    double v[4];
    LBM_CUDA(h, cudaMemcpyAsync(v, h->out(), sizeof(v), cudaMemcpyDeviceToHost, h->stream), "totals copy");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "totals");
    *sum_f = v[0];
    *sum_g = v[1];
    return LBM_OK;
}

}  // extern "C"

namespace {

// CRC-32 (IEEE 802.3 polynomial, reflected, as in zlib), table driven.
uint32_t crc32_update(uint32_t crc, const unsigned char* p, size_t n) {
    static uint32_t table[256];
    static bool ready = false;
    if (!ready) {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : (c >> 1);
            table[i] = c;
        }
        ready = true;
    }
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return ~crc;
}

// FNV-1a over the problem statement, identifying the run a file belongs to.
uint64_t params_hash(const lbm_params& p) {
    const unsigned char* b = (const unsigned char*)&p;
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < sizeof(p); ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

struct CkptHeader {
    char magic[8];          // "LBMCKPT1"
    uint32_t version;       // 2
    int32_t precision;
    int32_t nx, ny, pitch, has_eps;
    int64_t steps;
    uint64_t params_hash;
    uint64_t payload_bytes; // state planes (17 populations or 9 moments) then the porosity field
    int32_t state_kind;     // 0 populations, 1 moments
    int32_t sources;        // moments: 1 once a step has run (0 right after set_fields)
};

}  // namespace

extern "C" {

lbm_status lbm_checkpoint(lbm_handle* h, const char* path, int save) {
    const NvtxRange range("lbm_checkpoint");
    if (!h || !path) return h ? fail(h, LBM_ERR_ARG, "null path") : LBM_ERR_ARG;
    const size_t es = elem_size(h->prm.precision);
    const bool mk = h->moments_kind();
    const size_t pop_bytes = h->L.plane_elems * es * (mk ? lbm::kMPlanes : lbm::NPLANES);
    void* state = mk ? h->mom(h->mcur) : h->buf(h->cur);
    const size_t eps_es = h->prm.precision == LBM_F64 ? 8 : 4;
    const void* eps_dev = h->prm.precision == LBM_F64 ? (const void*)h->k64.eps_field : (const void*)h->k32.eps_field;
    if (save) {
        lbm_status s = lbm_sync(h);
        if (s != LBM_OK) return s;
        const size_t eps_bytes = eps_dev ? h->N() * eps_es : 0;
        std::string payload(pop_bytes + eps_bytes, '\0');
        LBM_CUDA(h, cudaMemcpy(&payload[0], state, pop_bytes, cudaMemcpyDeviceToHost), "state read");
        if (eps_dev)
            LBM_CUDA(h, cudaMemcpy(&payload[pop_bytes], eps_dev, eps_bytes, cudaMemcpyDeviceToHost), "field read");
        CkptHeader hd;
        memset(&hd, 0, sizeof(hd));
        memcpy(hd.magic, "LBMCKPT1", 8);
        hd.version = 2;
        hd.state_kind = mk ? 1 : 0;
        hd.sources = mk ? (h->msources ? 1 : 0) : 1;
        hd.precision = h->prm.precision;
        hd.nx = h->prm.nx;
        hd.ny = h->prm.ny;
        hd.pitch = h->L.pitch;
        hd.has_eps = eps_dev ? 1 : 0;
        hd.steps = h->steps;
        hd.params_hash = params_hash(h->prm);
        hd.payload_bytes = payload.size();
        const uint32_t crc = crc32_update(0, (const unsigned char*)payload.data(), payload.size());
        FILE* f = fopen(path, "wb");
        if (!f) return fail(h, LBM_ERR_ARG, std::string("cannot open ") + path + " for writing");
        bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(payload.data(), 1, payload.size(), f) == payload.size() &&
                  fwrite(&crc, sizeof(crc), 1, f) == 1;
        ok = (fclose(f) == 0) && ok;
        if (!ok) return fail(h, LBM_ERR_ARG, std::string("write failed: ") + path);
        return LBM_OK;
    }
    FILE* f = fopen(path, "rb");
    if (!f) return fail(h, LBM_ERR_ARG, std::string("cannot open ") + path);
    CkptHeader hd;
    if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, "LBMCKPT1", 8) != 0 || hd.version != 2) {
        fclose(f);
        return fail(h, LBM_ERR_ARG, "not a checkpoint of this library");
    }
    if (hd.precision != h->prm.precision || hd.nx != h->prm.nx || hd.ny != h->prm.ny || hd.pitch != h->L.pitch ||
        hd.params_hash != params_hash(h->prm) || hd.state_kind != (mk ? 1 : 0)) {
        fclose(f);
        return fail(h, LBM_ERR_ARG, "checkpoint belongs to a different problem or precision");
    }
    const size_t expect = pop_bytes + (hd.has_eps ? h->N() * eps_es : 0);
    if (hd.payload_bytes != expect) {
        fclose(f);
        return fail(h, LBM_ERR_ARG, "checkpoint payload has the wrong size");
    }
    std::string payload(expect, '\0');
    uint32_t crc = 0;
    const bool ok = fread(&payload[0], 1, expect, f) == expect && fread(&crc, sizeof(crc), 1, f) == 1;
    fclose(f);
    if (!ok) return fail(h, LBM_ERR_ARG, "checkpoint truncated");
    if (crc32_update(0, (const unsigned char*)payload.data(), payload.size()) != crc)
        return fail(h, LBM_ERR_ARG, "checkpoint corrupted (CRC-32 mismatch)");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "stream synchronise");
    LBM_CUDA(h, cudaMemcpy(state, payload.data(), pop_bytes, cudaMemcpyHostToDevice), "state write");
    if (mk) {
        h->msources = hd.sources != 0;
        h->pops_valid = false;
    }
    if (hd.has_eps) {
        char* area = h->ws + h->L.off_eps;
        LBM_CUDA(h, cudaMemcpy(area, payload.data() + pop_bytes, h->N() * eps_es, cudaMemcpyHostToDevice), "field write");
        h->k64.eps_field = (const double*)area;
        h->k32.eps_field = (const float*)area;
    } else {
        h->k64.eps_field = nullptr;
        h->k32.eps_field = nullptr;
    }
    LBM_CUDA(h, cudaMemset(h->flag(), 0, sizeof(int)), "flag reset");
    h->steps = hd.steps;
    h->nonfinite = false;
    h->timeout = false;
    // the residual snapshot is not part of the file: the restored state
    // becomes the reference of the next lbm_residual
    lbm_status s = reset_snapshot(h);
    if (s != LBM_OK) return s;
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "residual snapshot of the restored state");
    return LBM_OK;
}

int64_t lbm_steps_done(const lbm_handle* h) { return h ? h->steps : -1; }

int64_t lbm_kernel_launches(const lbm_handle* h) { return h ? h->launches : -1; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Mean Nusselt number without any allocation (lbm_nusselt_noalloc).
//
// Some programs cannot let a library call cudaMalloc: a host application that
// reserves its whole device-memory budget at start-up and hands out slices
// of it, a plugin that must not grow the memory footprint of the process that
// loads it, or a loop that cannot afford the device-wide synchronisation a
// cudaMalloc/cudaFree implies.  Such a caller creates the handle on a
// workspace of its own (lbm_create with a non-NULL workspace) and reads the
// wall's mean Nusselt number with lbm_nusselt_noalloc, which keeps the
// per-node values in the fixed array below instead of in the workspace.
//
// The array is compiled into the library: every GPU that loads the library
// holds it until the process exits.  Its largest wall is kNoAllocMaxNodes
// nodes; one slot after them holds the mean.  Nothing in it needs to start at
// zero: each call writes all the per-node values it reads and the mean.  All
// calls share it and it keeps the last call's values, so two calls whose GPU
// work overlaps (different streams, or different handles on one device)
// race on it.
static constexpr int kNoAllocMaxNodes = 65536;
static __device__ __align__(256) double g_nu_scratch[kNoAllocMaxNodes + 32];

namespace {
// Device address of the scratch array on `device`, looked up on every call
// with that device current (the lookup is cheap, and nothing is cached that
// a device reset could leave stale).  In host code g_nu_scratch names a
// host-side stand-in, not device memory; only this address may be given to
// a kernel.
lbm_status nu_scratch_on(lbm_handle* h, int device, double** out) {
    int prev = -1;
    LBM_CUDA(h, cudaGetDevice(&prev), "current device");
    if (prev != device) LBM_CUDA(h, cudaSetDevice(device), "select the stream's device");
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_nu_scratch);
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(h, e, "address of the static Nusselt scratch");
    *out = (double*)p;
    return LBM_OK;
}
}  // namespace

extern "C" lbm_status lbm_nusselt_noalloc(lbm_handle* h, int side, double* nu_mean) {
    if (!h) return LBM_ERR_ARG;
    if (side < 0 || side > 3 || !nu_mean) return fail(h, LBM_ERR_ARG, "bad side or null output");
    const int n = side <= 1 ? h->prm.ny : h->prm.nx;
    const int across = side <= 1 ? h->prm.nx : h->prm.ny;
    if (across < 3) return fail(h, LBM_ERR_ARG, "the one-sided difference needs 3 nodes");
    LBM_POPS(h);
    if (n > kNoAllocMaxNodes)
        return fail(h, LBM_ERR_ARG,
                    "wall longer than the 65536 nodes the static scratch of lbm_nusselt_noalloc holds");
    int device = 0;
    LBM_CUDA(h, cudaStreamGetDevice(h->stream, &device), "device of the handle's stream");
    double* scratch = nullptr;
    lbm_status s = nu_scratch_on(h, device, &scratch);
    if (s != LBM_OK) return s;
    double* mean = scratch + kNoAllocMaxNodes;
    cudaError_t e = dispatch(h, [&](auto& k, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_nusselt(k, h->diag, (const S*)h->buf(h->cur), side, scratch, mean, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "nusselt kernels");
    LBM_CUDA(h, cudaMemcpyAsync(nu_mean, mean, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
             "nusselt copy");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "nusselt");
    return LBM_OK;
}
