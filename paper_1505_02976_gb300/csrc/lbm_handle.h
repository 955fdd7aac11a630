// lbm_handle.h -- the single-lattice handle behind the C ABI (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lbm_host.h"
#include "lbm_internal.h"

struct lbm_handle {
    lbm_params prm;
    lbm_host::Derived d;
    lbm_host::Layout L;
    cudaStream_t stream;
    char* ws;
    bool owns_ws;
    int cur;
    int64_t steps, launches;
    // moment state: current buffer, whether it holds force/source terms (not
    // after set_fields), and whether the expansion in buf(0) is up to date
    int mcur;
    bool msources, pops_valid;
    int msegments;  // row segments per band of the moment step
    // FP32 / FP16 walled lattices: the step with TMA-staged rows (tensor maps
    // of the two population buffers, whether they could be made, whether
    // the step uses them) and its rows per block segment
    bool tma, tma_ready;
    CUtensorMap tmap[2];
    int tma_rows;
    bool nonfinite, timeout;
    lbm::KConst<double> k64;
    lbm::KConst<float> k32;
    lbm::DiagConst diag;
    std::string err;

    void* buf(int i) const { return ws + L.off_buf[i]; }
    void* mom(int i) const { return ws + L.off_mom[i]; }
    bool moments_kind() const { return prm.moment_state != 0; }
    double* fields() const { return (double*)(ws + L.off_fields); }
    double* snap() const { return (double*)(ws + L.off_snap); }
    double* nu() const { return (double*)(ws + L.off_nu); }
    double* partial() const { return (double*)(ws + L.off_partial); }
    double* out() const { return (double*)(ws + L.off_out); }
    int* flag() const { return (int*)(ws + L.off_flag); }
    size_t N() const { return (size_t)prm.nx * prm.ny; }
};

// Record a failure on h (or the thread's create error when h is NULL).
lbm_status lbm_handle_fail(lbm_handle* h, lbm_status s, const std::string& m);
