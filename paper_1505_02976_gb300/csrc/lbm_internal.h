// lbm_internal.h -- launch wrappers shared by the host API and the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// Double-precision constants for the diagnostics (temperatures for the
// Nusselt number are taken in FP64 from the stored populations).
struct DiagConst {
    double T0, inv_sigma, Q, L, dT;
    double T_bc[4];
};

// One time step from src to dst; step seeds the stochastic rounding of FP16
// storage (unused otherwise).
template <class R, class S>
cudaError_t launch_step(const KConst<R>& k, const S* src, S* dst, uint32_t step, cudaStream_t st);

template <class R, class S>
cudaError_t launch_init(const KConst<R>& k, S* dst, const double* T, const double* ux,
                        const double* uy, double T_init, cudaStream_t st);

template <class R, class S>
cudaError_t launch_moments(const KConst<R>& k, const S* src, double* p, double* ux, double* uy,
                           double* T, cudaStream_t st);

template <class R, class S>
cudaError_t launch_get_state(const KConst<R>& k, const S* src, double* f, double* g,
                             double sT0, cudaStream_t st);

template <class R, class S>
cudaError_t launch_set_state(const KConst<R>& k, S* dst, const double* f, const double* g,
                             double sT0, cudaStream_t st);

// Local Nusselt numbers along one side into nu_local, then their trapezoid
// mean into out[0] (deterministic single-block reduction).
template <class R, class S>
cudaError_t launch_nusselt(const KConst<R>& k, const DiagConst& d, const S* src, int side,
                           double* nu_local, double* out, cudaStream_t st);

// Residual sums (|du|, |u|, |dT|, |T|) into out[0..3] against snap (3 planes
// of nx*ny values of the compute type R: ux, uy, T, in a region sized for
// doubles), which is overwritten with the current fields.
// partial must hold 4 doubles per block of the launch (see residual_blocks).
template <class R, class S>
cudaError_t launch_residual(const KConst<R>& k, const S* src, double* snap, double* partial,
                            double* out, cudaStream_t st);

long long residual_blocks(int nx, int ny);

// out[0] = sum over nodes of sum_{i=1..8} f_i, out[1] = sum over nodes of
// sum_{i=0..8} g_i (FP64, fixed order); partial as for launch_residual.
template <class R, class S>
cudaError_t launch_totals(const KConst<R>& k, const S* src, double sT0, double* partial, double* out,
                          cudaStream_t st);

// Stream function psi [ny][nx] from u_x [ny][nx] (psi = 0 along y = 0,
// trapezoid rule up each column); range[0..1] = min, max of psi.
cudaError_t launch_stream_function(const double* ux, int nx, int ny, double* psi, double* range,
                                   cudaStream_t st);

// out[i] = R(in[i]) for i < n.
template <class R>
cudaError_t launch_convert(const double* in, R* out, long long n, cudaStream_t st);

// ---------------------------------------------------------------- batches
// One cavity of a batch: its constants (pitch and plane relative to its own
// planes) and the element offset of its first plane in the batch buffers.
template <class R>
struct BatchCavity {
    KConst<R> k;
    DiagConst d;
    long long offset;
};

// Work item of the batched step.  kind 0: a tile of tile_x x (128/tile_x)
// nodes with origin (a, b) -- its interior nodes only; kind 1: the wall
// nodes a .. a + b - 1 (b <= 128) of the cavity in perimeter order (S row,
// N row, W column, E column, walled sides only).
struct BatchItem {
    int cavity, a, b, kind;
};

// One time step of every cavity: block k of the `grid` blocks takes the
// contiguous work-list range [bounds[k], bounds[k + 1]) (ranges balanced by
// estimated cost on the host); tile_x in {32, 64, 128}.
template <class R, class S>
cudaError_t launch_step_batch(const BatchCavity<R>* cav, const BatchItem* items, const int* bounds,
                              int tile_x, int grid, const S* src, S* dst, uint32_t step,
                              cudaStream_t st);

// Mean Nusselt number of every cavity on one side into out[c].
template <class R, class S>
cudaError_t launch_nusselt_batch(const BatchCavity<R>* cav, int n, const S* src, int side,
                                 double* out, cudaStream_t st);

// --------------------------------------------------- moment state (tau = 1)
// One step of the moment state (9 planes: p, u, S, T - T0, grad T) from src
// to dst; sources = false when src is the state written by launch_init_m
// (equilibria without force and source terms).  segments: row segments per
// band (clamped so that each keeps >= 3 rows).
template <class R>
cudaError_t launch_step_m(const KConst<R>& k, const R* src, R* dst, bool sources, int segments, cudaStream_t st);

// Post-collision populations (17 planes, as the population kernels store
// them) of the moment state src.
template <class R>
cudaError_t launch_expand_m(const KConst<R>& k, const R* src, R* dst, bool sources, cudaStream_t st);

template <class R>
cudaError_t launch_init_m(const KConst<R>& k, R* dst, const double* T, const double* ux, const double* uy,
                          double T_init, cudaStream_t st);

// Row segments per band that fill the GPU's resident blocks once.
template <class R>
int moment_segments_default(const KConst<R>& k);

// ------------------------------------------- step with TMA-staged rows
// Lattices walled on all four sides, FP32 or FP16 storage (S): the tensor
// map of a population buffer (false if the CUDA driver's encoder is unavailable
// or rejects it), the default rows per block segment, and the launch (step
// numbers the FP16 stochastic rounding).
bool tma_step_supported(const KConst<float>& k);
template <class S>
bool make_step_tensor_map(const KConst<float>& k, const S* buf, CUtensorMap* out);
int tma_rows_default(const KConst<float>& k);
template <class S>
cudaError_t launch_step_tma(const KConst<float>& k, const CUtensorMap& tm, const S* src, S* dst, int rows,
                            uint32_t step, cudaStream_t st);
// Work item of the staged batched step: the band of 128 columns from x0 and
// the segment of rows from y0 of a cavity ny rows high.
struct StagedItem {
    int cavity, x0, y0, ny;
};

// Staged step of a batch of FP32 cavities walled on all four sides: one
// block per work item (bands of 128 columns, segments of tma_batch_rows()
// rows; the segments holding wall rows first, each group cavity by cavity);
// maps[c] is cavity c's tensor map of the source buffer.
cudaError_t launch_step_batch_tma(const BatchCavity<float>* cav, const CUtensorMap* maps, const StagedItem* items,
                                  int n_items, const float* src, float* dst, uint32_t step, cudaStream_t st);
int tma_batch_rows();

// Layout of one cavity's items in the persistent work list: items first ..
// first + ns * nb - 1, segment-major (item first + seg * nb + band).
struct PersistCavity {
    int first, nb, ns, pad;
};

// Persistent staged batch step: `nsteps` steps of every cavity in one
// cooperative launch (one block per SM slot), the items ordered as
// PersistCavity describes; maps[buffer * n_cav + c] is cavity c's tensor map
// of buffer `buffer`; done[n_items] and abort_word are scratch of the call
// (reset on the stream before the launch).  buf0/buf1: the two population
// buffers, cur: the one that holds the current state.
cudaError_t launch_step_batch_persist(const BatchCavity<float>* cav, const PersistCavity* pcav, const CUtensorMap* maps,
                                      const StagedItem* items, int n_items, int n_cav, float* buf0, float* buf1,
                                      int cur, uint32_t step0, int nsteps, int* done, int* abort_word, int* flag,
                                      int sms, cudaStream_t st);
// One wait that must give up (nothing arrives): sets bit 1 of *flag.
cudaError_t launch_wait_selftest(int* flag, cudaStream_t st);

// Resident blocks per SM of the batched step kernel.
template <class R, class S>
int batch_blocks_per_sm(int tile_x);

}  // namespace lbm
