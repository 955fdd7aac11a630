// lbm_batch.cu -- the batch entry points of include/lbm.h: many independent
// cavities of different size and parameters advanced together.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "lbm_host.h"
#include "lbm_internal.h"

using namespace lbm_host;

namespace {

thread_local std::string g_batch_create_error;
constexpr int kTiles[3] = {32, 64, 128};
constexpr int kGraphChunk = 50;  // steps per captured graph (even: the ping-pong parity returns)
constexpr int kMaxGrid = 1 << 16;
constexpr double kWallCost = 4.0;  // a packed wall node costs about 4 interior nodes (out-of-line path)

}  // namespace

struct lbm_batch {
    int n;
    int precision;
    cudaStream_t stream;
    char* ws;
    bool owns_ws;
    size_t ws_bytes;
    std::vector<lbm_params> prm;
    std::vector<lbm::BatchCavity<double>> cav64;
    std::vector<lbm::BatchCavity<float>> cav32;
    std::vector<long long> offset;     // element offset of each cavity's planes
    size_t buf_elems;                  // elements per population buffer
    size_t max_cells;
    size_t off_buf[2], off_cav, off_items[3], off_bounds, off_fields, off_nu, off_flag;
    int n_items[3];
    std::vector<double> cum[3];        // cumulative estimated cost of the work lists
    int bounds_tile, bounds_grid;      // launch shape the uploaded block ranges belong to
    int cur;
    int tile_x, grid;                  // chosen launch shape
    int sms;
    int64_t steps, launches;
    bool nonfinite, timeout;
    // FP32 batches of cavities walled on all four sides: the staged kernel
    // (one block per 128-column x 4-row item), its work list and the tensor
    // maps of every cavity in both buffers (device: maps[buffer * n + c])
    bool staged, staged_ready;
    size_t off_maps, off_sitems;
    // the persistent form of the staged step: its work list (cavity by
    // cavity, segment-major), the per-cavity layout of that list, and the
    // per-item step counters and abort word of a call
    size_t off_pitems, off_pcav, off_done;
    std::vector<size_t> guards;        // offsets of the guard words after each region
    int n_sitems;
    std::vector<CUtensorMap> hmaps[2];
    cudaGraphExec_t graph[2];          // captured kGraphChunk steps, one per starting buffer
    int graph_tile, graph_grid;
    std::string err;

    void* buf(int i) const { return ws + off_buf[i]; }
    double* fields() const { return (double*)(ws + off_fields); }
    double* nu() const { return (double*)(ws + off_nu); }
    int* flag() const { return (int*)(ws + off_flag); }
    const lbm::BatchItem* items(int t) const { return (const lbm::BatchItem*)(ws + off_items[t]); }
    int* bounds() const { return (int*)(ws + off_bounds); }
    const CUtensorMap* maps(int buffer) const { return (const CUtensorMap*)(ws + off_maps) + (size_t)buffer * n; }
    const lbm::StagedItem* sitems() const { return (const lbm::StagedItem*)(ws + off_sitems); }
    const lbm::StagedItem* pitems() const { return (const lbm::StagedItem*)(ws + off_pitems); }
    const lbm::PersistCavity* pcav() const { return (const lbm::PersistCavity*)(ws + off_pcav); }
    int* done() const { return (int*)(ws + off_done); }
    size_t es() const { return precision == LBM_F64 ? 8 : 4; }
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& m) {
    if (b) b->err = m;
    else g_batch_create_error = m;
    return s;
}

lbm_status bcuda(lbm_batch* b, cudaError_t e, const char* what) {
    return bfail(b, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_BCUDA(b, call, what)                                \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return bcuda((b), e_, (what));   \
    } while (0)

int tile_index(int tile_x) { return tile_x == 32 ? 0 : (tile_x == 64 ? 1 : 2); }

// Number of wall nodes of a cavity (the perimeter order of the batched kernel).
int perimeter_count(const lbm_params& p) {
    const bool wS = p.bc[2] != LBM_BC_PERIODIC, wN = p.bc[3] != LBM_BC_PERIODIC;
    const int rows = (wS ? p.nx : 0) + (wN ? p.nx : 0);
    const int inner = (wN ? p.ny - 1 : p.ny) - (wS ? 1 : 0);
    const int cols = (p.bc[0] != LBM_BC_PERIODIC ? inner : 0) + (p.bc[1] != LBM_BC_PERIODIC ? inner : 0);
    return rows + cols;
}

// Work items of every cavity for tile width tile_x (tiles tile_x x 128/tile_x,
// their interior nodes), then its wall nodes in chunks of 128; cum receives the
// cumulative estimated cost.
std::vector<lbm::BatchItem> make_items(const std::vector<lbm_params>& prm, int tile_x, std::vector<double>* cum) {
    const int ty = 128 / tile_x;
    std::vector<lbm::BatchItem> v;
    double acc = 0.0;
    if (cum) cum->assign(1, 0.0);
    for (int c = 0; c < (int)prm.size(); ++c) {
        for (int y0 = 0; y0 < prm[c].ny; y0 += ty)
            for (int x0 = 0; x0 < prm[c].nx; x0 += tile_x) {
                v.push_back({c, x0, y0, 0});
                const int w = std::min(tile_x, prm[c].nx - x0) * std::min(ty, prm[c].ny - y0);
                acc += w;
                if (cum) cum->push_back(acc);
            }
        const int nw = perimeter_count(prm[c]);
        for (int a = 0; a < nw; a += 128) {
            const int n = std::min(128, nw - a);
            v.push_back({c, a, n, 1});
            acc += kWallCost * n;
            if (cum) cum->push_back(acc);
        }
    }
    return v;
}

// Whether every cavity can take the staged kernel (FP32, walled on all four
// sides, at least 4 x 4 nodes).
bool stageable(const std::vector<lbm_params>& prm) {
    for (const lbm_params& p : prm) {
        if (p.precision != LBM_F32 || p.nx < 4 || p.ny < 4) return false;
        for (int q = 0; q < 4; ++q)
            if (p.bc[q] == LBM_BC_PERIODIC) return false;
    }
    return true;
}

// Work items of the staged kernel: every cavity's bands of 128 columns x
// segments of `rows` rows, cavity by cavity.  The segments holding a cavity's
// S or N wall row (a full row of out-of-line wall updates) come first, so
// that the blocks the hardware starts last are plain interior ones.
// Segments do not share source rows, so the order costs no extra traffic.
std::vector<lbm::StagedItem> make_staged_items(const std::vector<lbm_params>& prm, int rows) {
    std::vector<lbm::StagedItem> walls, inner;
    for (int c = 0; c < (int)prm.size(); ++c)
        for (int y0 = 0; y0 < prm[c].ny; y0 += rows) {
            std::vector<lbm::StagedItem>& v = (y0 == 0 || y0 + rows >= prm[c].ny) ? walls : inner;
            for (int x0 = 0; x0 < prm[c].nx; x0 += 128) v.push_back({c, x0, y0, prm[c].ny});
        }
    walls.insert(walls.end(), inner.begin(), inner.end());
    return walls;
}

// Work list of the persistent staged step: every cavity's segments of `rows`
// rows x bands of 128 columns, cavity by cavity, segment-major, and the
// position of each cavity's items in it.
std::vector<lbm::StagedItem> make_persist_items(const std::vector<lbm_params>& prm, int rows,
                                                std::vector<lbm::PersistCavity>* pc) {
    std::vector<lbm::StagedItem> v;
    if (pc) pc->clear();
    for (int c = 0; c < (int)prm.size(); ++c) {
        const int nb = (prm[c].nx + 127) / 128, ns = (prm[c].ny + rows - 1) / rows;
        if (pc) pc->push_back({(int)v.size(), nb, ns, 0});
        for (int g = 0; g < ns; ++g)
            for (int bd = 0; bd < nb; ++bd) v.push_back({c, bd * 128, g * rows, prm[c].ny});
    }
    return v;
}

// Block ranges of equal estimated cost: bounds[k] is the first item of block k.
std::vector<int> make_bounds(const std::vector<double>& cum, int grid) {
    const int n = (int)cum.size() - 1;
    std::vector<int> bnd(grid + 1);
    const double total = cum.back();
    int it = 0;
    for (int k = 0; k <= grid; ++k) {
        const double target = total * k / grid;
        while (it < n && cum[it] < target) ++it;
        bnd[k] = (k == grid) ? n : it;
    }
    return bnd;
}

// Layout of a batch; fills the offsets of b (b may be a scratch object).
lbm_status batch_layout(const lbm_params* p, int n, lbm_batch* b, std::string* why) {
    const int prec = p[0].precision;
    if (prec != LBM_F64 && prec != LBM_F32) { *why = "batches store FP64 or FP32 populations"; return LBM_ERR_ARG; }
    for (int c = 0; c < n; ++c)
        if (p[c].moment_state) { *why = "batches store populations (moment_state must be 0)"; return LBM_ERR_ARG; }
    b->n = n;
    b->precision = prec;
    b->prm.assign(p, p + n);
    b->offset.resize(n);
    const size_t es = prec == LBM_F64 ? 8 : 4;
    size_t elems = 0;
    b->max_cells = 0;
    for (int c = 0; c < n; ++c) {
        lbm_status s = check_shape(&p[c], why);
        if (s != LBM_OK) return s;
        if (p[c].precision != prec) { *why = "all cavities of a batch share one precision"; return LBM_ERR_ARG; }
        const Layout L = layout(&p[c]);
        b->offset[c] = (long long)elems;
        elems += align256(L.plane_elems * es * lbm::NPLANES) / es;
        b->max_cells = std::max(b->max_cells, (size_t)p[c].nx * p[c].ny);
    }
    if (elems >= (size_t)1 << 40) { *why = "batch too large"; return LBM_ERR_ARG; }
    b->buf_elems = elems;
    size_t o = 0;
    b->guards.clear();
    // each region is followed by a guard word (see lbm_batch_check_guards)
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        b->guards.push_back(o);
        o += kGuardBytes;
        return at;
    };
    b->off_buf[0] = take(elems * es);
    b->off_buf[1] = take(elems * es);
    b->off_cav = take((size_t)n * (prec == LBM_F64 ? sizeof(lbm::BatchCavity<double>) : sizeof(lbm::BatchCavity<float>)));
    for (int t = 0; t < 3; ++t) {
        b->n_items[t] = (int)make_items(b->prm, kTiles[t], &b->cum[t]).size();
        b->off_items[t] = take((size_t)b->n_items[t] * sizeof(lbm::BatchItem));
    }
    b->off_bounds = take((size_t)(kMaxGrid + 1) * sizeof(int));
    b->n_sitems = 0;
    b->off_maps = b->off_sitems = b->off_pitems = b->off_pcav = b->off_done = o;
    if (stageable(b->prm)) {
        const size_t ns = make_staged_items(b->prm, lbm::tma_batch_rows()).size();
        if (ns >= (size_t)1 << 31) { *why = "batch too large"; return LBM_ERR_ARG; }
        b->n_sitems = (int)ns;
        b->off_maps = take((size_t)2 * n * sizeof(CUtensorMap));
        b->off_sitems = take(ns * sizeof(lbm::StagedItem));
        b->off_pitems = take(ns * sizeof(lbm::StagedItem));
        b->off_pcav = take((size_t)n * sizeof(lbm::PersistCavity));
        b->off_done = take((ns + 1) * sizeof(int));
    }
    b->off_fields = take(4 * b->max_cells * sizeof(double));
    b->off_nu = take((size_t)n * sizeof(double));
    b->off_flag = take(256);
    b->ws_bytes = o;
    return LBM_OK;
}

template <class R>
lbm::BatchCavity<R> cavity_desc(const lbm_params& p, long long offset, int* flag) {
    Derived d;
    std::string why;
    derive(&p, &d, &why);
    const Layout L = layout(&p);
    lbm::BatchCavity<R> c;
    memset(&c, 0, sizeof(c));
    c.k = make_kconst<R>(&p, d, L, flag);
    c.d.T0 = d.T0;
    c.d.inv_sigma = 1.0 / p.sigma;
    c.d.Q = d.Q;
    c.d.L = d.L;
    c.d.dT = d.dT;
    for (int q = 0; q < 4; ++q) c.d.T_bc[q] = p.T_bc[q];
    c.offset = offset;
    return c;
}

template <class F>
cudaError_t bdispatch(lbm_batch* b, F&& fn) {
    if (b->precision == LBM_F64)
        return fn((const lbm::BatchCavity<double>*)(b->ws + b->off_cav), b->cav64, (double*)nullptr);
    return fn((const lbm::BatchCavity<float>*)(b->ws + b->off_cav), b->cav32, (float*)nullptr);
}

// Upload the block ranges of launch shape (tile_x, grid) (stream ordered).
cudaError_t set_bounds(lbm_batch* b, int tile_x, int grid) {
    if (b->bounds_tile == tile_x && b->bounds_grid == grid) return cudaSuccess;
    const std::vector<int> bnd = make_bounds(b->cum[tile_index(tile_x)], grid);
    cudaError_t e = cudaMemcpyAsync(b->bounds(), bnd.data(), bnd.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) {
        b->bounds_tile = tile_x;
        b->bounds_grid = grid;
    }
    return e;
}

cudaError_t fused_step(lbm_batch* b, int tile_x, int grid) {
    const int t = tile_index(tile_x);
    const int src = b->cur, dst = 1 - b->cur;
    if (b->staged)
        return lbm::launch_step_batch_tma((const lbm::BatchCavity<float>*)(b->ws + b->off_cav), b->maps(src),
                                          b->sitems(), b->n_sitems, (const float*)b->buf(src), (float*)b->buf(dst),
                                          (uint32_t)b->steps, b->stream);
    cudaError_t e = set_bounds(b, tile_x, grid);
    if (e != cudaSuccess) return e;
    return bdispatch(b, [&](auto* dcav, auto&, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_step_batch(dcav, b->items(t), b->bounds(), tile_x, grid, (const S*)b->buf(src),
                                      (S*)b->buf(dst), (uint32_t)b->steps, b->stream);
    });
}

cudaError_t per_case_step(lbm_batch* b) {
    const int src = b->cur, dst = 1 - b->cur;
    if (b->staged) {
        for (int c = 0; c < b->n; ++c) {
            const long long o = b->cav32[c].offset;
            cudaError_t e = lbm::launch_step_tma(b->cav32[c].k, b->hmaps[src][c], (const float*)b->buf(src) + o,
                                                 (float*)b->buf(dst) + o, lbm::tma_batch_rows(), (uint32_t)b->steps,
                                                 b->stream);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    return bdispatch(b, [&](auto*, auto& hc, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        for (int c = 0; c < b->n; ++c) {
            cudaError_t e = lbm::launch_step(hc[c].k, (const S*)b->buf(src) + hc[c].offset,
                                             (S*)b->buf(dst) + hc[c].offset, (uint32_t)b->steps, b->stream);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    });
}

void drop_graphs(lbm_batch* b) {
    for (int i = 0; i < 2; ++i)
        if (b->graph[i]) {
            cudaGraphExecDestroy(b->graph[i]);
            b->graph[i] = nullptr;
        }
}

// Capture kGraphChunk fused steps starting from buffer `start`.
lbm_status capture(lbm_batch* b, int start) {
    const int saved_cur = b->cur;
    const int64_t saved_steps = b->steps;
    b->cur = start;
    cudaGraph_t g = nullptr;
    LBM_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kGraphChunk && e == cudaSuccess; ++i) {
        e = fused_step(b, b->tile_x, b->grid);
        b->cur = 1 - b->cur;
        ++b->steps;
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    b->cur = saved_cur;
    b->steps = saved_steps;
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return bcuda(b, e, "captured step"); }
    if (e2 != cudaSuccess) return bcuda(b, e2, "end capture");
    e = cudaGraphInstantiate(&b->graph[start], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(b, e, "graph instantiate");
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_workspace_size(const lbm_params* p, int32_t n, size_t* bytes) {
    if (!p || n < 1 || !bytes) return LBM_ERR_ARG;
    lbm_batch b;
    std::string why;
    lbm_status s = batch_layout(p, n, &b, &why);
    if (s != LBM_OK) return bfail(nullptr, s, why);
    *bytes = b.ws_bytes;
    return LBM_OK;
}

lbm_status lbm_batch_create(const lbm_params* p, int32_t n, void* stream, void* workspace,
                            size_t workspace_bytes, lbm_batch** out) {
    if (!p || n < 1 || !out) return bfail(nullptr, LBM_ERR_ARG, "null argument or empty batch");
    *out = nullptr;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ERR_OOM, "host allocation failed");
    std::string why;
    lbm_status s = batch_layout(p, n, b, &why);
    if (s == LBM_OK)
        for (int c = 0; c < n && s == LBM_OK; ++c) {
            Derived d;
            s = derive(&p[c], &d, &why);
        }
    if (s != LBM_OK) {
        delete b;
        return bfail(nullptr, s, why);
    }
    if (workspace && (workspace_bytes < b->ws_bytes || ((uintptr_t)workspace & 255))) {
        delete b;
        return bfail(nullptr, LBM_ERR_OOM, "workspace too small or not 256-byte aligned");
    }
    b->stream = (cudaStream_t)stream;
    b->owns_ws = workspace == nullptr;
    b->ws = (char*)workspace;
    if (b->owns_ws) {
        cudaError_t e = cudaMalloc((void**)&b->ws, b->ws_bytes);
        if (e != cudaSuccess) {
            delete b;
            return bfail(nullptr, LBM_ERR_OOM, std::string("cudaMalloc of the batch workspace: ") + cudaGetErrorString(e));
        }
    }
    b->cur = 0;
    b->steps = b->launches = 0;
    b->nonfinite = b->timeout = false;
    b->staged = b->staged_ready = false;
    b->graph[0] = b->graph[1] = nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->sms < 1) b->sms = 1;
    // descriptors
    for (int c = 0; c < n; ++c) {
        if (b->precision == LBM_F64) b->cav64.push_back(cavity_desc<double>(p[c], b->offset[c], b->flag()));
        else b->cav32.push_back(cavity_desc<float>(p[c], b->offset[c], b->flag()));
    }
    auto upload = [&](size_t off, const void* src, size_t bytes, const char* what) -> lbm_status {
        cudaError_t e = cudaMemcpyAsync(b->ws + off, src, bytes, cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, what);
        return LBM_OK;
    };
    for (size_t g = 0; g < b->guards.size() && s == LBM_OK; ++g) {
        const cudaError_t e = cudaMemsetAsync(b->ws + b->guards[g], kGuardByte, kGuardBytes, b->stream);
        if (e != cudaSuccess) s = bcuda(b, e, "guard words");
    }
    if (s == LBM_OK)
        s = b->precision == LBM_F64
                ? upload(b->off_cav, b->cav64.data(), n * sizeof(lbm::BatchCavity<double>), "descriptors")
                : upload(b->off_cav, b->cav32.data(), n * sizeof(lbm::BatchCavity<float>), "descriptors");
    for (int t = 0; t < 3 && s == LBM_OK; ++t) {
        std::vector<lbm::BatchItem> it = make_items(b->prm, kTiles[t], nullptr);
        s = upload(b->off_items[t], it.data(), it.size() * sizeof(lbm::BatchItem), "work list");
        if (s == LBM_OK) s = (cudaStreamSynchronize(b->stream) == cudaSuccess) ? LBM_OK : LBM_ERR_CUDA;
    }
    if (s == LBM_OK && b->n_sitems > 0) {
        bool ok = true;
        for (int i = 0; i < 2; ++i) {
            b->hmaps[i].resize(n);
            for (int c = 0; c < n && ok; ++c)
                ok = lbm::make_step_tensor_map(b->cav32[c].k, (const float*)b->buf(i) + b->cav32[c].offset,
                                               &b->hmaps[i][c]);
        }
        if (ok) {
            std::vector<lbm::StagedItem> it = make_staged_items(b->prm, lbm::tma_batch_rows());
            s = upload(b->off_sitems, it.data(), it.size() * sizeof(lbm::StagedItem), "staged work list");
            std::vector<lbm::PersistCavity> pc;
            std::vector<lbm::StagedItem> pit = make_persist_items(b->prm, lbm::tma_batch_rows(), &pc);
            if (s == LBM_OK && (int)pit.size() != b->n_sitems) s = bfail(b, LBM_ERR_ARG, "persistent work list size");
            if (s == LBM_OK) s = upload(b->off_pitems, pit.data(), pit.size() * sizeof(lbm::StagedItem), "persistent work list");
            if (s == LBM_OK) s = upload(b->off_pcav, pc.data(), pc.size() * sizeof(lbm::PersistCavity), "persistent layout");
            for (int i = 0; i < 2 && s == LBM_OK; ++i)
                s = upload(b->off_maps + (size_t)i * n * sizeof(CUtensorMap), b->hmaps[i].data(),
                           (size_t)n * sizeof(CUtensorMap), "tensor maps");
            if (s == LBM_OK) s = (cudaStreamSynchronize(b->stream) == cudaSuccess) ? LBM_OK : LBM_ERR_CUDA;
            b->staged = b->staged_ready = s == LBM_OK;
        }
    }
    // default launch shape: 32-wide tiles, one wave of resident blocks
    b->tile_x = 32;
    int occ = 0;
    if (b->precision == LBM_F64) occ = lbm::batch_blocks_per_sm<double, double>(32);
    else occ = lbm::batch_blocks_per_sm<float, float>(32);
    b->grid = std::min(b->sms * std::max(occ, 1), kMaxGrid);
    b->bounds_tile = b->bounds_grid = -1;
    if (s == LBM_OK) s = lbm_batch_set_fields(b, -1, nullptr, nullptr, nullptr);
    if (s != LBM_OK) {
        g_batch_create_error = b->err;
        lbm_batch_destroy(b);
        return s;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    drop_graphs(b);
    if (b->owns_ws && b->ws) {
        cudaStreamSynchronize(b->stream);
        cudaFree(b->ws);
    }
    delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) {
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

lbm_status lbm_batch_set_fields(lbm_batch* b, int32_t cavity, const double* T, const double* ux,
                                const double* uy) {
    if (!b) return LBM_ERR_ARG;
    if (cavity < -1 || cavity >= b->n) return bfail(b, LBM_ERR_ARG, "cavity index out of range");
    const int first = cavity < 0 ? 0 : cavity, last = cavity < 0 ? b->n : cavity + 1;
    if (cavity < 0 && (T || ux || uy)) return bfail(b, LBM_ERR_ARG, "fields are given one cavity at a time");
    double* F = b->fields();
    for (int c = first; c < last; ++c) {
        const size_t N = (size_t)b->prm[c].nx * b->prm[c].ny;
        const double* src[3] = {T, ux, uy};
        const double* dev[3] = {nullptr, nullptr, nullptr};
        for (int q = 0; q < 3; ++q)
            if (src[q]) {
                LBM_BCUDA(b, cudaMemcpyAsync(F + q * N, src[q], N * sizeof(double), cudaMemcpyHostToDevice, b->stream),
                          "copy of an input field");
                dev[q] = F + q * N;
            }
        // both buffers: a cavity's state lives in the current one
        cudaError_t e = bdispatch(b, [&](auto*, auto& hc, auto* tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            return lbm::launch_init(hc[c].k, (S*)b->buf(b->cur) + hc[c].offset, dev[0], dev[1], dev[2],
                                    b->prm[c].T_init, b->stream);
        });
        if (e != cudaSuccess) return bcuda(b, e, "init kernel");
        LBM_BCUDA(b, cudaStreamSynchronize(b->stream), "set_fields");
    }
    LBM_BCUDA(b, cudaMemsetAsync(b->flag(), 0, sizeof(int), b->stream), "flag reset");
    LBM_BCUDA(b, cudaStreamSynchronize(b->stream), "set_fields");
    if (cavity < 0) b->steps = 0;
    b->nonfinite = b->timeout = false;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t n, int mode) {
    const NvtxRange range("lbm_batch_step");
    if (!b || n < 0) return b ? bfail(b, LBM_ERR_ARG, "negative step count") : LBM_ERR_ARG;
    if (b->timeout) return bfail(b, LBM_ERR_TIMEOUT, "a bounded wait of the staged step gave up");
    if (b->nonfinite) return bfail(b, LBM_ERR_NONFINITE, "non-finite velocity or temperature");
    if (mode < LBM_BATCH_FUSED || mode > LBM_BATCH_PERSISTENT) return bfail(b, LBM_ERR_ARG, "unknown mode");
    if (mode == LBM_BATCH_PERSISTENT) {
        if (!b->staged) return bfail(b, LBM_ERR_ARG, "the persistent step needs the staged kernel (FP32, walled cavities)");
        if (n == 0) return LBM_OK;
        if (n > (int64_t)1 << 30) return bfail(b, LBM_ERR_ARG, "too many steps for one persistent launch");
        int* done = b->done();
        cudaError_t e = lbm::launch_step_batch_persist(
            (const lbm::BatchCavity<float>*)(b->ws + b->off_cav), b->pcav(), b->maps(0), b->pitems(), b->n_sitems, b->n,
            (float*)b->buf(0), (float*)b->buf(1), b->cur, (uint32_t)b->steps, (int)n, done, done + b->n_sitems,
            b->flag(), b->sms, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "persistent batched step");
        b->launches += 1;
        b->steps += n;
        if (n & 1) b->cur = 1 - b->cur;
        return LBM_OK;
    }
    if (mode == LBM_BATCH_GRAPH && b->stream == nullptr)
        return bfail(b, LBM_ERR_ARG, "graph mode needs a stream other than the legacy default stream");
    int64_t done = 0;
    if (mode == LBM_BATCH_GRAPH) {
        if (b->graph_tile != b->tile_x || b->graph_grid != b->grid) drop_graphs(b);
        while (n - done >= kGraphChunk) {
            if (!b->graph[b->cur]) {
                // the block ranges are uploaded outside the capture
                LBM_BCUDA(b, set_bounds(b, b->tile_x, b->grid), "work ranges");
                lbm_status s = capture(b, b->cur);
                if (s != LBM_OK) return s;
                b->graph_tile = b->tile_x;
                b->graph_grid = b->grid;
            }
            LBM_BCUDA(b, cudaGraphLaunch(b->graph[b->cur], b->stream), "graph launch");
            b->steps += kGraphChunk;
            b->launches += kGraphChunk;
            done += kGraphChunk;  // kGraphChunk is even: the current buffer is unchanged
        }
    }
    for (; done < n; ++done) {
        cudaError_t e = (mode == LBM_BATCH_PER_CASE) ? per_case_step(b) : fused_step(b, b->tile_x, b->grid);
        if (e != cudaSuccess) return bcuda(b, e, "batched step");
        b->launches += (mode == LBM_BATCH_PER_CASE) ? b->n : 1;
        b->cur = 1 - b->cur;
        ++b->steps;
    }
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int32_t steps_per_candidate, int32_t* tile_x, int32_t* grid) {
    if (!b || steps_per_candidate < 1) return LBM_ERR_ARG;
    if (b->nonfinite) return bfail(b, LBM_ERR_NONFINITE, "non-finite velocity or temperature");
    cudaEvent_t e0, e1;
    LBM_BCUDA(b, cudaEventCreate(&e0), "event");
    LBM_BCUDA(b, cudaEventCreate(&e1), "event");
    float best = 1e30f;
    int best_tile = b->tile_x, best_grid = b->grid;
    for (int t = 0; t < 3; ++t) {
        int occ = b->precision == LBM_F64 ? lbm::batch_blocks_per_sm<double, double>(kTiles[t])
                                          : lbm::batch_blocks_per_sm<float, float>(kTiles[t]);
        occ = std::max(occ, 1);
        for (int waves = 1; waves <= 4; waves *= 2) {
            const int g = std::min(b->sms * occ * waves, kMaxGrid);
            // these are real steps of the run: every launch shape computes the
            // same values, so tuning does not change the results
            cudaError_t e = fused_step(b, kTiles[t], g);
            b->cur = 1 - b->cur; ++b->steps; ++b->launches;
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            for (int i = 0; i < steps_per_candidate && e == cudaSuccess; ++i) {
                e = fused_step(b, kTiles[t], g);
                b->cur = 1 - b->cur; ++b->steps; ++b->launches;
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return bcuda(b, e, "autotune");
            }
            if (ms < best) { best = ms; best_tile = kTiles[t]; best_grid = g; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tile_x = best_tile;
    b->grid = best_grid;
    drop_graphs(b);
    if (tile_x) *tile_x = best_tile;
    if (grid) *grid = best_grid;
    return LBM_OK;
}

lbm_status lbm_batch_set_launch(lbm_batch* b, int32_t tile_x, int32_t grid) {
    if (!b) return LBM_ERR_ARG;
    if ((tile_x != 32 && tile_x != 64 && tile_x != 128) || grid < 1 || grid > kMaxGrid)
        return bfail(b, LBM_ERR_ARG, "bad launch shape");
    b->tile_x = tile_x;
    b->grid = grid;
    drop_graphs(b);
    return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b) {
    if (!b) return LBM_ERR_ARG;
    LBM_BCUDA(b, cudaStreamSynchronize(b->stream), "stream synchronise");
    int flag = 0;
    LBM_BCUDA(b, cudaMemcpy(&flag, b->flag(), sizeof(int), cudaMemcpyDeviceToHost), "flag read");
    if (flag & 2) b->timeout = true;
    if (flag & 1) b->nonfinite = true;
    if (b->timeout) return bfail(b, LBM_ERR_TIMEOUT, "a bounded wait of the staged step gave up");
    if (b->nonfinite) return bfail(b, LBM_ERR_NONFINITE, "non-finite velocity or temperature");
    return LBM_OK;
}

lbm_status lbm_batch_set_staging(lbm_batch* b, int32_t staged) {
    if (!b) return LBM_ERR_ARG;
    if (staged && !b->staged_ready)
        return bfail(b, LBM_ERR_ARG, "staged rows need FP32 cavities walled on all sides");
    if (b->staged != (staged != 0)) drop_graphs(b);
    b->staged = staged != 0;
    return LBM_OK;
}

int32_t lbm_batch_staged(const lbm_batch* b) { return b && b->staged ? 1 : 0; }

lbm_status lbm_batch_check_guards(lbm_batch* b) {
    if (!b) return LBM_ERR_ARG;
    LBM_BCUDA(b, cudaStreamSynchronize(b->stream), "stream synchronise");
    unsigned char w[kGuardBytes];
    for (size_t g = 0; g < b->guards.size(); ++g) {
        LBM_BCUDA(b, cudaMemcpy(w, b->ws + b->guards[g], kGuardBytes, cudaMemcpyDeviceToHost), "guard read");
        for (size_t i = 0; i < kGuardBytes; ++i)
            if (w[i] != kGuardByte)
                return bfail(b, LBM_ERR_GUARD,
                             "guard word after workspace region " + std::to_string(g) + " overwritten at byte " +
                                 std::to_string(i));
    }
    return LBM_OK;
}

lbm_status lbm_batch_nusselt(lbm_batch* b, int side, double* nu_mean) {
    if (!b || side < 0 || side > 3 || !nu_mean) return b ? bfail(b, LBM_ERR_ARG, "bad side or null output") : LBM_ERR_ARG;
    for (int c = 0; c < b->n; ++c)
        if ((side <= 1 ? b->prm[c].nx : b->prm[c].ny) < 3) return bfail(b, LBM_ERR_ARG, "a cavity is too thin");
    cudaError_t e = bdispatch(b, [&](auto* dcav, auto&, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_nusselt_batch(dcav, b->n, (const S*)b->buf(b->cur), side, b->nu(), b->stream);
    });
    if (e != cudaSuccess) return bcuda(b, e, "nusselt kernel");
    LBM_BCUDA(b, cudaMemcpyAsync(nu_mean, b->nu(), b->n * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
              "nusselt copy");
    LBM_BCUDA(b, cudaStreamSynchronize(b->stream), "nusselt");
    return LBM_OK;
}

lbm_status lbm_batch_moments(lbm_batch* b, int32_t cavity, double* p, double* ux, double* uy, double* T) {
    if (!b) return LBM_ERR_ARG;
    if (cavity < 0 || cavity >= b->n) return bfail(b, LBM_ERR_ARG, "cavity index out of range");
    const size_t N = (size_t)b->prm[cavity].nx * b->prm[cavity].ny;
    double* F = b->fields();
    cudaError_t e = bdispatch(b, [&](auto*, auto& hc, auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return lbm::launch_moments(hc[cavity].k, (const S*)b->buf(b->cur) + hc[cavity].offset, F, F + N,
                                   F + 2 * N, F + 3 * N, b->stream);
    });
    if (e != cudaSuccess) return bcuda(b, e, "moments kernel");
    double* outs[4] = {p, ux, uy, T};
    for (int q = 0; q < 4; ++q)
        if (outs[q])
            LBM_BCUDA(b, cudaMemcpyAsync(outs[q], F + q * N, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
                      "moment copy");
    LBM_BCUDA(b, cudaStreamSynchronize(b->stream), "moments");
    return LBM_OK;
}

int64_t lbm_batch_steps_done(const lbm_batch* b) { return b ? b->steps : -1; }

int64_t lbm_batch_kernel_launches(const lbm_batch* b) { return b ? b->launches : -1; }

}  // extern "C"
