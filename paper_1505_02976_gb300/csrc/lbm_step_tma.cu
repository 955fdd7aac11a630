// lbm_step_tma.cu -- the FP32 / FP16-storage step with its loads staged by
// the tensor memory accelerator (TMA).
//
// Same per-node arithmetic as k_step (fast_moments and fast_collide for
// interior nodes, the out-of-line NEES path for wall nodes), but the 17
// pulled values of every interior node reach the block through shared
// memory.  Pull streaming reads plane i of output row y from global row
// y - c_iy, so each plane of each global row is used by exactly one output
// row: a slot holds the 17 planes one output row needs, each plane loaded by
// one 3-D tensor copy (128 + 2 halo columns x 1 row x 1 plane) from its own
// source row.  A block owns a band of 128 columns and a segment of up to
// kTRows rows.  One thread issues all of the block's copies at its start (17
// plane rows per output row, 37 KB for 4 FP32 rows), and each thread waits
// on each row's mbarrier instead of on its own global loads; the slots are
// written once, so no block barrier separates the rows.  Many short blocks
// keep the SMs busy to the end of the step: on the 2048^2 and 8192^2 FP32
// cavities, 4-row segments beat 2, 3, 5, 6, 8, 16, 32 and 64 rows streamed
// through a ring of 2 to 6 row slots, and the global-load step.
//
// Wall nodes (the segment's part of the W and E columns, and the S and N
// rows) are updated before the row loop, all in parallel, while the copies
// are in flight; the row loop then runs interior nodes only.
//
// Used for FP32 and FP16 storage on lattices walled on all four sides (a
// periodic side would need wrapped halo columns, which the tile copy does not
// give): every interior node pulls only from nodes inside the lattice, and
// the zero fill of out-of-range boxes is never read.  Waits are bounded: a
// wait that gives up sets bit 1 of the handle's flag (LBM_ERR_TIMEOUT) and
// the block stops after its copies in flight have landed.
#include <cuda.h>
#include <math.h>

#include <type_traits>

#include "lbm_internal.h"
#include "lbm_pair.cuh"
#include "lbm_step.cuh"

namespace lbm {

constexpr int kTBand = 128;  // output columns per band = threads per block
#ifndef LBM_TMA_ROWS
#define LBM_TMA_ROWS 4
#endif
constexpr int kTRows = LBM_TMA_ROWS;  // output rows staged per block (the segment's interior rows)
#ifndef LBM_ALT_SWEEP
#define LBM_ALT_SWEEP 1
#endif
constexpr unsigned long long kTWaitNs = 2000000000ull;  // a wait gives up after 2 s
constexpr long long kTWaitPolls = 1ll << 28;             // ... or after this many polls

// Shared-memory layout of the staged rows: storage type S, BAND output
// columns per block, ROWS output rows.  A copy starts `halo` columns left of
// the band so that its x coordinate stays a multiple of 16 bytes; a copy's
// shared-memory destination must be 128-byte aligned, so each plane row of a
// slot is padded to a multiple of 128 bytes.
template <class S, int BAND, int ROWS, int HALO = 16 / (int)sizeof(S)>
struct StageLayout {
    using type = S;
    static constexpr int band = BAND;
    static constexpr int rows = ROWS;
    static constexpr int halo = HALO;                                       // 4 (FP32), LBM_H_INNER (FP16)
    static constexpr int box = BAND + 2 * halo;                             // columns copied per plane row
    static constexpr int plane = ((box * (int)sizeof(S) + 127) / 128) * 128 / (int)sizeof(S);
    static constexpr int slot = NPLANES * plane;                            // elements per slot
    static constexpr unsigned bytes = (unsigned)(NPLANES * box * sizeof(S));  // bytes landing per slot
    // slots, barriers, and room to round the first slot up to 128 bytes
    static constexpr size_t smem = 128 + (size_t)ROWS * slot * sizeof(S) + ROWS * sizeof(uint64_t);
    // resident blocks per SM that the shared memory allows (228 KB per SM,
    // 1 KB reserved per block), at most 8
    static constexpr int blocks = (int)((228 * 1024) / (smem + 1024)) < 8 ? (int)((228 * 1024) / (smem + 1024)) : 8;
    static_assert(plane * sizeof(S) % 128 == 0, "plane rows must stay 128-byte aligned");
};
// FP32 storage: one node per thread, a band of 128 columns, kTRows rows.
template <class S> struct TmaLayoutOf;
template <> struct TmaLayoutOf<float> { using type = StageLayout<float, kTBand, kTRows>; };
// FP16 storage: two x-adjacent nodes per thread (one pair per thread), a
// band of 256 columns, kHRows rows.
#ifndef LBM_TMA_ROWS_H
#define LBM_TMA_ROWS_H 4
#endif
constexpr int kHRows = LBM_TMA_ROWS_H;
// FP16 copies are 4-D boxes whose innermost dimension holds LBM_H_INNER
// columns; the band's halo is one such group on each side.
#ifndef LBM_H_INNER
#define LBM_H_INNER 32
#endif
constexpr int kHInner = LBM_H_INNER;
template <> struct TmaLayoutOf<__half> { using type = StageLayout<__half, 2 * kTBand, kHRows, kHInner>; };
template <class S> using TmaLayout = typename TmaLayoutOf<S>::type;
// Resident blocks per SM the kernels are compiled for (registers: 65536 /
// (threads x blocks) each): FP16 threads carry two nodes.
#ifndef LBM_TMA_BLOCKS_H
#define LBM_TMA_BLOCKS_H 5
#endif
template <class S> struct TmaBlocks { static constexpr int value = TmaLayout<S>::blocks; };
template <> struct TmaBlocks<__half> {
    static constexpr int value = TmaLayout<__half>::blocks < LBM_TMA_BLOCKS_H ? TmaLayout<__half>::blocks : LBM_TMA_BLOCKS_H;
};

// Source row offset (-c_iy) and column offset (-c_ix) of each stored plane:
// planes 0..7 hold f_1..f_8, planes 8..16 h_0..h_8; c: 1 (+1,0) 2 (0,+1)
// 3 (-1,0) 4 (0,-1) 5 (+1,+1) 6 (-1,+1) 7 (-1,-1) 8 (+1,-1).
__host__ __device__ constexpr int plane_dy(int p) {
    constexpr int d[NPLANES] = {0, -1, 0, 1, -1, -1, 1, 1, 0, 0, -1, 0, 1, -1, -1, 1, 1};
    return d[p];
}
__host__ __device__ constexpr int plane_dx(int p) {
    constexpr int d[NPLANES] = {-1, 0, 1, 0, -1, 1, 1, -1, 0, -1, 0, 1, 0, -1, 1, 1, -1};
    return d[p];
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// The 17 plane rows output row y pulls from, into one slot: plane p from
// global row y + plane_dy(p), columns x0 - halo .. x0 + 127 + halo.
// FP16 rows are described to the copy engine as 4-D, (8 columns, columns / 8,
// rows, planes): a box dimension holds at most 256 elements, and the 272
// columns of an FP16 band (256 + 2 x 8 halo) become a box of (8, 34, 1, 1),
// still one contiguous run in shared memory.  The innermost coordinate is
// always 0 and the column-group coordinate x / 8 may be -1 at the left edge
// (zero fill, never read).
template <class S>
__device__ __forceinline__ void tma_load_slot(const CUtensorMap* tm, S* slot, uint64_t* bar, int x, int y) {
    using L = TmaLayout<S>;
    const uint32_t b = smem_addr(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(L::bytes) : "memory");
#pragma unroll
    for (int p = 0; p < NPLANES; ++p) {
        if constexpr (sizeof(S) == 2)
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4, %5}], [%6];" ::"r"(smem_addr(slot + p * L::plane)),
                "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(x / kHInner), "r"(y + plane_dy(p)), "r"(p), "r"(b)
                : "memory");
        else
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4}], [%5];" ::"r"(smem_addr(slot + p * L::plane)),
                "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y + plane_dy(p)), "r"(p), "r"(b)
                : "memory");
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase `parity` of an mbarrier; false if it gave up
// (after limit_ns of the global timer, or kTWaitPolls polls).
__device__ __forceinline__ bool tma_wait(uint64_t* bar, uint32_t parity,
                                         unsigned long long limit_ns = kTWaitNs) {
    const uint32_t b = smem_addr(bar);
    const unsigned long long t0 = global_ns();
    for (long long i = 0; i < kTWaitPolls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 31) == 31 && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Shared memory of a staged block: the slots (128-byte aligned) and one
// mbarrier per slot, initialised by thread 0 (the caller synchronises the
// block before any thread waits on them).
template <class S>
__device__ __forceinline__ void staged_setup(unsigned char* smem_raw, S*& stage, uint64_t*& bar) {
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    stage = reinterpret_cast<S*>(base);
    bar = reinterpret_cast<uint64_t*>(base + (size_t)TmaLayout<S>::rows * TmaLayout<S>::slot * sizeof(S));
    if (threadIdx.x == 0) {
        for (int s = 0; s < TmaLayout<S>::rows; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar + s)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

// The tensor copies of one block (one thread): output row r of the interior
// rows yb .. ye - 1 of the segment y0 .. y0 + rows - 1 lands in slot r - yb
// (each slot and barrier is used once).
template <class S>
__device__ __forceinline__ void staged_issue(const CUtensorMap* tm, S* stage, uint64_t* bar, int x0, int y0, int rows,
                                             int ny, uint32_t /*phases*/ = 0u) {
    const int yb = max(y0, 1), ye = min(min(y0 + rows, ny), ny - 1);
    for (int r = yb; r < ye; ++r)
        tma_load_slot(tm, stage + (r - yb) * TmaLayout<S>::slot, bar + (r - yb), x0 - TmaLayout<S>::halo, r);
}

// The same copies issued by lane 0 of every warp, one row each (warp w takes
// rows yb + w, yb + w + warps, ...), so that the rows' copies leave together.
// The barriers must be initialised and visible to every warp.
template <class S>
__device__ __forceinline__ void staged_issue_warps(const CUtensorMap* tm, S* stage, uint64_t* bar, int x0, int y0,
                                                   int rows, int ny) {
    const int yb = max(y0, 1), ye = min(min(y0 + rows, ny), ny - 1);
    if ((threadIdx.x & 31) != 0) return;
    for (int r = yb + (int)(threadIdx.x >> 5); r < ye; r += (int)(blockDim.x >> 5))
        tma_load_slot(tm, stage + (r - yb) * TmaLayout<S>::slot, bar + (r - yb), x0 - TmaLayout<S>::halo, r);
}

// One block of the staged step once its copies are issued and its barriers
// are visible: columns x0 .. x0 + 127 and rows y0 .. y0 + rows - 1 (rows <=
// kTRows) of the lattice k with population buffers src / dst.  step: the
// step number (the stochastic rounding of FP16 stores draws from it).
// hot: the block's stores ask L2 to keep them (FP32; the FP16 form below
// does the same for its interior pairs).
template <class S, bool EPS_FIELD, bool TAU1>
__device__ __forceinline__ bool staged_rows(const KConst<float>& k, const S* __restrict__ src, S* __restrict__ dst,
                                            int x0, int y0, int rows, uint32_t step, const S* stage, uint64_t* bar,
                                            uint32_t phases = 0u, bool hot = false) {
    using L = TmaLayout<S>;
    const int tid = threadIdx.x;
    const int y1 = min(y0 + rows, k.ny);
    const int yb = max(y0, 1), ye = min(y1, k.ny - 1);  // interior rows of the segment (at most kTRows)
    const int x = x0 + tid;
    // wall nodes of the segment, in parallel, while the copies fly
    if (x < k.nx) {
        if (y0 == 0) wall_update(k, src, dst, x, 0, step);
        if (y1 == k.ny) wall_update(k, src, dst, x, k.ny - 1, step);
    }
    if (x0 == 0)
        for (int y = yb + tid; y < ye; y += kTBand) wall_update(k, src, dst, 0, y, step);
    if (x0 <= k.nx - 1 && k.nx - 1 < x0 + kTBand)
        for (int y = yb + tid; y < ye; y += kTBand) wall_update(k, src, dst, k.nx - 1, y, step);
    const bool active = x >= 1 && x <= k.nx - 2;
    const int c = tid + L::halo;
    // FP16 storage at tau = 1 folds its scale into the collision weights, as
    // the global-load kernel does
    constexpr bool prescale = TAU1 && std::is_same<S, __half>::value;
    // Each thread waits for its rows on its own: the slots are written once
    // and only read afterwards, so warps need no block barrier and run
    // decoupled.  Thread 0 waits for every row (inactive or not), so that
    // all copies have landed before the block can release its shared memory.
    bool ok = true;
    for (int y = yb; y < ye && (active || tid == 0); ++y) {
        if (!tma_wait(bar + (y - yb), (phases >> (y - yb)) & 1u)) {
            ok = false;
            break;
        }
        if (active) {
            const S* sl = stage + (y - yb) * L::slot + c;
            float f[9], h[9];
#pragma unroll
            for (int i = 1; i < 9; ++i) f[i] = load_pop<S, float>(sl + ((i - 1) * L::plane + plane_dx(i - 1)), k.scale);
#pragma unroll
            for (int i = 0; i < 9; ++i) h[i] = load_pop<S, float>(sl + ((8 + i) * L::plane + plane_dx(8 + i)), k.scale);
            float fo[9], ho[9];
            auto collide = [&](const KConst<float>& kk) {
                const FastState<float> st = fast_moments(kk, f, h, y);
                if constexpr (TAU1) fast_collide<float, true>(kk, st, f, h, fo, ho, prescale ? kk.inv_scale : 1.0f);
                else fast_collide<float, false>(kk, st, f, h, fo, ho);
            };
            if constexpr (EPS_FIELD) {
                KConst<float> kc = k;
                apply_eps(kc, node_eps(k, x, y));
                collide(kc);
            } else {
                collide(k);
            }
            const int at = y * k.pitch + x;
            Dither dither((uint32_t)at, step);
            store_planes<S, float>(dst + at, k.plane32, fo, ho, prescale ? 1.0f : k.inv_scale, &dither, hot);
        }
    }
    if (!ok) {
        atomicOr(k.flag, 2);
        // let this block's copies land before its shared memory is released
        if (tid == 0)
            for (int r = yb; r < ye; ++r) (void)tma_wait(bar + (r - yb), (phases >> (r - yb)) & 1u);
    }
    return ok;
}

// The FP16 form of staged_rows: one pair of x-adjacent nodes per thread,
// columns x0 + 2 tid (node a) and x0 + 2 tid + 1 (node b) of a band of 256
// columns.  Node a's slot column c is even, so each plane's two pulled
// values come from one aligned 32-bit word (no x shift) or from the halves
// of two neighbouring words (shift of one column); they are packed into one
// half2 per plane, node a in the lower half.  Both nodes' 17 values are then
// stored as pairs: one stochastic-rounding conversion and one 32-bit store
// per plane (a pair with a wall or out-of-range member stores its interior
// node alone, with the same rounding).
template <bool EPS_FIELD, bool TAU1>
__device__ __forceinline__ void staged_rows_pair(const KConst<float>& k, const __half* __restrict__ src,
                                                 __half* __restrict__ dst, int x0, int y0, int rows, uint32_t step,
                                                 const __half* stage, uint64_t* bar, bool hot = false) {
    using L = TmaLayout<__half>;
    const int tid = threadIdx.x;
    const int y1 = min(y0 + rows, k.ny);
    const int yb = max(y0, 1), ye = min(y1, k.ny - 1);  // interior rows of the segment
    const int xa = x0 + 2 * tid;
    // wall nodes of the segment, in parallel, while the copies fly
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (xa + q < k.nx) {
            if (y0 == 0) wall_update(k, src, dst, xa + q, 0, step);
            if (y1 == k.ny) wall_update(k, src, dst, xa + q, k.ny - 1, step);
        }
    }
    if (x0 == 0)
        for (int y = yb + tid; y < ye; y += kTBand) wall_update(k, src, dst, 0, y, step);
    if (x0 <= k.nx - 1 && k.nx - 1 < x0 + L::band)
        for (int y = yb + tid; y < ye; y += kTBand) wall_update(k, src, dst, k.nx - 1, y, step);
    const bool act0 = xa >= 1 && xa <= k.nx - 2;
    const bool act1 = xa + 1 <= k.nx - 2;
    const int c = 2 * tid + L::halo;
    // the storage scale folds into the collision weights at tau = 1
    const float out_scale = TAU1 ? 1.0f : k.inv_scale;
    bool ok = true;
    for (int y = yb; y < ye && (act0 || act1 || tid == 0); ++y) {
        if (!tma_wait(bar + (y - yb), 0u)) {
            ok = false;
            break;
        }
        if (!(act0 || act1)) continue;
        const __half* sl = stage + (y - yb) * L::slot + c;
        __half2 pk[NPLANES];
#pragma unroll
        for (int p = 0; p < NPLANES; ++p) {
            const __half* q = sl + p * L::plane;
            if (plane_dx(p) == 0) {
                pk[p] = *reinterpret_cast<const __half2*>(q);
            } else if (plane_dx(p) < 0) {
                const __half2 w0 = *reinterpret_cast<const __half2*>(q - 2);
                const __half2 w1 = *reinterpret_cast<const __half2*>(q);
                pk[p] = __halves2half2(__high2half(w0), __low2half(w1));
            } else {
                const __half2 w0 = *reinterpret_cast<const __half2*>(q);
                const __half2 w1 = *reinterpret_cast<const __half2*>(q + 2);
                pk[p] = __halves2half2(__high2half(w0), __low2half(w1));
            }
        }
        const int at = y * k.pitch + xa;
        if constexpr (TAU1 && !EPS_FIELD) {
            if (act0 && act1) {
                // both nodes interior: the lane form on the pair, node a in
                // .x and node b in .y of every packed value (the compiler
                // may fuse some of its multiplies into the following adds,
                // so the pair's values can differ from those of the
                // one-node path by FP32 rounding; the stored FP16 values
                // then differ by at most one rounding step)
                float2 f2[9], h2[9], fo2[9], ho2[9];
                const float2 sc = make_float2(k.scale, k.scale);
#pragma unroll
                for (int i = 1; i < 9; ++i) f2[i] = lmul(__half22float2(pk[i - 1]), sc);
#pragma unroll
                for (int i = 0; i < 9; ++i) h2[i] = lmul(__half22float2(pk[8 + i]), sc);
                const LaneState<float2> st = lane_moments<float2>(k, f2, h2, y);
                lane_collide<float2>(k, st, fo2, ho2, k.inv_scale);
                const Dither dither((uint32_t)at, step);
                uint32_t* wd = reinterpret_cast<uint32_t*>(dst + at);
                const int pw = k.plane32 >> 1;
                if (hot) {
                    uint64_t pol;
                    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
#pragma unroll
                    for (int i = 1; i < 9; ++i)
                        asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(wd + (i - 1) * pw),
                                     "r"(half2_sr(fo2[i].y, fo2[i].x, dither.word(i - 1))), "l"(pol) : "memory");
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(wd + (8 + i) * pw),
                                     "r"(half2_sr(ho2[i].y, ho2[i].x, dither.word(8 + i))), "l"(pol) : "memory");
                    continue;
                }
#pragma unroll
                for (int i = 1; i < 9; ++i) wd[(i - 1) * pw] = half2_sr(fo2[i].y, fo2[i].x, dither.word(i - 1));
#pragma unroll
                for (int i = 0; i < 9; ++i) wd[(8 + i) * pw] = half2_sr(ho2[i].y, ho2[i].x, dither.word(8 + i));
                continue;
            }
        }
        float fo[2][9], ho[2][9];
#pragma unroll
        for (int n = 0; n < 2; ++n) {
            if (!(n == 0 ? act0 : act1)) continue;
            float f[9], h[9];
#pragma unroll
            for (int i = 1; i < 9; ++i) f[i] = (n == 0 ? __low2float(pk[i - 1]) : __high2float(pk[i - 1])) * k.scale;
#pragma unroll
            for (int i = 0; i < 9; ++i) h[i] = (n == 0 ? __low2float(pk[8 + i]) : __high2float(pk[8 + i])) * k.scale;
            auto collide = [&](const KConst<float>& kk) {
                const FastState<float> st = fast_moments(kk, f, h, y);
                if constexpr (TAU1) fast_collide<float, true>(kk, st, f, h, fo[n], ho[n], kk.inv_scale);
                else fast_collide<float, false>(kk, st, f, h, fo[n], ho[n]);
            };
            if constexpr (EPS_FIELD) {
                KConst<float> kc = k;
                apply_eps(kc, node_eps(k, xa + n, y));
                collide(kc);
            } else {
                collide(k);
            }
        }
        if (act0 && act1) {
            const Dither dither((uint32_t)at, step);
            store_pair_half<float>(dst + at, k.plane32, fo[0], ho[0], fo[1], ho[1], out_scale, dither);
        } else {
            if (act0) {
                Dither d0((uint32_t)at, step);
                store_planes_half<float>(dst + at, k.plane32, fo[0], ho[0], out_scale, &d0);
            }
            if (act1) {
                Dither d1((uint32_t)(at + 1), step);
                store_planes_half<float>(dst + at + 1, k.plane32, fo[1], ho[1], out_scale, &d1);
            }
        }
    }
    if (!ok) {
        atomicOr(k.flag, 2);
        // let this block's copies land before its shared memory is released
        if (tid == 0)
            for (int r = yb; r < ye; ++r) (void)tma_wait(bar + (r - yb), 0u);
    }
}

// The staged step of one lattice: block (bx, by) owns band bx and a segment
// of `rows` rows.  The two segments holding the S and N wall rows (a full row
// of out-of-line wall updates each) are taken by the first two block rows,
// so that the blocks the hardware starts last are plain interior ones.
template <class S, bool EPS_FIELD, bool TAU1>
__global__ void __launch_bounds__(kTBand, TmaBlocks<S>::value)
k_step_tma(const __grid_constant__ KConst<float> k, const __grid_constant__ CUtensorMap tm,
           const S* __restrict__ src, S* __restrict__ dst, int rows, uint32_t step) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    S* stage;
    uint64_t* bar;
    staged_setup<S>(smem_raw, stage, bar);
    const int by = (int)blockIdx.y, nseg = (int)gridDim.y;
    // The two wall-row segments first; then the interior segments bottom-up
    // on even steps and top-down on odd ones, so that the first blocks of a
    // step read the rows the previous step wrote last, while they are still
    // in L2 (the order changes no value: every node depends on the previous
    // state alone).
    int seg = by == 0 ? 0 : (by == 1 ? nseg - 1 : by - 1);
#if LBM_ALT_SWEEP
    if (step & 1u) seg = by == 0 ? nseg - 1 : (by == 1 ? 0 : nseg - by);
#endif
    const int x0 = blockIdx.x * TmaLayout<S>::band, y0 = seg * rows;
    // the segments the hardware starts last (the last k.l2_hot nodes of the
    // sweep) are the rows the next step, sweeping the other way, reads first
    const bool hot = (long long)(nseg - by) * rows * k.nx <= k.l2_hot;
    __syncthreads();  // barriers initialised
    // the previous step's writes must be visible before the first copy
    asm volatile("griddepcontrol.wait;" ::: "memory");
    staged_issue_warps<S>(&tm, stage, bar, x0, y0, rows, k.ny);
    if constexpr (std::is_same<S, __half>::value)
        staged_rows_pair<EPS_FIELD, TAU1>(k, src, dst, x0, y0, rows, step, stage, bar, hot);
    else
        staged_rows<S, EPS_FIELD, TAU1>(k, src, dst, x0, y0, rows, step, stage, bar, 0u, hot);
}

// The staged step of a batch of FP32 cavities walled on all four sides: block
// i takes work item i = (cavity, band origin x0, segment origin y0, cavity
// height) of the work list.  The block copies the cavity's constants into
// shared memory; once the previous step has finished, lane 0 of each warp
// issues the copies of one row (the cavity's tensor map for the source
// buffer is read from global memory) and every thread goes on to the wall
// nodes and its rows.
__global__ void __launch_bounds__(kTBand, TmaLayout<float>::blocks)
k_step_batch_tma(const BatchCavity<float>* __restrict__ cav, const CUtensorMap* __restrict__ maps,
                 const StagedItem* __restrict__ items, const float* __restrict__ src, float* __restrict__ dst,
                 uint32_t step) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ KConst<float> ks;
    __shared__ long long off;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const StagedItem w = items[blockIdx.x];
    float* stage;
    uint64_t* bar;
    staged_setup<float>(smem_raw, stage, bar);
    // the descriptors and maps are written once, before any step: they may be
    // read before the previous step has finished
    const int* from = reinterpret_cast<const int*>(&cav[w.cavity].k);
    int* to = reinterpret_cast<int*>(&ks);
    for (int q = threadIdx.x; q < (int)(sizeof(KConst<float>) / sizeof(int)); q += kTBand) to[q] = from[q];
    if (threadIdx.x == 0) off = cav[w.cavity].offset;
    __syncthreads();  // constants, offset and barriers
    // the previous step's writes must be visible before the copies
    asm volatile("griddepcontrol.wait;" ::: "memory");
    staged_issue_warps<float>(maps + w.cavity, stage, bar, w.x0, w.y0, kTRows, w.ny);
    if (ks.omf == 0.f && ks.omT == 0.f)
        staged_rows<float, false, true>(ks, src + off, dst + off, w.x0, w.y0, kTRows, step, stage, bar);
    else
        staged_rows<float, false, false>(ks, src + off, dst + off, w.x0, w.y0, kTRows, step, stage, bar);
}

// Persistent form of the staged batch step: one cooperative launch runs
// `nsteps` steps.  Every resident block takes the work items i = blockIdx.x,
// blockIdx.x + gridDim.x, ... of the list (cavity by cavity, segment-major,
// so item first + seg * nb + band of a cavity) in the same order at every
// step.  Before it updates item i at step s it waits until the up to eight
// neighbouring items of the same cavity (bands and segments +-1) have
// completed step s - 1 (done[j] >= s): their outputs of step s - 1 are the
// values item i pulls, and their reads of step s - 1 were of the buffer item
// i now writes.  A block completes an item by a release of done[i] = s + 1
// after all its threads' stores; the waiting thread acquires it and fences
// the async proxy before it issues the tensor copies.  All blocks are
// co-resident (cooperative launch) and take their items in the same order,
// so every wait ends: an item of step s needs only items of step s - 1,
// which their blocks finish before they start step s.  The waits are
// bounded: one that gives up sets the timeout bit of the flag and the abort
// word, and every block then leaves.
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Warp 0: wait until every neighbour of item (seg, band) of a cavity laid
// out as pc has done[j] >= need.  Lane j < 9 polls neighbour (seg + j / 3 - 1,
// band + j % 3 - 1) with relaxed loads, all nine in flight together; once
// every lane sees its counter, each takes an acquire fence and the warp
// synchronises, which orders the neighbours' released stores before
// everything thread 0 does next.  False if a wait gave up or another block
// aborted (the same answer in every lane).
__device__ bool wait_neighbours(const int* done, const PersistCavity& pc, int seg, int band, int need,
                                int* abort_word) {
    const int lane = threadIdx.x & 31;
    const int sg = seg + lane / 3 - 1, bd = band + lane % 3 - 1;
    const bool mine = lane < 9 && sg >= 0 && sg < pc.ns && bd >= 0 && bd < pc.nb;
    const int* d = done + pc.first + (mine ? sg * pc.nb + bd : 0);
    const unsigned long long t0 = global_ns();
    for (long long polls = 0;; ++polls) {
        const bool seen = !mine || ld_relaxed_gpu(d) >= need;
        if (__all_sync(0xffffffffu, seen)) break;
        if ((polls & 63) == 63) {
            const bool stop = *(volatile int*)abort_word != 0 || polls > kTWaitPolls || global_ns() - t0 > kTWaitNs;
            if (__any_sync(0xffffffffu, stop)) return false;
        }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    __syncwarp();
    return true;
}

__global__ void __launch_bounds__(kTBand, TmaLayout<float>::blocks)
k_step_batch_persist(const BatchCavity<float>* __restrict__ cav, const PersistCavity* __restrict__ pcav,
                     const CUtensorMap* __restrict__ maps, const StagedItem* __restrict__ items, int n_items,
                     int n_cav, float* buf0, float* buf1, int cur, uint32_t step0, int nsteps, int* done,
                     int* abort_word, int* flag) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ KConst<float> ks;
    __shared__ long long off;
    __shared__ int go;
    float* stage;
    uint64_t* bar;
    staged_setup<float>(smem_raw, stage, bar);
    __syncthreads();  // barriers initialised
    uint32_t phases = 0u;  // current parity of each slot's barrier
    int have = -1;         // cavity whose constants are in ks
    for (int s = 0; s < nsteps; ++s) {
        const int sb = (cur + s) & 1;
        const float* src = sb ? buf1 : buf0;
        float* dst = sb ? buf0 : buf1;
        for (int i = blockIdx.x; i < n_items; i += gridDim.x) {
            const StagedItem w = items[i];
            if (threadIdx.x < 32) {
                const PersistCavity pc = pcav[w.cavity];
                const bool ok = wait_neighbours(done, pc, w.y0 / kTRows, w.x0 / kTBand, s, abort_word);
                if (threadIdx.x == 0) {
                    if (ok) {
                        // order the acquired generic-proxy writes before the copies
                        asm volatile("fence.proxy.async.global;" ::: "memory");
                        staged_issue<float>(maps + (size_t)sb * n_cav + w.cavity, stage, bar, w.x0, w.y0, kTRows,
                                            w.ny, phases);
                    } else {
                        atomicOr(flag, 2);
                        atomicExch(abort_word, 1);
                    }
                    go = ok;
                }
            }
            if (w.cavity != have) {
                const int* from = reinterpret_cast<const int*>(&cav[w.cavity].k);
                int* to = reinterpret_cast<int*>(&ks);
                for (int q = threadIdx.x; q < (int)(sizeof(KConst<float>) / sizeof(int)); q += kTBand) to[q] = from[q];
                if (threadIdx.x == 0) off = cav[w.cavity].offset;
                have = w.cavity;
            }
            __syncthreads();  // go, constants, offset
            if (!go) return;
            bool ok;
            if (ks.omf == 0.f && ks.omT == 0.f)
                ok = staged_rows<float, false, true>(ks, src + off, dst + off, w.x0, w.y0, kTRows, step0 + s, stage,
                                                     bar, phases);
            else
                ok = staged_rows<float, false, false>(ks, src + off, dst + off, w.x0, w.y0, kTRows, step0 + s, stage,
                                                      bar, phases);
            // the stores of this item become visible to the copies of the
            // blocks that pull from it at the next step
            asm volatile("fence.proxy.async.global;" ::: "memory");
            const int used = min(min(w.y0 + kTRows, w.ny), w.ny - 1) - max(w.y0, 1);  // slots armed
            phases ^= used > 0 ? ((1u << used) - 1u) : 0u;
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicExch(abort_word, 1);
                return;
            }
            if (threadIdx.x == 0) {
                __threadfence();
                st_release_gpu(done + i, s + 1);
            }
        }
    }
}

// Self-test of the bounded wait: an mbarrier that nothing arrives on, waited
// on with a 20 ms limit; the wait gives up and sets the timeout bit of the
// flag, exactly as a step whose copies never landed would.
__global__ void k_wait_selftest(int* flag) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = __syncthreads_and(tma_wait(&bar, 0u, 20000000ull));
    if (!ok && threadIdx.x == 0) atomicOr(flag, 2);
}

cudaError_t launch_wait_selftest(int* flag, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(flag);
    return cudaGetLastError();
}

template <class S> struct TmaType;
template <> struct TmaType<float> { static constexpr CUtensorMapDataType value = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; };
template <> struct TmaType<__half> { static constexpr CUtensorMapDataType value = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; };

// The tensor map of one population buffer: dims (x: nx, y: ny, plane: 17),
// box (128 + 2 halo, 1, 1), zero fill outside.
template <class S>
bool make_step_tensor_map(const KConst<float>& k, const S* buf, CUtensorMap* out) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<Encode>(fn);
    }
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    if constexpr (sizeof(S) == 2) {
        // (8 columns, column groups, rows, planes); the pitch is a multiple of
        // 64 columns, so every group of 8 up to nx rounded up lies in the row
        constexpr int g = kHInner;
        static_assert(TmaLayout<S>::box % g == 0, "FP16 boxes are whole groups of columns");
        static_assert(g * sizeof(S) % 16 == 0 && 64 % g == 0, "groups of 16-byte multiples dividing the pitch");
        const cuuint64_t dims[4] = {(cuuint64_t)g, (cuuint64_t)((k.nx + g - 1) / g), (cuuint64_t)k.ny,
                                    (cuuint64_t)NPLANES};
        const cuuint64_t strides[3] = {g * sizeof(S), (cuuint64_t)k.pitch * sizeof(S), (cuuint64_t)k.plane * sizeof(S)};
        const cuuint32_t box[4] = {(cuuint32_t)g, (cuuint32_t)(TmaLayout<S>::box / g), 1u, 1u};
        return encode(out, TmaType<S>::value, 4, const_cast<S*>(buf), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    } else {
        const cuuint64_t dims[3] = {(cuuint64_t)k.nx, (cuuint64_t)k.ny, (cuuint64_t)NPLANES};
        const cuuint64_t strides[2] = {(cuuint64_t)k.pitch * sizeof(S), (cuuint64_t)k.plane * sizeof(S)};
        const cuuint32_t box[3] = {(cuuint32_t)TmaLayout<S>::box, 1u, 1u};
        return encode(out, TmaType<S>::value, 3, const_cast<S*>(buf), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
}

bool tma_step_supported(const KConst<float>& k) {
    for (int s = 0; s < 4; ++s)
        if (k.bc[s] == BC_PERIODIC) return false;
    return k.nx >= 4 && k.ny >= 4;
}

int tma_rows_default(const KConst<float>&) { return kTRows; }

// Slots beyond the default 48 KB of dynamic shared memory need the
// function's opt-in, once per device.
template <class S, bool E, bool T>
static cudaError_t allow_tma_smem() {
    if (TmaLayout<S>::smem <= 48 * 1024) return cudaSuccess;
    constexpr int kMaxDev = 64;
    static bool done[kMaxDev] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < kMaxDev && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_step_tma<S, E, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TmaLayout<S>::smem);
    if (e == cudaSuccess && dev < kMaxDev) done[dev] = true;
    return e;
}

template <class S, bool E, bool T>
static cudaError_t launch_tma(const cudaLaunchConfig_t& cfg, const KConst<float>& k, const CUtensorMap& tm,
                              const S* src, S* dst, int rows, uint32_t step) {
    cudaError_t e = allow_tma_smem<S, E, T>();
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, k_step_tma<S, E, T>, k, tm, src, dst, rows, step);
}

template <class S>
cudaError_t launch_step_tma(const KConst<float>& k, const CUtensorMap& tm, const S* src, S* dst, int rows,
                            uint32_t step, cudaStream_t st) {
    if (rows < 1) return cudaErrorInvalidValue;
    if (rows > TmaLayout<S>::rows) rows = TmaLayout<S>::rows;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((k.nx + TmaLayout<S>::band - 1) / TmaLayout<S>::band),
                       (unsigned)((k.ny + rows - 1) / rows));
    cfg.blockDim = dim3(kTBand);
    cfg.dynamicSmemBytes = TmaLayout<S>::smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool tau1 = k.omf == 0.f && k.omT == 0.f;
    if (k.eps_field)
        return tau1 ? launch_tma<S, true, true>(cfg, k, tm, src, dst, rows, step)
                    : launch_tma<S, true, false>(cfg, k, tm, src, dst, rows, step);
    return tau1 ? launch_tma<S, false, true>(cfg, k, tm, src, dst, rows, step)
                : launch_tma<S, false, false>(cfg, k, tm, src, dst, rows, step);
}

cudaError_t launch_step_batch_tma(const BatchCavity<float>* cav, const CUtensorMap* maps, const StagedItem* items,
                                  int n_items, const float* src, float* dst, uint32_t step, cudaStream_t st) {
    if (n_items < 1) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_items);
    cfg.blockDim = dim3(kTBand);
    cfg.dynamicSmemBytes = TmaLayout<float>::smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step_batch_tma, cav, maps, items, src, dst, step);
}

cudaError_t launch_step_batch_persist(const BatchCavity<float>* cav, const PersistCavity* pcav, const CUtensorMap* maps,
                                      const StagedItem* items, int n_items, int n_cav, float* buf0, float* buf1,
                                      int cur, uint32_t step0, int nsteps, int* done, int* abort_word, int* flag,
                                      int sms, cudaStream_t st) {
    if (n_items < 1 || nsteps < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_step_batch_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TmaLayout<float>::smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_batch_persist, kTBand, TmaLayout<float>::smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    const int grid = min(n_items, per_sm * sms);
    e = cudaMemsetAsync(done, 0, (size_t)n_items * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(abort_word, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kTBand);
    cfg.dynamicSmemBytes = TmaLayout<float>::smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step_batch_persist, cav, pcav, maps, items, n_items, n_cav, buf0, buf1, cur,
                              step0, nsteps, done, abort_word, flag);
}

int tma_batch_rows() { return kTRows; }

template bool make_step_tensor_map<float>(const KConst<float>&, const float*, CUtensorMap*);
template bool make_step_tensor_map<__half>(const KConst<float>&, const __half*, CUtensorMap*);
template cudaError_t launch_step_tma<float>(const KConst<float>&, const CUtensorMap&, const float*, float*, int,
                                            uint32_t, cudaStream_t);
template cudaError_t launch_step_tma<__half>(const KConst<float>&, const CUtensorMap&, const __half*, __half*, int,
                                             uint32_t, cudaStream_t);

}  // namespace lbm
