// mtb_pyramid.cu -- the pyramid pass.
//
// One read of the interleaved RGB8 exposures produces, for every exposure:
//   * the gray image (Sec. III-A: exposures are converted to gray-scale),
//   * pyramid levels 1..tile_levels-1 (Sec. III-A: halve both dimensions, each
//     level made from the previous one as in Sec. III-B),
//   * the 256-bin histogram of each of those levels and its median (Sec. III-A,
//     Sec. III-B).
// A CTA owns 32-row x 256-column tiles of full-resolution pixels.  Level-l
// pixels of a tile have their whole 2^l x 2^l source block inside it (l <= 5),
// so the tile's part of levels 1..5 is built on chip from the gray tile.  HBM
// traffic per full-resolution pixel: 3 bytes read (RGB) + 4/3 bytes written
// (gray levels).
//
// Instruction budget: at HBM speed the pass has about 17 thread-instructions per
// pixel, so the gray conversion uses two two-way dot products per pixel on the
// RGB words as loaded, gray is packed with byte permutes, the 2x2 shrink is
// done on 16-bit lanes, histogram counts are shared-memory reductions on
// 32-bit shared addresses, and (widths a multiple of 16) levels 1..5 come from
// registers and warp shuffles rather than shared-memory round trips.
#include "mtb_pyramid_dev.cuh"

namespace mtb {
namespace {

// Widths that are a multiple of 16.  Once level 0 of the current tile has
// consumed its RGB, the next tile's RGB is loaded into the same registers (3
// CTAs per SM leave room for it) and stays in flight while levels 1..5 are
// built; after the tile's one barrier, levels 3..5 are built by half of the
// warps (alternating with the tile, from one of two level-2 buffers) while the
// others go on.
__device__ __forceinline__ void pyramid_aligned(const uint8_t *__restrict__ images, const mtb_layout_t &L,
                                                uint8_t *__restrict__ ws, int tiles_x, int tiles_per_exp, int t0,
                                                int t1, PyrShared &sm) {
    const int K = L.tile_levels - 1;
    const int tiles_y = tiles_per_exp / tiles_x;
    TileCursor cc, nc;
    cc.init(t0, tiles_x, tiles_per_exp);
    nc = cc;
    TileRgb cur, nxt;
    if (t0 < t1) {
        const int y0 = cc.ty * kTileRows, x0 = cc.tx * kTileCols;
        tile_load_rgb(images, L, cc.e, y0, x0, min(kTileRows, L.h - y0), min(kTileCols, L.w - x0), cur);
    }
    int cur_e = -1, done = 0;
    bool waited = false;
    uint8_t *ebase = ws;
    for (int t = t0; t < t1; ++t) {
        const int e = cc.e, y0 = cc.ty * kTileRows, x0 = cc.tx * kTileCols;
        if (e != cur_e) {
            if (cur_e >= 0) {
                if (!waited) pdl_wait();  // the histograms were cleared by the previous kernel
                waited = true;
                flush_exposure(L, ws, cur_e, done, tiles_per_exp, K, sm);
            }
            cur_e = e;
            done = 0;
            ebase = ws + (size_t)e * L.gray_exposure_stride;
        }
        const int rows = min(kTileRows, L.h - y0);
        const int cols = min(kTileCols, L.w - x0);
        const bool full = rows == kTileRows && cols == kTileCols;
        uint8_t *lv2 = sm.lv + ((t - t0) & 1) * kLv2Bytes;
        uint4 v[2];
        if (full) tile_level0<true>(cur, L, ebase, y0, x0, rows, cols, sm, v);
        else tile_level0<false>(cur, L, ebase, y0, x0, rows, cols, sm, v);
        // the current tile's RGB is consumed: its registers take the next one,
        // in flight while levels 1..5 are built
        nc.next(tiles_x, tiles_y);
        if (t + 1 < t1) {
            const int y1 = nc.ty * kTileRows, x1 = nc.tx * kTileCols;
            tile_load_rgb(images, L, nc.e, y1, x1, min(kTileRows, L.h - y1), min(kTileCols, L.w - x1), nxt);
        }
        if (K >= 1) {
            if (full) tile_levels12_pair<true>(v, L, ebase, y0, x0, K, sm, lv2);
            else tile_levels12_pair<false>(v, L, ebase, y0, x0, K, sm, lv2);
        }
        __syncthreads();  // level 2 of the tile is in lv2
        // lv2 is written again two tiles later, after the next barrier, which
        // every warp passes only after its share of this tile's tail
        const int a = (threadIdx.x >> 5) - (((t - t0) & 1) ? 4 : 0);
        if (K >= 3 && a >= 0 && a < 4) {
            if (full) tile_tail<true>(L, ebase, y0, x0, K, sm, lv2, a);
            else tile_tail<false>(L, ebase, y0, x0, K, sm, lv2, a);
        }
        ++done;
        cur = nxt;
        cc = nc;
    }
    if (cur_e >= 0) {
        if (!waited) pdl_wait();
        flush_exposure(L, ws, cur_e, done, tiles_per_exp, K, sm);
    }
}

// Any width: level 0 of each tile through shared memory (groups clipped to the
// rows' pixel runs), then levels 1..5 from it.
__device__ __forceinline__ void pyramid_general(const uint8_t *__restrict__ images, const mtb_layout_t &L,
                                                uint8_t *__restrict__ ws, int tiles_x, int tiles_per_exp, int t0,
                                                int t1, PyrShared &sm) {
    const int K = L.tile_levels - 1;
    int cur_e = -1, done = 0;
    bool waited = false;
    for (int t = t0; t < t1; ++t) {
        const int e = t / tiles_per_exp;
        const int rt = t - e * tiles_per_exp;
        const int ty = rt / tiles_x;
        const int y0 = ty * kTileRows, x0 = (rt - ty * tiles_x) * kTileCols;
        if (e != cur_e) {
            if (cur_e >= 0) {
                if (!waited) pdl_wait();
                waited = true;
                flush_exposure(L, ws, cur_e, done, tiles_per_exp, K, sm);
            }
            cur_e = e;
            done = 0;
        }
        const int rows = min(kTileRows, L.h - y0);
        const int cols = min(kTileCols, L.w - x0);
        tile_level0_general(images, L, ws, e, y0, x0, rows, cols, sm);
        __syncthreads();
        tile_store_level0(L, ws, e, y0, x0, rows, cols, sm);
        if (K >= 1) tile_levels12(L, ws, e, y0, x0, K, sm);
        __syncthreads();
        // levels 3..5, a 32-column block per warp; the next tile's level 0 only
        // writes level 0 of the shared buffer
        if (K >= 3) tile_block_tail(L, ws, e, y0, x0, K, sm);
        ++done;
    }
    if (cur_e >= 0) {
        if (!waited) pdl_wait();
        flush_exposure(L, ws, cur_e, done, tiles_per_exp, K, sm);
    }
}

template <bool kAligned>
__global__ void __launch_bounds__(kPyrThreads, kAligned ? 3 : 4)
k_pyramid(const uint8_t *__restrict__ images, const mtb_layout_t L, uint8_t *__restrict__ ws, int tiles_x,
          int tiles_per_exp, int tile_begin, int tile_count) {
    static_assert(kPyrThreads == 256, "one thread per histogram bin in the flush");
    static_assert(2 * kLv2Bytes <= kLvBytes, "two level-2 buffers fit the shared level buffer");
    __shared__ PyrShared sm;
    const int tid = threadIdx.x;
    for (int v = tid; v < 2 * kPyrWarps * 256; v += kPyrThreads) (&sm.h01[0][0][0])[v] = 0;
    for (int v = tid; v < (kTileLog2 - 1) * 256; v += kPyrThreads) (&sm.hs[0][0])[v] = 0;
    __syncthreads();

    pdl_trigger();
    // tiles [tile_begin, tile_begin + tile_count) of the stack (all of them, or
    // the rows of one exposure whose copy has landed), split into runs
    const int t0 = tile_begin + (int)(((long long)blockIdx.x * tile_count) / gridDim.x);
    const int t1 = tile_begin + (int)(((long long)(blockIdx.x + 1) * tile_count) / gridDim.x);
    if (kAligned) pyramid_aligned(images, L, ws, tiles_x, tiles_per_exp, t0, t1, sm);
    else pyramid_general(images, L, ws, tiles_x, tiles_per_exp, t0, t1, sm);
}

// Clears n 32-bit words (the histograms and counters of a stack).  Launched
// chained behind whatever the stream ran before (usually the previous call's
// search), so its launch overlaps that kernel's end; it waits for it before
// it lets the pyramid pass start, because the pyramid pass writes gray planes
// that the previous call's bitmap pass may still read.  The pyramid pass in
// turn writes only gray planes, nothing cleared here, before its own wait.
__global__ void k_clear(uint32_t *p, int n) {
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0;
}

int g_pyr_blocks_per_sm[2] = {0, 0};

}  // namespace

cudaError_t launch_clear_stack(const mtb_layout_t &L, uint8_t *ws, cudaStream_t s) {
    // everything after the bit planes (histograms, counters, errors, medians,
    // bases, shifts, window tables, status) is small and adjacent: one launch
    // clears it, so that a search chained to this pyramid needs no clearing of
    // its own and can start while the bitmaps are still being packed
    const long long words = (long long)(L.total_bytes - L.hist_offset) / 4;
    const long long cap = 4ll * device_sm_count();
    const long long blocks = (words + 1023) / 1024 < cap ? (words + 1023) / 1024 : cap;
    if (words > 0x7fffffffLL) return cudaErrorInvalidValue;
    return launch_k(k_clear, dim3((unsigned)blocks), dim3(256), s, true,
                    reinterpret_cast<uint32_t *>(ws + L.hist_offset), (int)words);
}

long long pyramid_tiles_per_exposure(const mtb_layout_t &L) {
    return (long long)((L.w + kTileCols - 1) / kTileCols) * ((L.h + kTileRows - 1) / kTileRows);
}

cudaError_t launch_pyramid_range(const uint8_t *images, const mtb_layout_t &L, uint8_t *ws, long long tile_begin,
                                 long long tile_end, cudaStream_t s, bool chained) {
    const int tiles_x = (L.w + kTileCols - 1) / kTileCols;
    const long long per_exp = pyramid_tiles_per_exposure(L);
    const long long total = per_exp * L.n;
    if (total > 0x7fffffffLL || tile_begin < 0 || tile_end > total || tile_begin >= tile_end)
        return cudaErrorInvalidValue;
    const bool aligned = (L.w % 16) == 0;
    int &nb = g_pyr_blocks_per_sm[aligned ? 1 : 0];
    if (nb == 0) {
        int v = 0;
        const cudaError_t err =
            aligned ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_pyramid<true>, kPyrThreads, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_pyramid<false>, kPyrThreads, 0);
        if (err != cudaSuccess) return err;
        nb = v > 0 ? v : 1;
    }
    const long long count = tile_end - tile_begin;
    const long long cap_p = (long long)device_sm_count() * nb;
    const int grid = (int)(count < cap_p ? count : cap_p);
    if (aligned)
        return launch_k(k_pyramid<true>, dim3(grid), dim3(kPyrThreads), s, chained, images, L, ws, tiles_x,
                        (int)per_exp, (int)tile_begin, (int)count);
    return launch_k(k_pyramid<false>, dim3(grid), dim3(kPyrThreads), s, chained, images, L, ws, tiles_x,
                    (int)per_exp, (int)tile_begin, (int)count);
}

cudaError_t launch_pyramid(const uint8_t *images, const mtb_layout_t &L, uint8_t *ws, cudaStream_t s) {
    const cudaError_t err = launch_clear_stack(L, ws, s);
    if (err != cudaSuccess) return err;
    return launch_pyramid_range(images, L, ws, 0, pyramid_tiles_per_exposure(L) * L.n, s, true);
}

}  // namespace mtb
