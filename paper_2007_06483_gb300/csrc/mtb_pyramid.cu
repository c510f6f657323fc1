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
// so the tile's part of levels 1..5 is built in shared memory from the gray
// tile.  HBM traffic per full-resolution pixel: 3 bytes read (RGB) + 4/3 bytes
// written (gray levels).
//
// Instruction budget: at HBM speed the pass has about 17 thread-instructions per
// pixel, so the gray conversion uses two two-way dot products per pixel on the
// RGB words as loaded, gray is packed with byte permutes, the 2x2 shrink is
// done on 16-bit lanes, and a 16-pixel group of one value adds to the histogram
// with a single shared atomic (saturated regions would otherwise serialise 32
// lanes on one bin).
#include "mtb_pyramid_dev.cuh"

namespace mtb {
namespace {

// kAligned (W a multiple of 16): the RGB of tile t+1 is loaded into registers
// while the CTA builds levels 1..5 of tile t (3 CTAs per SM leave room for it).
template <bool kAligned>
__global__ void __launch_bounds__(kPyrThreads, kAligned ? 3 : 4)
k_pyramid(const uint8_t *__restrict__ images, const mtb_layout_t L, uint8_t *__restrict__ ws, int tiles_x,
          int tiles_per_exp, int total_tiles) {
    static_assert(kPyrThreads == 256, "one thread per histogram bin in the flush");
    __shared__ PyrShared sm;
    const int tid = threadIdx.x;
    const int K = L.tile_levels - 1;
    for (int v = tid; v < 2 * kPyrWarps * 256; v += kPyrThreads) (&sm.h01[0][0][0])[v] = 0;
    for (int v = tid; v < (kTileLog2 - 1) * 256; v += kPyrThreads) (&sm.hs[0][0])[v] = 0;
    __syncthreads();

    pdl_trigger();
    const int t0 = (int)(((long long)blockIdx.x * total_tiles) / gridDim.x);
    const int t1 = (int)(((long long)(blockIdx.x + 1) * total_tiles) / gridDim.x);
    auto origin = [&](int t, int *e, int *y0, int *x0) {
        *e = t / tiles_per_exp;
        const int rt = t - *e * tiles_per_exp;
        const int ty = rt / tiles_x;
        *y0 = ty * kTileRows;
        *x0 = (rt - ty * tiles_x) * kTileCols;
    };
    TileRgb cur, nxt;
    if (kAligned && t0 < t1) {
        int e, y0, x0;
        origin(t0, &e, &y0, &x0);
        tile_load_rgb(images, L, e, y0, x0, min(kTileRows, L.h - y0), min(kTileCols, L.w - x0), cur);
    }
    int cur_e = -1, done = 0;
    bool waited = false;
    for (int t = t0; t < t1; ++t) {
        int e, y0, x0;
        origin(t, &e, &y0, &x0);
        if (e != cur_e) {
            if (cur_e >= 0) {
                if (!waited) pdl_wait();  // the histograms were cleared by the previous kernel
                waited = true;
                flush_exposure(L, ws, cur_e, done, tiles_per_exp, K, sm);
            }
            cur_e = e;
            done = 0;
        }
        const int rows = min(kTileRows, L.h - y0);
        const int cols = min(kTileCols, L.w - x0);
        if (kAligned) {
            tile_level0_loaded(cur, L, ws, e, y0, x0, rows, cols, sm);
            if (t + 1 < t1) {  // in flight while levels 1..5 of this tile are built
                int e1, y1, x1;
                origin(t + 1, &e1, &y1, &x1);
                tile_load_rgb(images, L, e1, y1, x1, min(kTileRows, L.h - y1), min(kTileCols, L.w - x1), nxt);
            }
        } else {
            tile_level0_general(images, L, ws, e, y0, x0, rows, cols, sm);
        }
        __syncthreads();
        if (!kAligned) tile_store_level0(L, ws, e, y0, x0, rows, cols, sm);
        if (K >= 1) tile_levels12(L, ws, e, y0, x0, K, sm);
        __syncthreads();
        // levels 3..5, a 32-column block per warp; the next tile's level 0 only
        // writes level 0 of the shared buffer
        if (K >= 3) tile_block_tail(L, ws, e, y0, x0, K, sm);
        ++done;
        if (kAligned) cur = nxt;
    }
    if (cur_e >= 0) {
        if (!waited) pdl_wait();
        flush_exposure(L, ws, cur_e, done, tiles_per_exp, K, sm);
    }
}

// Clears n 32-bit words (the histograms and counters of a stack).
__global__ void k_clear(uint32_t *p, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0;
}

int g_pyr_blocks_per_sm[2] = {0, 0};

}  // namespace

cudaError_t launch_pyramid(const uint8_t *images, const mtb_layout_t &L, uint8_t *ws, cudaStream_t s) {
    const int tiles_x = (L.w + kTileCols - 1) / kTileCols;
    const int tiles_y = (L.h + kTileRows - 1) / kTileRows;
    const long long per_exp = (long long)tiles_x * tiles_y;
    const long long total = per_exp * L.n;
    if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
    // everything after the bit planes (histograms, counters, errors, medians,
    // bases, shifts, window tables, status) is small and adjacent: one launch
    // clears it, so that a search chained to this pyramid needs no clearing of
    // its own and can start while the bitmaps are still being packed
    const long long words = (long long)(L.total_bytes - L.hist_offset) / 4;
    const long long cap = 4ll * device_sm_count();
    const long long blocks = (words + 1023) / 1024 < cap ? (words + 1023) / 1024 : cap;
    if (words > 0x7fffffffLL) return cudaErrorInvalidValue;
    cudaError_t err = launch_k(k_clear, dim3((unsigned)blocks), dim3(256), s, false,
                               reinterpret_cast<uint32_t *>(ws + L.hist_offset), (int)words);
    if (err != cudaSuccess) return err;
    const bool aligned = (L.w % 16) == 0;
    int &nb = g_pyr_blocks_per_sm[aligned ? 1 : 0];
    if (nb == 0) {
        int v = 0;
        err = aligned ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_pyramid<true>, kPyrThreads, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_pyramid<false>, kPyrThreads, 0);
        if (err != cudaSuccess) return err;
        nb = v > 0 ? v : 1;
    }
    const long long cap_p = (long long)device_sm_count() * nb;
    const int grid = (int)(total < cap_p ? total : cap_p);
    if (aligned)
        return launch_k(k_pyramid<true>, dim3(grid), dim3(kPyrThreads), s, true, images, L, ws, tiles_x, (int)per_exp,
                        (int)total);
    return launch_k(k_pyramid<false>, dim3(grid), dim3(kPyrThreads), s, true, images, L, ws, tiles_x, (int)per_exp,
                    (int)total);
}

}  // namespace mtb
