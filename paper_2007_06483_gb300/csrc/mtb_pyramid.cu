// mtb_pyramid.cu -- the pyramid pass.
//
// One read of the interleaved RGB8 exposures produces, for every exposure:
//   * the gray image (Sec. III-A: exposures are converted to gray-scale),
//   * pyramid levels 1..tile_levels-1 (Sec. III-A: halve both dimensions, each
//     level made from the previous one as in Sec. III-B),
//   * the 256-bin histogram of each of those levels and its median (Sec. III-A,
//     Sec. III-B).
// A CTA owns runs of 32-row blocks of full-resolution pixels: 32 x 512 units
// (two 16 x 512 tiles) when the width is a multiple of 16, 32 x 256 tiles
// otherwise.  Level-l pixels of a block have their whole 2^l x 2^l source
// block inside it (l <= 5), so the block's part of levels 1..5 is built on
// chip from its gray.  HBM
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

// ---- widths that are a multiple of 16: units of 32 x 512 pixels ----
// A unit is two 16 x 512 tiles, the top one and the bottom one.  A tile row is
// 1,536 contiguous bytes of RGB, which the DRAM serves faster than the 768 of
// a 32 x 256 tile (the same reads and writes with no arithmetic: 117 against
// 125 us on 6000x4000x7).  Levels 1..4 of a tile come from the tile itself;
// level 5 (32 x 32 blocks) from the level-4 row of both tiles of the unit.
// Thread u = 32 w + 16 h + q owns the 16-pixel column group 16 (w & 1) + q of
// tile rows 2j and 2j + 1, j = 2 (w >> 1) + h: level 1 (row j) comes from its
// own registers, level 2 (row w >> 1) from one exchange with lane u ^ 16, which
// holds the same columns of rows 2 (j ^ 1) and 2 (j ^ 1) + 1.
constexpr int kWideRows = 16, kWideCols = 512;
constexpr int kUnitRows = 2 * kWideRows;
static_assert(kUnitRows == kTileRows, "a unit spans the rows of one 32-row tile row");
static_assert((kWideCols / 16) * (kWideRows / 2) == kPyrThreads, "one pair of 16-pixel groups per thread");
static_assert((kWideRows >> 2) * (kWideCols >> 2) == kLv2Bytes, "a wide tile's level 2 fills a level-2 buffer");

__device__ __forceinline__ void wide_map(int &j, int &c) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    j = 2 * (w >> 1) + (l >> 4);
    c = (16 * (w & 1) + (l & 15)) << 4;
}

__device__ __forceinline__ void wide_load_rgb(const uint8_t *__restrict__ images, const mtb_layout_t &L, int e,
                                              int y0, int x0, int rows, int cols, TileRgb &t) {
    int j, c;
    wide_map(j, c);
    const uint64_t W = (uint64_t)L.w;
    const uint64_t e0 = (uint64_t)e * W * (uint64_t)L.h;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int r = 2 * j + k;
        if (r < rows && c < cols) {
            const uint4 *src = reinterpret_cast<const uint4 *>(images + 3 * (e0 + (uint64_t)(y0 + r) * W + x0 + c));
            t.raw[k][0] = __ldcs(src);
            t.raw[k][1] = __ldcs(src + 1);
            t.raw[k][2] = __ldcs(src + 2);
        }
    }
}

// Level 0 of the thread's groups: gray, stored and counted; v gets the packed
// gray words (rows 2j, 2j + 1).  kFull: the tile lies inside the image.
template <bool kFull>
__device__ __forceinline__ void wide_level0(const TileRgb &t, const mtb_layout_t &L, uint8_t *ebase, int y0, int x0,
                                            int rows, int cols, PyrShared &sm, uint4 (&v)[2]) {
    int j, c;
    wide_map(j, c);
    uint8_t *g0 = ebase + L.gray_offset[0];
    const size_t gp0 = (size_t)L.gray_pitch[0];
    const uint32_t h0 = smem_addr(sm.h01[0][threadIdx.x >> 5]);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        uint32_t g[16];
        v[k] = gray16(t.raw[k][0], t.raw[k][1], t.raw[k][2], g);
        const int r = 2 * j + k;
        if (kFull || (r < rows && c < cols)) {
            *reinterpret_cast<uint4 *>(g0 + (size_t)(y0 + r) * gp0 + x0 + c) = v[k];
#pragma unroll
            for (int q = 0; q < 16; ++q) smem_count(h0 + 4 * g[q]);
        }
    }
}

// Levels 1 and 2 of the thread's groups from their level-0 words; level 2 also
// goes to lv2 (4 rows x 128 pixels) for the tail.  A pixel exists iff its whole
// source block does, so the level bounds cover groups that were not loaded.
template <bool kFull>
__device__ __forceinline__ void wide_levels12(const uint4 (&v)[2], const mtb_layout_t &L, uint8_t *ebase, int y0,
                                              int x0, int K, PyrShared &sm, uint8_t *lv2) {
    const int lane = threadIdx.x & 31;
    int j, c;
    wide_map(j, c);
    const int cg = c >> 4;
    const uint32_t w1a = __byte_perm(shrink2(v[0].x, v[1].x), shrink2(v[0].y, v[1].y), 0x6420u);
    const uint32_t w1b = __byte_perm(shrink2(v[0].z, v[1].z), shrink2(v[0].w, v[1].w), 0x6420u);
    {
        const int W1 = L.width[1], H1 = L.height[1];
        const int yl = (y0 >> 1) + j, xl = (x0 >> 1) + 8 * cg;
        if (kFull || (yl < H1 && xl < W1)) {
            const uint32_t h1 = smem_addr(sm.h01[1][threadIdx.x >> 5]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (kFull || xl + q < W1) smem_count(h1 + 4 * __byte_perm(w1a, 0u, 0x4440u + q));
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (kFull || xl + 4 + q < W1) smem_count(h1 + 4 * __byte_perm(w1b, 0u, 0x4440u + q));
        }
        if (kFull || (yl < H1 && xl < L.gray_pitch[1]))
            *reinterpret_cast<uint2 *>(ebase + L.gray_offset[1] + (size_t)yl * L.gray_pitch[1] + xl) =
                make_uint2(w1a, w1b);
    }
    if (K < 2) return;
    const bool top = lane < 16;
    const uint32_t recv = __shfl_xor_sync(0xffffffffu, top ? w1b : w1a, 16);
    const uint32_t w2 = __byte_perm(top ? shrink2(w1a, recv) : shrink2(recv, w1b), 0u, 0x4420u);
    const int m = threadIdx.x >> 6, xc = 4 * cg + (top ? 0 : 2);
    *reinterpret_cast<uint16_t *>(lv2 + m * (kWideCols >> 2) + xc) = (uint16_t)w2;
    const int yl = (y0 >> 2) + m, xl = (x0 >> 2) + xc;
    if (kFull || yl < L.height[2]) {
        const int W2 = L.width[2];
        const uint32_t hs = smem_addr(sm.hs[0]);
        if (kFull || xl < W2) smem_count(hs + 4 * (w2 & 0xffu));
        if (kFull || xl + 1 < W2) smem_count(hs + 4 * (w2 >> 8));
        if (kFull || xl < L.gray_pitch[2])
            *reinterpret_cast<uint16_t *>(ebase + L.gray_offset[2] + (size_t)yl * L.gray_pitch[2] + xl) = (uint16_t)w2;
    }
}

// Levels 3..5 of a tile by 4 warps (a = 0..3): lane s = 4r + c (r < 2, c < 4)
// of the 8-lane group b = 4a + (lane >> 3) makes level-3 pixel (r, c) of the
// tile's 32-column block b; lanes s = 0 and 2 add 2 x 2 of them for level 4
// (shuffles).  The top tile of a unit leaves its level-4 pixels in l4; the
// bottom tile adds them to its own for level 5 (lane s = 0).
template <bool kFull>
__device__ __forceinline__ void wide_tail(const mtb_layout_t &L, uint8_t *ebase, int y0, int x0, int K,
                                          PyrShared &sm, const uint8_t *lv2, int a, uint8_t *l4, bool bottom) {
    const int lane = threadIdx.x & 31;
    const int b = 4 * a + (lane >> 3), s = lane & 7, r = s >> 2, c = s & 3;
    constexpr int P2 = kWideCols >> 2;
    const uint32_t va = *reinterpret_cast<const uint16_t *>(lv2 + (2 * r) * P2 + 8 * b + 2 * c);
    const uint32_t vb = *reinterpret_cast<const uint16_t *>(lv2 + (2 * r + 1) * P2 + 8 * b + 2 * c);
    const uint32_t px3 = ((va & 0xffu) + (va >> 8) + (vb & 0xffu) + (vb >> 8) + 2u) >> 2;
    {
        const int yl = (y0 >> 3) + r, xl = (x0 >> 3) + 4 * b + c;
        if (kFull || yl < L.height[3]) {
            if (kFull || xl < L.width[3]) smem_count(smem_addr(sm.hs[1]) + 4 * px3);
            if (kFull || xl < L.gray_pitch[3]) ebase[L.gray_offset[3] + (size_t)yl * L.gray_pitch[3] + xl] = (uint8_t)px3;
        }
    }
    if (K < 4) return;
    const uint32_t s1 = px3 + __shfl_down_sync(0xffffffffu, px3, 1);
    const uint32_t s2 = s1 + __shfl_down_sync(0xffffffffu, s1, 4);
    const uint32_t px4 = (s2 + 2u) >> 2;  // valid at s = 0 (columns 0, 1) and s = 2 (2, 3)
    {
        const int yl = y0 >> 4, xl = (x0 >> 4) + 2 * b + (c >> 1);
        if ((s & 5) == 0 && (kFull || yl < L.height[4])) {
            if (kFull || xl < L.width[4]) smem_count(smem_addr(sm.hs[2]) + 4 * px4);
            if (kFull || xl < L.gray_pitch[4]) ebase[L.gray_offset[4] + (size_t)yl * L.gray_pitch[4] + xl] = (uint8_t)px4;
        }
    }
    if (K < 5) return;
    const uint32_t p4n = __shfl_down_sync(0xffffffffu, px4, 2);  // at s = 0: the level-4 pixel of columns 2, 3
    if (!bottom) {
        if (s == 0) *reinterpret_cast<uint16_t *>(l4 + 2 * b) = (uint16_t)(px4 | (p4n << 8));
        return;
    }
    const uint32_t t4 = *reinterpret_cast<const uint16_t *>(l4 + 2 * b);
    const uint32_t px5 = ((t4 & 0xffu) + (t4 >> 8) + px4 + p4n + 2u) >> 2;
    const int yl = y0 >> 5, xl = (x0 >> 5) + b;
    if (s == 0 && (kFull || yl < L.height[5])) {
        if (kFull || xl < L.width[5]) smem_count(smem_addr(sm.hs[3]) + 4 * px5);
        if (kFull || xl < L.gray_pitch[5]) ebase[L.gray_offset[5] + (size_t)yl * L.gray_pitch[5] + xl] = (uint8_t)px5;
    }
}

// Position of the k-th tile of a run of units: unit (e, uy, ux), half (0 top,
// 1 bottom), advanced one tile at a time (a unit whose bottom tile lies below
// the image has only its top tile).
struct WideCursor {
    int e, uy, ux, half;
    __device__ __forceinline__ void init(int u, int units_x, int units_per_exp) {
        e = u / units_per_exp;
        const int ru = u - e * units_per_exp;
        uy = ru / units_x;
        ux = ru - uy * units_x;
        half = 0;
    }
    __device__ __forceinline__ int y0() const { return uy * kUnitRows + half * kWideRows; }
    __device__ __forceinline__ int x0() const { return ux * kWideCols; }
    // to the next tile: the bottom tile of this unit when it lies inside the
    // image, else the top tile of the next unit (*u counts the units)
    __device__ __forceinline__ void next(int units_x, int units_y, int h, int *u) {
        if (half == 0 && uy * kUnitRows + kWideRows < h) {
            half = 1;
            return;
        }
        half = 0;
        ++*u;
        if (++ux == units_x) {
            ux = 0;
            if (++uy == units_y) {
                uy = 0;
                ++e;
            }
        }
    }
};

// Widths that are a multiple of 16.  A CTA takes a contiguous run of units,
// top tile then bottom tile.  Once level 0 of the current tile has consumed its
// RGB, the next tile's RGB is loaded into the same registers (3 CTAs per SM
// leave room for it) and stays in flight while levels 1..2 are built; after
// the tile's one barrier, levels 3..5 are built by half of the warps
// (alternating with the tile, from one of two level-2 buffers) while the
// others go on.
__device__ __forceinline__ void pyramid_aligned(const uint8_t *__restrict__ images, const mtb_layout_t &L,
                                                uint8_t *__restrict__ ws, int units_x, int units_per_exp, int u0,
                                                int u1, PyrShared &sm, uint8_t *l4) {
    const int K = L.tile_levels - 1;
    const int units_y = units_per_exp / units_x;
    WideCursor cc, nc;
    cc.init(u0, units_x, units_per_exp);
    nc = cc;
    int u = u0, un = u0;  // unit of the current tile, of the next one
    TileRgb cur, nxt;
    if (u0 < u1) {
        const int y0 = cc.y0(), x0 = cc.x0();
        wide_load_rgb(images, L, cc.e, y0, x0, min(kWideRows, L.h - y0), min(kWideCols, L.w - x0), cur);
    }
    int cur_e = -1, done = 0, i = 0;
    bool waited = false;
    uint8_t *ebase = ws;
    while (u < u1) {
        const int e = cc.e, y0 = cc.y0(), x0 = cc.x0();
        const bool bottom = cc.half == 1;
        if (e != cur_e) {
            if (cur_e >= 0) {
                if (!waited) pdl_wait();  // the histograms were cleared by the previous kernel
                waited = true;
                flush_exposure(L, ws, cur_e, done, units_per_exp, K, sm);
            }
            cur_e = e;
            done = 0;
            ebase = ws + (size_t)e * L.gray_exposure_stride;
        }
        const int rows = min(kWideRows, L.h - y0);
        const int cols = min(kWideCols, L.w - x0);
        const bool full = rows == kWideRows && cols == kWideCols;
        uint8_t *lv2 = sm.lv + (i & 1) * kLv2Bytes;
        uint4 v[2];
        if (full) wide_level0<true>(cur, L, ebase, y0, x0, rows, cols, sm, v);
        else wide_level0<false>(cur, L, ebase, y0, x0, rows, cols, sm, v);
        // the current tile's RGB is consumed: its registers take the next one,
        // in flight while levels 1..2 are built
        nc.next(units_x, units_y, L.h, &un);
        if (un < u1) {
            const int y1 = nc.y0(), x1 = nc.x0();
            wide_load_rgb(images, L, nc.e, y1, x1, min(kWideRows, L.h - y1), min(kWideCols, L.w - x1), nxt);
        }
        if (K >= 1) {
            if (full) wide_levels12<true>(v, L, ebase, y0, x0, K, sm, lv2);
            else wide_levels12<false>(v, L, ebase, y0, x0, K, sm, lv2);
        }
        __syncthreads();  // level 2 of the tile is in lv2 (and the top tile's level 4 in l4)
        // lv2 is written again two tiles later, and l4 by the next unit's top
        // tile, after the next barrier, which every warp passes only after its
        // share of this tile's tail
        const int a = (threadIdx.x >> 5) - ((i & 1) ? 4 : 0);
        if (K >= 3 && a >= 0 && a < 4) {
            if (full) wide_tail<true>(L, ebase, y0, x0, K, sm, lv2, a, l4, bottom);
            else wide_tail<false>(L, ebase, y0, x0, K, sm, lv2, a, l4, bottom);
        }
        if (un != u) ++done;  // the unit's last tile
        u = un;
        cur = nxt;
        cc = nc;
        ++i;
    }
    if (cur_e >= 0) {
        if (!waited) pdl_wait();
        flush_exposure(L, ws, cur_e, done, units_per_exp, K, sm);
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
    __shared__ alignas(16) uint8_t l4[2 * (kWideCols >> 5)];  // a unit's top level-4 row (aligned form)
    const int tid = threadIdx.x;
    for (int v = tid; v < 2 * kPyrWarps * 256; v += kPyrThreads) (&sm.h01[0][0][0])[v] = 0;
    for (int v = tid; v < (kTileLog2 - 1) * 256; v += kPyrThreads) (&sm.hs[0][0])[v] = 0;
    __syncthreads();

    pdl_trigger();
    // tiles [tile_begin, tile_begin + tile_count) of the stack (all of them, or
    // the rows of one exposure whose copy has landed), split into runs
    const int t0 = tile_begin + (int)(((long long)blockIdx.x * tile_count) / gridDim.x);
    const int t1 = tile_begin + (int)(((long long)(blockIdx.x + 1) * tile_count) / gridDim.x);
    if (kAligned) pyramid_aligned(images, L, ws, tiles_x, tiles_per_exp, t0, t1, sm, l4);
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

int pyramid_tiles_x(const mtb_layout_t &L) {
    return (L.w % 16) == 0 ? (L.w + kWideCols - 1) / kWideCols : (L.w + kTileCols - 1) / kTileCols;
}

long long pyramid_tiles_per_exposure(const mtb_layout_t &L) {
    return (long long)pyramid_tiles_x(L) * ((L.h + kTileRows - 1) / kTileRows);
}

cudaError_t launch_pyramid_range(const uint8_t *images, const mtb_layout_t &L, uint8_t *ws, long long tile_begin,
                                 long long tile_end, cudaStream_t s, bool chained) {
    const int tiles_x = pyramid_tiles_x(L);
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
