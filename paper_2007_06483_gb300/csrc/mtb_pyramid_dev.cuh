// mtb_pyramid_dev.cuh -- device functions of the pyramid pass (gray, levels
// 1..5 of a tile, histograms, medians), shared by the stage kernel and the
// engine.
#pragma once

#include "mtb_device.cuh"

namespace mtb {
namespace {

// Offset of level l's tile inside the shared level buffer.
__host__ __device__ constexpr int lv_offset(int l) {
    int off = 0;
    for (int k = 0; k < l; ++k) off += (kTileRows >> k) * (kTileCols >> k);
    return off;
}
constexpr int kLvBytes = lv_offset(kTileLog2 + 1);

struct PyrShared {
    alignas(16) uint8_t lv[kLvBytes];
    uint32_t h01[2][kPyrWarps][256];  // warp-private, levels 0 and 1
    uint32_t hs[kTileLog2 - 1][256];  // levels 2..5, one per CTA
    int last;
};

// 4 pixels = 12 RGB bytes in words w0..w2 -> their gray values and the packed
// word, by two-way dot products (16-bit weights times 2 bytes),
// with the weights and rounding term scaled by 4: 4 * (4899 R + 9617 G +
// 1868 B + 8192) < 2^24, and its byte 2 is (4899 R + 9617 G + 1868 B + 8192)
// >> 14, so the gray value is read off byte 2 with no shift.  Each pixel's
// three bytes are addressed where they lie (bytes 0..2, 3..5, 6..8, 9..11).
constexpr uint32_t kRG4 = (4899u * 4) | ((9617u * 4) << 16), kGB4 = (9617u * 4) | ((1868u * 4) << 16);
constexpr uint32_t kB04 = 1868u * 4, k0R4 = (4899u * 4) << 16, kBias4 = 8192u * 4;
__device__ __forceinline__ uint32_t gray4_dp2(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t *g) {
    const uint32_t p0 = __dp2a_hi(kB04, w0, __dp2a_lo(kRG4, w0, kBias4));  // R G | B .
    const uint32_t p1 = __dp2a_hi(k0R4, w0, __dp2a_lo(kGB4, w1, kBias4));  // . R | G B
    const uint32_t p2 = __dp2a_lo(kB04, w2, __dp2a_hi(kRG4, w1, kBias4));  // R G | B .
    const uint32_t p3 = __dp2a_hi(kGB4, w2, __dp2a_lo(k0R4, w2, kBias4));  // . R | G B
    g[0] = __byte_perm(p0, 0u, 0x4442u);
    g[1] = __byte_perm(p1, 0u, 0x4442u);
    g[2] = __byte_perm(p2, 0u, 0x4442u);
    g[3] = __byte_perm(p3, 0u, 0x4442u);
    return __byte_perm(__byte_perm(p0, p1, 0x7362u), __byte_perm(p2, p3, 0x7362u), 0x5410u);
}

// 16 pixels of one 48-byte group -> gray values and 4 packed words.
__device__ __forceinline__ uint4 gray16(const uint4 &a, const uint4 &b, const uint4 &c, uint32_t (&g)[16]) {
    uint4 v;
    v.x = gray4_dp2(a.x, a.y, a.z, g + 0);
    v.y = gray4_dp2(a.w, b.x, b.y, g + 4);
    v.z = gray4_dp2(b.z, b.w, c.x, g + 8);
    v.w = gray4_dp2(c.y, c.z, c.w, g + 12);
    return v;
}

// Histogram of a group's pixels q in [qa, qb); one atomic if all 16 are equal.
__device__ __forceinline__ void hist_group(uint32_t *h, const uint32_t (&g)[16], const uint4 &v, int qa, int qb) {
    const uint32_t b0 = __byte_perm(v.x, 0u, 0x0000u);
    if (qa == 0 && qb == 16 && v.x == b0 && v.y == b0 && v.z == b0 && v.w == b0) {
        atomicAdd(h + g[0], 16u);
        return;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q)
        if (q >= qa && q < qb) atomicAdd(h + g[q], 1u);
}

// Two shrunk pixels (16-bit lanes) from 4 pixels of each of two rows.
__device__ __forceinline__ uint32_t shrink2(uint32_t a, uint32_t b) {
    const uint32_t s = __byte_perm(a, 0u, 0x4240u) + __byte_perm(a, 0u, 0x4341u) + __byte_perm(b, 0u, 0x4240u) +
                       __byte_perm(b, 0u, 0x4341u) + 0x00020002u;
    return (s >> 2) & 0x00ff00ffu;
}

// ---- widths that are a multiple of 16 ----
// Thread u of the CTA owns the 16-pixel column group cg = u % 16 of tile rows
// 2j and 2j + 1 (j = u / 16): level 1 (row j, 8 pixels) comes from its own
// registers, level 2 (row j / 2 = the warp) from one exchange with lane u ^ 16,
// and levels 3..5 from shuffles inside a warp, so no level between 0 and 2
// passes through shared memory and a tile needs one CTA barrier.

// The RGB of the thread's two groups (2 x 48 bytes), loaded one tile ahead.
struct TileRgb {
    uint4 raw[2][3];
};

__device__ __forceinline__ void tile_load_rgb(const uint8_t *__restrict__ images, const mtb_layout_t &L, int e,
                                              int y0, int x0, int rows, int cols, TileRgb &t) {
    const int tid = threadIdx.x;
    const int j = tid >> 4, c = (tid & 15) << 4;
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

// Adds 1 to the shared-memory counter at 32-bit shared address `addr`.
__device__ __forceinline__ void smem_count(uint32_t addr) {
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

constexpr int kLv2Bytes = (kTileRows >> 2) * (kTileCols >> 2);  // level 2 of one tile: 8 x 64

// Level 0 of the thread's groups: gray, stored and counted; v gets the packed
// gray words (row 2j, row 2j + 1) for levels 1 and 2.  `ebase`: exposure e's
// base in the workspace (plane l at ebase + gray_offset[l]).  kFull: the tile
// lies inside the image, so is every pixel of its levels 1..5 (2^5 divides the
// tile's sides), and no bound is checked.
template <bool kFull>
__device__ __forceinline__ void tile_level0(const TileRgb &t, const mtb_layout_t &L, uint8_t *ebase, int y0, int x0,
                                            int rows, int cols, PyrShared &sm, uint4 (&v)[2]) {
    const int tid = threadIdx.x;
    const int j = tid >> 4, c = (tid & 15) << 4;
    uint8_t *g0 = ebase + L.gray_offset[0];
    const size_t gp0 = (size_t)L.gray_pitch[0];
    const uint32_t h0 = smem_addr(sm.h01[0][tid >> 5]);
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

// Levels 1 and 2 of the thread's groups from their level-0 words v; level 2
// also goes to lv2 for the tail.
template <bool kFull>
__device__ __forceinline__ void tile_levels12_pair(const uint4 (&v)[2], const mtb_layout_t &L, uint8_t *ebase,
                                                   int y0, int x0, int K, PyrShared &sm, uint8_t *lv2) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int j = tid >> 4, cg = tid & 15;
    // level 1, row j, columns 8cg..8cg+7 (a pixel exists iff both its rows and
    // both its columns do, so the level-1 bounds cover the garbage of groups
    // that were not loaded)
    const uint32_t w1a = __byte_perm(shrink2(v[0].x, v[1].x), shrink2(v[0].y, v[1].y), 0x6420u);
    const uint32_t w1b = __byte_perm(shrink2(v[0].z, v[1].z), shrink2(v[0].w, v[1].w), 0x6420u);
    {
        const int W1 = L.width[1], H1 = L.height[1];
        const int yl = (y0 >> 1) + j, xl = (x0 >> 1) + 8 * cg;
        if (kFull || (yl < H1 && xl < W1)) {
            const uint32_t h1 = smem_addr(sm.h01[1][tid >> 5]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (kFull || xl + q < W1) smem_count(h1 + 4 * __byte_perm(w1a, 0u, 0x4440u + q));
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (kFull || xl + 4 + q < W1) smem_count(h1 + 4 * __byte_perm(w1b, 0u, 0x4440u + q));
        }
        if (kFull || (yl < H1 && xl < L.gray_pitch[1]))  // 8 bytes inside the pitch (a multiple of 32)
            *reinterpret_cast<uint2 *>(ebase + L.gray_offset[1] + (size_t)yl * L.gray_pitch[1] + xl) =
                make_uint2(w1a, w1b);
    }
    if (K < 2) return;
    // level 2, row m = warp: the top lane (level-1 row 2m) makes columns 4cg
    // and 4cg + 1 from the first halves of both rows, the bottom lane 4cg + 2
    // and 4cg + 3 from the second halves
    const bool top = lane < 16;
    const uint32_t recv = __shfl_xor_sync(0xffffffffu, top ? w1b : w1a, 16);
    const uint32_t w2 = __byte_perm(top ? shrink2(w1a, recv) : shrink2(recv, w1b), 0u, 0x4420u);
    const int m = tid >> 5, xc = 4 * cg + (top ? 0 : 2);
    *reinterpret_cast<uint16_t *>(lv2 + m * (kTileCols >> 2) + xc) = (uint16_t)w2;
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

// Levels 3..K of the tile from lv2 by 4 warps: warp a (0..3) of the group
// takes the 32-column blocks 2a (lanes 0-15) and 2a + 1 (lanes 16-31); lane
// q = 4r + c of a half makes level-3 pixel (r, c) of its block, lanes with r
// and c even add the 2x2 for level 4 by shuffles, lane 0 of the half level 5.
template <bool kFull>
__device__ __forceinline__ void tile_tail(const mtb_layout_t &L, uint8_t *ebase, int y0, int x0, int K,
                                          PyrShared &sm, const uint8_t *lv2, int a) {
    const int lane = threadIdx.x & 31;
    const int b = 2 * a + (lane >> 4);
    const int q = lane & 15, r = q >> 2, c = q & 3;
    const uint32_t va = *reinterpret_cast<const uint16_t *>(lv2 + (2 * r) * (kTileCols >> 2) + 8 * b + 2 * c);
    const uint32_t vb = *reinterpret_cast<const uint16_t *>(lv2 + (2 * r + 1) * (kTileCols >> 2) + 8 * b + 2 * c);
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
    const uint32_t px4 = (s2 + 2u) >> 2;
    {
        const int yl = (y0 >> 4) + (r >> 1), xl = (x0 >> 4) + 2 * b + (c >> 1);
        if ((q & 5) == 0 && (kFull || yl < L.height[4])) {
            if (kFull || xl < L.width[4]) smem_count(smem_addr(sm.hs[2]) + 4 * px4);
            if (kFull || xl < L.gray_pitch[4]) ebase[L.gray_offset[4] + (size_t)yl * L.gray_pitch[4] + xl] = (uint8_t)px4;
        }
    }
    if (K < 5) return;
    const uint32_t u1 = px4 + __shfl_down_sync(0xffffffffu, px4, 2);
    const uint32_t u2 = u1 + __shfl_down_sync(0xffffffffu, u1, 8);
    const uint32_t px5 = (u2 + 2u) >> 2;
    {
        const int yl = y0 >> 5, xl = (x0 >> 5) + b;
        if (q == 0 && (kFull || yl < L.height[5])) {
            if (kFull || xl < L.width[5]) smem_count(smem_addr(sm.hs[3]) + 4 * px5);
            if (kFull || xl < L.gray_pitch[5]) ebase[L.gray_offset[5] + (size_t)yl * L.gray_pitch[5] + xl] = (uint8_t)px5;
        }
    }
}

// Position of tile t (exposure, tile row, tile column), advanced one tile at a
// time so the loop divides by nothing.
struct TileCursor {
    int e, ty, tx;
    __device__ __forceinline__ void init(int t, int tiles_x, int tiles_per_exp) {
        e = t / tiles_per_exp;
        const int rt = t - e * tiles_per_exp;
        ty = rt / tiles_x;
        tx = rt - ty * tiles_x;
    }
    __device__ __forceinline__ void next(int tiles_x, int tiles_y) {
        if (++tx == tiles_x) {
            tx = 0;
            if (++ty == tiles_y) {
                ty = 0;
                ++e;
            }
        }
    }
};

// Any W: the tile row's pixels are a flat run [p0, p0 + cols) that starts
// anywhere inside a 16-pixel group, so groups are clipped to it.
__device__ __forceinline__ void tile_level0_general(const uint8_t *__restrict__ images, const mtb_layout_t &L,
                                                    uint8_t *ws, int e, int y0, int x0, int rows, int cols,
                                                    PyrShared &sm) {
    const int tid = threadIdx.x;
    const uint64_t W = (uint64_t)L.w;
    const uint64_t plane_px = W * (uint64_t)L.h;
    const uint64_t total_px = plane_px * (uint64_t)L.n;
    const uint64_t e0 = (uint64_t)e * plane_px;
    uint32_t *h0 = sm.h01[0][tid >> 5];
    for (int s = tid; s < kTileRows * kGroupsPerRow; s += kPyrThreads) {
        const int r = s / kGroupsPerRow;
        const int j = s - r * kGroupsPerRow;
        if (r >= rows) continue;
        const uint64_t p0 = e0 + (uint64_t)(y0 + r) * W + x0;
        const uint64_t gp = ((p0 >> 4) + j) << 4;
        if (gp >= p0 + cols) continue;
        uint32_t g[16];
        uint4 v;
        if (gp + 16 <= total_px) {
            const uint4 *src = reinterpret_cast<const uint4 *>(images + 3 * gp);
            v = gray16(__ldcs(src), __ldcs(src + 1), __ldcs(src + 2), g);
        } else {  // the buffer's last group: pixels past its end are not read
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                g[q] = 0;
                if (gp + q < total_px) {
                    const uint8_t *p = images + 3 * (gp + q);
                    g[q] = luma(p[0], p[1], p[2]);
                }
            }
            v.x = g[0] | (g[1] << 8) | (g[2] << 16) | (g[3] << 24);
            v.y = g[4] | (g[5] << 8) | (g[6] << 16) | (g[7] << 24);
            v.z = g[8] | (g[9] << 8) | (g[10] << 16) | (g[11] << 24);
            v.w = g[12] | (g[13] << 8) | (g[14] << 16) | (g[15] << 24);
        }
        const int c0 = (int)((int64_t)gp - (int64_t)p0);  // tile column of pixel 0 of the group; may be < 0
        const int qa = max(0, -c0), qb = min(16, cols - c0);
        uint8_t *row = sm.lv + r * kTileCols;
        if (qa == 0 && qb == 16 && (c0 & 15) == 0) {
            *reinterpret_cast<uint4 *>(row + c0) = v;
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (q >= qa && q < qb) row[c0 + q] = (uint8_t)g[q];
        }
        hist_group(h0, g, v, qa, qb);
    }
}

// Level 0 of the tile from shared memory to global (16-byte stores); used when
// the level-0 groups were clipped and written byte by byte.
__device__ __forceinline__ void tile_store_level0(const mtb_layout_t &L, uint8_t *ws, int e, int y0, int x0,
                                                  int rows, int cols, const PyrShared &sm) {
    uint8_t *g0 = Planes::gray(ws, L, e, 0);
    const size_t gp0 = (size_t)L.gray_pitch[0];
    for (int s = threadIdx.x; s < kTileRows * (kTileCols / 16); s += kPyrThreads) {
        const int r = s >> 4;
        const int c = (s & 15) << 4;
        if (r < rows && c < cols)
            *reinterpret_cast<uint4 *>(g0 + (size_t)(y0 + r) * gp0 + x0 + c) =
                *reinterpret_cast<const uint4 *>(sm.lv + r * kTileCols + c);
    }
}

// ---- levels 1 and 2 of one tile in one pass ----
// Thread u takes level-2 pixels (r2, c2..c2+1): level-1 pixels rows 2r2, 2r2+1,
// columns 2c2..2c2+3, from level-0 rows 4r2..4r2+3, columns 4c2..4c2+7.  Level 1
// goes to global only; level 2 also to shared memory for levels 3..5.
__device__ __forceinline__ void tile_levels12(const mtb_layout_t &L, uint8_t *ws, int e, int y0, int x0, int K,
                                              PyrShared &sm) {
    static_assert((kTileRows / 4) * (kTileCols / 8) == kPyrThreads, "one level-2 pixel pair per thread");
    const int u = threadIdx.x;
    const int r2 = u / (kTileCols / 8), c2 = (u % (kTileCols / 8)) * 2;
    const uint8_t *src = sm.lv + (4 * r2) * kTileCols + 4 * c2;
    const uint2 a0 = *reinterpret_cast<const uint2 *>(src);
    const uint2 a1 = *reinterpret_cast<const uint2 *>(src + kTileCols);
    const uint2 a2 = *reinterpret_cast<const uint2 *>(src + 2 * kTileCols);
    const uint2 a3 = *reinterpret_cast<const uint2 *>(src + 3 * kTileCols);
    const uint32_t w1a = __byte_perm(shrink2(a0.x, a1.x), shrink2(a0.y, a1.y), 0x6420u);  // level-1 row 2r2
    const uint32_t w1b = __byte_perm(shrink2(a2.x, a3.x), shrink2(a2.y, a3.y), 0x6420u);  // level-1 row 2r2+1
    {
        const int W1 = L.width[1], H1 = L.height[1];
        const int gp1 = L.gray_pitch[1];
        uint8_t *g1 = Planes::gray(ws, L, e, 1);
        uint32_t *h1 = sm.h01[1][threadIdx.x >> 5];
        const int xl = (x0 >> 1) + 2 * c2;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int yl = (y0 >> 1) + 2 * r2 + rr;
            const uint32_t w = rr ? w1b : w1a;
            if (yl < H1) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (xl + q < W1) atomicAdd(h1 + ((w >> (8 * q)) & 0xffu), 1u);
                if (xl < gp1) *reinterpret_cast<uint32_t *>(g1 + (size_t)yl * gp1 + xl) = w;
            }
        }
    }
    if (K < 2) return;
    const uint32_t p2 = shrink2(w1a, w1b);                     // [p0, 0, p1, 0] bytes
    const uint16_t w2 = (uint16_t)__byte_perm(p2, 0u, 0x4420u);  // p0 | p1 << 8
    *reinterpret_cast<uint16_t *>(sm.lv + lv_offset(2) + r2 * (kTileCols >> 2) + c2) = w2;
    const int W2 = L.width[2], H2 = L.height[2];
    const int gp2 = L.gray_pitch[2];
    const int yl = (y0 >> 2) + r2, xl = (x0 >> 2) + c2;
    if (yl < H2) {
        if (xl < W2) atomicAdd(sm.hs[0] + (w2 & 0xffu), 1u);
        if (xl + 1 < W2) atomicAdd(sm.hs[0] + (w2 >> 8), 1u);
        if (xl < gp2) *reinterpret_cast<uint16_t *>(Planes::gray(ws, L, e, 2) + (size_t)yl * gp2 + xl) = w2;
    }
}

// ---- levels 3..K of one tile, from level 2 in shared memory ----
// Level-5 pixel w of the tile sums the tile's 32-column block w, so warp w
// builds levels 3..5 of block w (16, 4 and 1 pixels): every warp does the same
// small share and none holds the others up at the next barrier.
__device__ __forceinline__ void tile_block_tail(const mtb_layout_t &L, uint8_t *ws, int e, int y0, int x0, int K,
                                                PyrShared &sm) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int l = 3; l <= kTileLog2; ++l) {
        if (l > K) break;
        const int side = kTileRows >> l;                // block side at level l: 4, 2, 1
        const int ppitch = kTileCols >> (l - 1), pitch = kTileCols >> l;
        if (lane < side * side) {
            const int r = lane / side, c = w * side + lane % side;
            const uint8_t *a = sm.lv + lv_offset(l - 1) + (2 * r) * ppitch + 2 * c;
            const uint32_t px = ((uint32_t)a[0] + a[1] + a[ppitch] + a[ppitch + 1] + 2u) >> 2;
            sm.lv[lv_offset(l) + r * pitch + c] = (uint8_t)px;
            const int yl = (y0 >> l) + r, xl = (x0 >> l) + c;
            if (yl < L.height[l]) {
                if (xl < L.width[l]) atomicAdd(sm.hs[l - 2] + px, 1u);
                if (xl < L.gray_pitch[l]) Planes::gray(ws, L, e, l)[(size_t)yl * L.gray_pitch[l] + xl] = (uint8_t)px;
            }
        }
        __syncwarp();
    }
}

// Adds the CTA's histograms of exposure e to the global ones, clears them and
// counts the CTA's ntiles tiles of e as done.  The CTA that completes the
// exposure's last tile computes the medians of levels 0..K (Sec. III-A).
__device__ void flush_exposure(const mtb_layout_t &L, uint8_t *ws, int e, int ntiles, int tiles_per_exp, int K,
                               PyrShared &sm) {
    const int tid = threadIdx.x;
    __syncthreads();
    for (int l = 0; l <= K; ++l) {
        uint32_t *gh = Planes::hist(ws, L, e, l);
        const int v = tid;  // kPyrThreads == 256 bins
        uint32_t sum = 0;
        if (l <= 1) {
#pragma unroll
            for (int w = 0; w < kPyrWarps; ++w) {
                sum += sm.h01[l][w][v];
                sm.h01[l][w][v] = 0;
            }
        } else {
            sum = sm.hs[l - 2][v];
            sm.hs[l - 2][v] = 0;
        }
        if (sum) atomicAdd(gh + v, sum);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const int old = atomicAdd(Ctr::tiles(ws, L, e), ntiles);
        sm.last = old + ntiles == tiles_per_exp;
    }
    __syncthreads();
    if (sm.last) {
        __threadfence();
        const int warp = tid >> 5;
        if (warp <= K) {
            const int m = warp_median<true>(Planes::hist(ws, L, e, warp));
            if ((tid & 31) == 0) *Planes::median(ws, L, e, warp) = m;
        }
        cta_signal(Ctr::pyr_ready(ws, L, e));  // gray planes, histograms and medians of e are complete
    }
    __syncthreads();
}

}  // namespace
}  // namespace mtb
