// mtb_pyramid.cu -- the pyramid pass.
//
// One read of the interleaved RGB8 exposures produces, for every exposure:
//   * the gray image (Sec. III-A: exposures are converted to gray-scale),
//   * pyramid levels 1..tile_levels-1 (Sec. III-A: halve both dimensions, the
//     next level made from the previous one, Sec. III-B),
//   * the 256-bin histogram of each of those levels (Sec. III-B).
// The CTA owns a 32-row x 256-column tile of full-resolution pixels.  Level l
// pixels of the tile have their whole 2^l x 2^l source block inside the tile
// (l <= 5), so the tile's part of levels 1..5 is built in shared memory from
// the gray tile without touching HBM again.  HBM traffic per full-resolution
// pixel: 3 bytes read (RGB) + 4/3 bytes written (gray levels).
#include "mtb_internal.cuh"

namespace mtb {
namespace {

// Offset of level l's tile inside the shared level buffer.
__host__ __device__ constexpr int lv_offset(int l) {
    int off = 0;
    for (int k = 0; k < l; ++k) off += (kTileRows >> k) * (kTileCols >> k);
    return off;
}
constexpr int kLvBytes = lv_offset(kTileLog2 + 1);

__device__ __forceinline__ uint32_t byte_of(const uint32_t (&w)[12], int k) {
    return (w[k >> 2] >> ((k & 3) * 8)) & 0xffu;
}

// Gray values of the 16 pixels starting at flat pixel index gp (a multiple of
// 16, so the 48 RGB bytes are one 16-byte aligned run).  Pixels at or past
// total_px (only in the last group of the buffer) are read one byte at a time
// and left 0.
__device__ __forceinline__ void gray_group(const uint8_t *__restrict__ images, uint64_t gp,
                                           uint64_t total_px, uint32_t (&g)[16]) {
    if (gp + 16 <= total_px) {
        const uint4 *src = reinterpret_cast<const uint4 *>(images + 3 * gp);
        const uint4 a = __ldcs(src), b = __ldcs(src + 1), c = __ldcs(src + 2);
        const uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
        for (int q = 0; q < 16; ++q) g[q] = luma(byte_of(w, 3 * q), byte_of(w, 3 * q + 1), byte_of(w, 3 * q + 2));
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            g[q] = 0;
            if (gp + q < total_px) {
                const uint8_t *p = images + 3 * (gp + q);
                g[q] = luma(p[0], p[1], p[2]);
            }
        }
    }
}

__global__ void __launch_bounds__(kPyrThreads)
k_pyramid(const uint8_t *__restrict__ images, const mtb_layout_t L, uint8_t *__restrict__ ws,
          int tiles_x, int tiles_per_exp, int total_tiles) {
    __shared__ __align__(16) uint8_t s_lv[kLvBytes];
    __shared__ uint32_t s_h01[2][kPyrWarps][256];    // warp-private, levels 0 and 1
    __shared__ uint32_t s_hs[kTileLog2 - 1][256];     // levels 2..5, one per CTA

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int K = L.tile_levels - 1;
    const int W = L.w, H = L.h;
    const uint64_t plane_px = (uint64_t)W * H;
    const uint64_t total_px = plane_px * L.n;

    for (int v = tid; v < 2 * kPyrWarps * 256; v += kPyrThreads) (&s_h01[0][0][0])[v] = 0;
    for (int v = tid; v < (kTileLog2 - 1) * 256; v += kPyrThreads) (&s_hs[0][0])[v] = 0;

    // Adds this CTA's histograms of exposure e to the global ones and clears them.
    auto flush = [&](int e) {
        __syncthreads();
        for (int l = 0; l <= K; ++l) {
            uint32_t *gh = Planes::hist(ws, L, e, l);
            for (int v = tid; v < 256; v += kPyrThreads) {
                uint32_t sum = 0;
                if (l <= 1) {
#pragma unroll
                    for (int w = 0; w < kPyrWarps; ++w) {
                        sum += s_h01[l][w][v];
                        s_h01[l][w][v] = 0;
                    }
                } else {
                    sum = s_hs[l - 2][v];
                    s_hs[l - 2][v] = 0;
                }
                if (sum) atomicAdd(gh + v, sum);
            }
        }
        __syncthreads();
    };

    const int t0 = (int)(((long long)blockIdx.x * total_tiles) / gridDim.x);
    const int t1 = (int)(((long long)(blockIdx.x + 1) * total_tiles) / gridDim.x);
    int cur_e = t0 < t1 ? t0 / tiles_per_exp : -1;
    __syncthreads();

    for (int t = t0; t < t1; ++t) {
        const int e = t / tiles_per_exp;
        if (e != cur_e) {
            flush(cur_e);
            cur_e = e;
        }
        const int rt = t - e * tiles_per_exp;
        const int ty = rt / tiles_x;
        const int tx = rt - ty * tiles_x;
        const int y0 = ty * kTileRows, x0 = tx * kTileCols;
        const int rows = min(kTileRows, H - y0);
        const int cols = min(kTileCols, W - x0);
        const uint64_t e0 = (uint64_t)e * plane_px;

        // ---- gray of level 0 into shared memory, histogram of level 0 ----
        uint32_t *h0 = s_h01[0][warp];
        for (int s = tid; s < kTileRows * kGroupsPerRow; s += kPyrThreads) {
            const int r = s / kGroupsPerRow;
            const int j = s - r * kGroupsPerRow;
            if (r >= rows) continue;
            const uint64_t p0 = e0 + (uint64_t)(y0 + r) * W + x0;  // first pixel of the row's span
            const uint64_t gp = ((p0 >> 4) + j) << 4;
            if (gp >= p0 + cols) continue;
            uint32_t g[16];
            gray_group(images, gp, total_px, g);
            const int c0 = (int)((int64_t)gp - (int64_t)p0);  // tile column of g[0]; may be < 0
            const int qa = max(0, -c0), qb = min(16, cols - c0);
            uint8_t *row = s_lv + r * kTileCols;
            if (qa == 0 && qb == 16 && (c0 & 15) == 0) {
                uint4 v;
                v.x = g[0] | (g[1] << 8) | (g[2] << 16) | (g[3] << 24);
                v.y = g[4] | (g[5] << 8) | (g[6] << 16) | (g[7] << 24);
                v.z = g[8] | (g[9] << 8) | (g[10] << 16) | (g[11] << 24);
                v.w = g[12] | (g[13] << 8) | (g[14] << 16) | (g[15] << 24);
                *reinterpret_cast<uint4 *>(row + c0) = v;
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (q >= qa && q < qb) row[c0 + q] = (uint8_t)g[q];
            }
            // runs of equal values go in with one shared-memory atomic each
            uint32_t run_v = 0xffffffffu, run_n = 0;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                if (q < qa || q >= qb) continue;
                if (g[q] == run_v) {
                    ++run_n;
                } else {
                    if (run_n) atomicAdd(h0 + run_v, run_n);
                    run_v = g[q];
                    run_n = 1;
                }
            }
            if (run_n) atomicAdd(h0 + run_v, run_n);
        }
        __syncthreads();

        // ---- level 0 to global (16-byte stores) ----
        {
            uint8_t *g0 = Planes::gray(ws, L, e, 0);
            const int gp0 = L.gray_pitch[0];
            for (int s = tid; s < kTileRows * (kTileCols / 16); s += kPyrThreads) {
                const int r = s / (kTileCols / 16);
                const int c = (s - r * (kTileCols / 16)) * 16;
                if (r < rows && c < cols)
                    *reinterpret_cast<uint4 *>(g0 + (size_t)(y0 + r) * gp0 + x0 + c) =
                        *reinterpret_cast<const uint4 *>(s_lv + r * kTileCols + c);
            }
        }

        // ---- levels 1..K from the previous level in shared memory ----
        for (int l = 1; l <= K; ++l) {
            const uint8_t *prev = s_lv + lv_offset(l - 1);
            const int ppitch = kTileCols >> (l - 1);
            uint8_t *cur = s_lv + lv_offset(l);
            const int cpitch = kTileCols >> l;
            const int upr = cpitch >> 2;  // 4-pixel units per row
            const int units = (kTileRows >> l) * upr;
            const int yl0 = y0 >> l, xl0 = x0 >> l;
            const int Wl = L.width[l], Hl = L.height[l], gpl = L.gray_pitch[l];
            uint8_t *gl = Planes::gray(ws, L, e, l);
            uint32_t *hl = l == 1 ? s_h01[1][warp] : s_hs[l - 2];
            for (int u = tid; u < units; u += kPyrThreads) {
                const int r = u / upr;
                const int c = (u - r * upr) << 2;
                const uint2 a = *reinterpret_cast<const uint2 *>(prev + (2 * r) * ppitch + 2 * c);
                const uint2 b = *reinterpret_cast<const uint2 *>(prev + (2 * r + 1) * ppitch + 2 * c);
                uint32_t out = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t ta = q < 2 ? a.x : a.y, tb = q < 2 ? b.x : b.y;
                    const int sh = (q & 1) * 16;
                    const uint32_t v = box2((ta >> sh) & 0xffu, (ta >> (sh + 8)) & 0xffu,
                                            (tb >> sh) & 0xffu, (tb >> (sh + 8)) & 0xffu);
                    out |= v << (8 * q);
                }
                *reinterpret_cast<uint32_t *>(cur + r * cpitch + c) = out;
                const int yl = yl0 + r, xl = xl0 + c;
                if (yl < Hl) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (xl + q < Wl) atomicAdd(hl + ((out >> (8 * q)) & 0xffu), 1u);
                    if (xl < gpl) *reinterpret_cast<uint32_t *>(gl + (size_t)yl * gpl + xl) = out;
                }
            }
            __syncthreads();
        }
        if (K == 0) __syncthreads();
    }
    if (cur_e >= 0) flush(cur_e);
}

int g_pyr_blocks_per_sm = 0;

}  // namespace

cudaError_t launch_pyramid(const uint8_t *images, const mtb_layout_t &L, uint8_t *ws, cudaStream_t s) {
    const int tiles_x = (L.w + kTileCols - 1) / kTileCols;
    const int tiles_y = (L.h + kTileRows - 1) / kTileRows;
    const long long per_exp = (long long)tiles_x * tiles_y;
    const long long total = per_exp * L.n;
    if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (g_pyr_blocks_per_sm == 0) {
        int nb = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pyramid, kPyrThreads, 0);
        if (err != cudaSuccess) return err;
        g_pyr_blocks_per_sm = nb > 0 ? nb : 1;
    }
    const long long cap = (long long)device_sm_count() * g_pyr_blocks_per_sm;
    const int grid = (int)(total < cap ? total : cap);
    k_pyramid<<<grid, kPyrThreads, 0, s>>>(images, L, ws, tiles_x, (int)per_exp, (int)total);
    return cudaGetLastError();
}

}  // namespace mtb
