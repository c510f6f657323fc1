// mtb_bitmaps_dev.cuh -- device functions of the bitmap pass, shared by the
// stage kernel and the engine.
#pragma once

#include "mtb_device.cuh"

namespace mtb {
namespace {

constexpr uint32_t kHi = 0x80808080u;
constexpr uint32_t kLo7 = 0x7f7f7f7fu;

// Per-byte x >= t test for a fixed t in [0, 255], result in each byte's MSB.
struct ByteGE {
    uint32_t t_lo7, not_t;
    __device__ __forceinline__ explicit ByteGE(uint32_t t) {
        const uint32_t T = t * 0x01010101u;
        t_lo7 = T & kLo7;
        not_t = ~T;
    }
    __device__ __forceinline__ uint32_t operator()(uint32_t x) const {
        const uint32_t d = (x | kHi) - t_lo7;
        return (x & not_t) | ((x ^ not_t) & d);
    }
};

// The thresholds of one (exposure, level): tb = [g >= m + 1] and, since
// g < m - tol or g > m + tol is |g - m| > tol, eb = [|g - m| >= tol + 1] on the
// per-byte absolute difference (one SIMD instruction); a test that can never
// hold (m = 255, tol = 255) clears its whole output word instead.
struct Thresholds {
    uint32_t m4;  // the median in every byte
    ByteGE tb, eb;
    uint32_t tb_all, eb_all;
    __device__ __forceinline__ Thresholds(int m, int tol)
        : m4((uint32_t)m * 0x01010101u), tb((uint32_t)min(m + 1, 255)), eb((uint32_t)min(tol + 1, 255)),
          tb_all(m < 255 ? 0xffffffffu : 0u), eb_all(tol < 255 ? 0xffffffffu : 0u) {}
};

// The flags (byte MSBs) of two gray words k and k + 1 -> one product whose top
// byte holds the 8 flags in pixel order: word k's MSBs moved to bits 3, 11,
// 19, 27 and word k + 1's at 7, 15, 23, 31, times 2^21 + 2^14 + 2^7 + 1, put
// bit 8j + 3 on 24 + j and bit 8j + 7 on 28 + j; every other partial product
// lands on a distinct bit below 24 or past 31, so nothing carries into the top
// byte.
__device__ __forceinline__ uint32_t gather_pair(uint32_t r0, uint32_t r1) {
    return ((((r0 & kHi) >> 4) | (r1 & kHi)) * 0x00204081u);
}
// The top bytes of four such products, in order, as one word.
__device__ __forceinline__ uint32_t top_bytes(uint32_t p0, uint32_t p1, uint32_t p2, uint32_t p3) {
    return __byte_perm(__byte_perm(p0, p1, 0x0073u), __byte_perm(p2, p3, 0x0073u), 0x5410u);
}

// tb and eb words of 32 gray pixels in 8 little-endian words; only the first
// nvalid pixels can be set.
__device__ __forceinline__ uint2 pack_bits(const uint32_t (&v)[8], const Thresholds &th, int nvalid) {
    uint32_t pt[4], pe[4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        pt[k / 2] = gather_pair(th.tb(v[k]), th.tb(v[k + 1]));
        pe[k / 2] = gather_pair(th.eb(__vabsdiffu4(v[k], th.m4)), th.eb(__vabsdiffu4(v[k + 1], th.m4)));
    }
    const uint32_t keep = nvalid >= 32 ? 0xffffffffu : ((1u << nvalid) - 1u);
    return make_uint2(top_bytes(pt[0], pt[1], pt[2], pt[3]) & keep & th.tb_all,
                      top_bytes(pe[0], pe[1], pe[2], pe[3]) & keep & th.eb_all);
}

// Levels tile_levels..levels-1 of exposure e, built by one CTA.  Each level
// reads the previous one, which this CTA wrote itself for all but the first,
// so those reads go through L2 (ld.global.cg) after a CTA barrier.
__device__ void deep_levels(const mtb_layout_t &L, uint8_t *ws, int tol, int e, uint32_t *s_hist, int *s_med) {
    const int tid = threadIdx.x;
    for (int l = L.tile_levels; l < L.levels; ++l) {
        for (int v = tid; v < 256; v += blockDim.x) s_hist[v] = 0;
        __syncthreads();
        const uint8_t *src = Planes::gray(ws, L, e, l - 1);
        const int spitch = L.gray_pitch[l - 1];
        uint8_t *dst = Planes::gray(ws, L, e, l);
        const int Wl = L.width[l], Hl = L.height[l], gpl = L.gray_pitch[l];
        const int npx = Wl * Hl;
        for (int idx = tid; idx < npx; idx += blockDim.x) {
            const int y = idx / Wl, x = idx - y * Wl;
            const uint8_t *s0 = src + (size_t)(2 * y) * spitch + 2 * x;
            const uint8_t *s1 = s0 + spitch;
            const uint32_t v = box2(__ldcg(s0), __ldcg(s0 + 1), __ldcg(s1), __ldcg(s1 + 1));
            dst[(size_t)y * gpl + x] = (uint8_t)v;
            atomicAdd(s_hist + v, 1u);
        }
        __syncthreads();
        uint32_t *gh = Planes::hist(ws, L, e, l);
        for (int v = tid; v < 256; v += blockDim.x) gh[v] = s_hist[v];
        if (tid < 32) {
            const int m = warp_median<false>(s_hist);
            if (tid == 0) {
                *s_med = m;
                *Planes::median(ws, L, e, l) = m;
            }
        }
        __syncthreads();
        const Thresholds th(*s_med, tol);
        const int bp = L.bits_pitch[l];
        uint2 *out = Planes::bits(ws, L, e, l);
        for (int idx = tid; idx < bp * Hl; idx += blockDim.x) {
            const int y = idx / bp, q = idx - y * bp;
            const int x = q * 32;
            uint2 r = make_uint2(0u, 0u);
            if (x < Wl) {
                const uint4 *p = reinterpret_cast<const uint4 *>(dst + (size_t)y * gpl + x);
                const uint4 a = __ldcg(p), b = __ldcg(p + 1);
                const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
                r = pack_bits(v, th, min(32, Wl - x));
            }
            out[idx] = r;
        }
        cta_signal(Ctr::bit_done(ws, L, e, l));  // level l of exposure e is complete
    }
}

// Chunk `item` (of a level's chunk_words-word chunks, tile levels in order) of
// one exposure -> level and chunk within the level.
__device__ __forceinline__ void bitmap_chunk_of(const mtb_layout_t &L, int item, int chunk_words, int *level,
                                                int *chunk) {
    int l = 0, c = item;
    for (; l < L.tile_levels - 1; ++l) {
        const int ch = bitmap_chunks(L, l, chunk_words);
        if (c < ch) break;
        c -= ch;
    }
    *level = l;
    *chunk = c;
}

// Chunk c of level l (a tile level) of exposure e: threshold against the
// median from the pyramid pass, pack, and count the chunk as done.  Thread t
// takes words c * chunk_words + t, + blockDim, ...; their (row, word) positions
// advance by a fixed step, so only the first is a division.
__device__ void bitmap_chunk(const mtb_layout_t &L, uint8_t *ws, int tol, int e, int l, int c, int chunk_words,
                             int *s_med) {
    constexpr int kGroup = 4;  // words whose gray loads a thread issues together
    const int Wl = L.width[l], Hl = L.height[l], bp = L.bits_pitch[l], gpl = L.gray_pitch[l];
    const uint8_t *__restrict__ g = Planes::gray(ws, L, e, l);
    uint2 *__restrict__ out = Planes::bits(ws, L, e, l);
    const int words = bp * Hl;
    const int w_end = min(words, (c + 1) * chunk_words);
    const int step = (int)blockDim.x, step_y = step / bp, step_q = step - step_y * bp;
    int i0 = c * chunk_words + (int)threadIdx.x;
    int y = i0 / bp, q = i0 - y * bp;  // position of word i0
    uint4 va[kGroup], vb[kGroup];
    int xs[kGroup];  // first pixel of each word (the word index itself is idx: rows are bp words)
    // the gray loads of a group are issued before any store (and the first
    // group's before the median is read), so they are all in flight together
    auto load_group = [&]() {
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            const int idx = i0 + j * step;
            xs[j] = q * 32;
            va[j] = vb[j] = make_uint4(0u, 0u, 0u, 0u);
            if (idx < w_end && xs[j] < Wl) {
                const uint4 *p = reinterpret_cast<const uint4 *>(g + (size_t)y * gpl + xs[j]);
                va[j] = __ldcs(p);
                vb[j] = __ldcs(p + 1);
            }
            q += step_q;
            y += step_y;
            if (q >= bp) {
                q -= bp;
                ++y;
            }
        }
    };
    load_group();
    if (threadIdx.x == 0) *s_med = *Planes::median(ws, L, e, l);
    __syncthreads();
    const Thresholds th(*s_med, tol);
    for (;;) {
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            const int idx = i0 + j * step;
            if (idx < w_end) {
                const uint32_t v[8] = {va[j].x, va[j].y, va[j].z, va[j].w, vb[j].x, vb[j].y, vb[j].z, vb[j].w};
                out[idx] = xs[j] < Wl ? pack_bits(v, th, min(32, Wl - xs[j])) : make_uint2(0u, 0u);
            }
        }
        i0 += kGroup * step;
        if (i0 >= w_end) break;
        load_group();
    }
    cta_signal(Ctr::bit_done(ws, L, e, l));
}

}  // namespace
}  // namespace mtb
