// mtb_bitmaps.cu -- median scan and bitmap packing.
//
// Sec. III-A: the median of each pyramid image comes from its histogram, and the
// median threshold bitmap (MTB) sets a pixel to 0 if it is <= the median, else 1.
// Sec. III-B: the exclusion bitmap (EB) removes pixels within +-tol of the median.
// Both maps are packed 1 bit per pixel (bit b of word q = pixel 32q + b) and
// stored as (tb, eb) word pairs, so the search kernel fetches both with one
// 8-byte load.  HBM traffic per pixel of a level: 1 byte read, 2 bits written.
//
// Levels deeper than the pyramid pass builds are small (at most 1/4096 of the
// full-resolution pixels); one CTA per exposure builds them here from the
// deepest tile level, with their histograms, medians and bitmaps.
#include "mtb_internal.cuh"

namespace mtb {
namespace {

// Lower median (smallest v with cumulative count >= ceil(N/2)) of a 256-bin
// histogram; called by all 32 lanes of one warp, returns the median to all.
__device__ int warp_median(const uint32_t *hist) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t c[8];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        c[k] = hist[lane * 8 + k];
        s += c[k];
    }
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(full, inc, o);
        if (lane >= o) inc += t;
    }
    const uint32_t total = __shfl_sync(full, inc, 31);
    const uint32_t half = total / 2 + (total & 1u);  // ceil(total / 2)
    const uint32_t before = inc - s;
    const unsigned owner_mask = __ballot_sync(full, half > before && half <= inc);
    if (owner_mask == 0) return 0;
    const int owner = __ffs(owner_mask) - 1;
    int m = 0;
    if (lane == owner) {
        uint32_t cum = before;
        m = lane * 8 + 7;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            cum += c[k];
            if (cum >= half) {
                m = lane * 8 + k;
                break;
            }
        }
    }
    return __shfl_sync(full, m, owner);
}

// tb and eb bits of 32 gray pixels held in 8 little-endian words; only the
// first nvalid pixels can be set.
__device__ __forceinline__ uint2 pack_bits(const uint32_t (&v)[8], int m, int tol, int nvalid) {
    const int lo = m - tol;
    const uint32_t band = 2u * (uint32_t)tol;
    uint32_t tb = 0, eb = 0;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        const int g = (int)((v[b >> 2] >> ((b & 3) * 8)) & 0xffu);
        tb |= (uint32_t)(g > m) << b;
        // outside [m - tol, m + tol]  <=>  (g - lo) does not lie in [0, 2 tol]
        eb |= (uint32_t)((uint32_t)(g - lo) > band) << b;
    }
    const uint32_t keep = nvalid >= 32 ? 0xffffffffu : ((1u << nvalid) - 1u);
    return make_uint2(tb & keep, eb & keep);
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
            const int m = warp_median(s_hist);
            if (tid == 0) {
                *s_med = m;
                *Planes::median(ws, L, e, l) = m;
            }
        }
        __syncthreads();
        const int m = *s_med;
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
                r = pack_bits(v, m, tol, min(32, Wl - x));
            }
            out[idx] = r;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBitThreads)
k_bitmaps(const mtb_layout_t L, uint8_t *__restrict__ ws, int tol, int deep_ctas, int chunks_per_exp) {
    __shared__ uint32_t s_hist[256];
    __shared__ int s_med;
    if ((int)blockIdx.x < deep_ctas) {
        deep_levels(L, ws, tol, blockIdx.x, s_hist, &s_med);
        return;
    }
    const int item = blockIdx.x - deep_ctas;
    const int e = item / chunks_per_exp;
    int c = item - e * chunks_per_exp;
    int l = 0;
    for (; l < L.tile_levels - 1; ++l) {
        const int words = L.bits_pitch[l] * L.height[l];
        const int ch = (words + kBitWordsPerCta - 1) / kBitWordsPerCta;
        if (c < ch) break;
        c -= ch;
    }
    if (threadIdx.x < 32) {
        const int m = warp_median(Planes::hist(ws, L, e, l));
        if (threadIdx.x == 0) {
            s_med = m;
            if (c == 0) *Planes::median(ws, L, e, l) = m;
        }
    }
    __syncthreads();
    const int m = s_med;
    const int Wl = L.width[l], Hl = L.height[l], bp = L.bits_pitch[l], gpl = L.gray_pitch[l];
    const uint8_t *g = Planes::gray(ws, L, e, l);
    uint2 *out = Planes::bits(ws, L, e, l);
    const int words = bp * Hl;
    const int w_end = min(words, (c + 1) * kBitWordsPerCta);
    for (int idx = c * kBitWordsPerCta + threadIdx.x; idx < w_end; idx += kBitThreads) {
        const int y = idx / bp, q = idx - y * bp;
        const int x = q * 32;
        uint2 r = make_uint2(0u, 0u);
        if (x < Wl) {
            const uint4 *p = reinterpret_cast<const uint4 *>(g + (size_t)y * gpl + x);
            const uint4 a = __ldcs(p), b = __ldcs(p + 1);
            const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            r = pack_bits(v, m, tol, min(32, Wl - x));
        }
        out[idx] = r;
    }
}

}  // namespace

cudaError_t launch_bitmaps(const mtb_layout_t &L, int noise_tol, uint8_t *ws, cudaStream_t s) {
    long long per_exp = 0;
    for (int l = 0; l < L.tile_levels; ++l) {
        const long long words = (long long)L.bits_pitch[l] * L.height[l];
        per_exp += (words + kBitWordsPerCta - 1) / kBitWordsPerCta;
    }
    const int deep = L.levels > L.tile_levels ? L.n : 0;
    const long long grid = deep + per_exp * L.n;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_bitmaps<<<(unsigned)grid, kBitThreads, 0, s>>>(L, ws, noise_tol, deep, (int)per_exp);
    return cudaGetLastError();
}

}  // namespace mtb
