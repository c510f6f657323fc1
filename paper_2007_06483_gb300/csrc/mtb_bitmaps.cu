// mtb_bitmaps.cu -- threshold and exclusion bitmaps.
//
// Sec. III-A: the median threshold bitmap (MTB) sets a pixel to 0 if it is <=
// the median of its pyramid image, else 1.  Sec. III-B: the exclusion bitmap
// (EB) removes pixels within +-tol of the median.  Both maps are packed 1 bit
// per pixel (bit b of word q = pixel 32q + b) and stored as (tb, eb) word pairs,
// so the search fetches both with one 8-byte load.  HBM traffic per pixel of a
// level: 1 byte read, 2 bits written.
//
// The medians of levels 0..tile_levels-1 come from the pyramid pass.  Deeper
// levels are small (at most 1/4096 of the full-resolution pixels): one CTA per
// exposure builds them here from the deepest tile level, with their histograms,
// medians and bitmaps.
//
// Comparisons run on 4 pixels at a time (SWAR on bytes): for a constant t,
// the MSB of every byte of
//     ge(x) = (x & ~T) | ((x ^ ~T) & ((x | 0x80..) - (T & 0x7f..)))
// is [x_byte >= t]  (T = t in every byte; the subtraction cannot borrow across
// bytes because each byte of the minuend is >= 0x80).  The MSBs of two words
// are merged into one (the first's shifted down by 4) and gathered into 8
// adjacent bits by one multiply: bits 3, 7, 11, ..., 31 times 2^21 + 2^14 +
// 2^7 + 1 land on bits 24..31 without carries; byte permutes then place the
// four top bytes.
// The exclusion test is that comparison on the per-byte absolute difference
// |g - m| (__vabsdiffu4, a single SIMD instruction): eb = [|g - m| >= tol + 1].
#include "mtb_bitmaps_dev.cuh"

namespace mtb {
namespace {

// CTAs are numbered deep levels first, then the tile levels from the coarsest
// to level 0, each over all exposures: the planes a chained search needs first
// (its coarse levels) are finished first.
// 5 CTAs per SM (48 registers, no spills): 17.0 us for the 4000x3000x3 planes
// and 59.9 us for 6000x4000x7, against 18.9 and 70.4 us at 4 (54 registers).
// kChunk: the words a CTA packs (bit_chunk_words), a compile-time constant so
// that the chunk arithmetic folds (as a kernel argument it cost ~1 us a pass).
template <int kChunk>
__global__ void __launch_bounds__(kBitThreads, 5)
k_bitmaps(const mtb_layout_t L, uint8_t *__restrict__ ws, int tol, int deep_ctas) {
    __shared__ uint32_t s_hist[256];
    __shared__ int s_med;
    // Wait before letting the search launch.  The search of the same call
    // starts without waiting for this grid (it polls the bit_done counters),
    // and it reads words that the call's clearing kernel zeroes: its queue
    // head, those counters and the status word.  This wait returns only once
    // the pyramid pass has completed, and every pyramid CTA itself waited for
    // the clearing kernel, so a search that launches after this trigger sees
    // the cleared words, even on a workspace a previous call left dirty.
    pdl_wait();  // gray planes and medians come from the pyramid pass
    pdl_trigger();
    if ((int)blockIdx.x < deep_ctas) {
        deep_levels(L, ws, tol, blockIdx.x, s_hist, &s_med);
        return;
    }
    int item = blockIdx.x - deep_ctas;
    int l = L.tile_levels - 1;
    for (; l > 0; --l) {
        const int per_level = bitmap_chunks(L, l, kChunk) * L.n;
        if (item < per_level) break;
        item -= per_level;
    }
    const int ch = bitmap_chunks(L, l, kChunk);
    const int e = item / ch;
    bitmap_chunk(L, ws, tol, e, l, item - e * ch, kChunk, &s_med);
}

}  // namespace

cudaError_t launch_bitmaps(const mtb_layout_t &L, int noise_tol, uint8_t *ws, cudaStream_t s, bool chained) {
    const int cw = bit_chunk_words(L);
    long long per_exp = 0;
    for (int l = 0; l < L.tile_levels; ++l) {
        const long long words = (long long)L.bits_pitch[l] * L.height[l];
        per_exp += (words + cw - 1) / cw;
    }
    const int deep = L.levels > L.tile_levels ? L.n : 0;
    const long long grid = deep + per_exp * L.n;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (cw == 2 * kBitWordsPerCta)
        return launch_k(k_bitmaps<2 * kBitWordsPerCta>, dim3((unsigned)grid), dim3(kBitThreads), s, chained, L, ws,
                        noise_tol, deep);
    return launch_k(k_bitmaps<kBitWordsPerCta>, dim3((unsigned)grid), dim3(kBitThreads), s, chained, L, ws, noise_tol,
                    deep);
}

}  // namespace mtb
