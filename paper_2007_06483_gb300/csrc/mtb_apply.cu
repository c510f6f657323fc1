// mtb_apply.cu -- moving the RGB exposures by the shifts the search found.
//
// The search's operator S (Sec. III-B moves the second image's maps by the
// candidate offset) applied to the images: out(x, y) = in(x - sx, y - sy), per
// channel, with 0 or the nearest edge pixel where the source lies outside.
// Pure data movement: 3 bytes read and 3 written per pixel.
//
// Within one output row the source is one row of the same exposure (the moved
// row, or the clamped one in edge mode) read at a constant byte offset 3*sx,
// so the row is a byte-shifted copy.  Threads own 16-byte aligned chunks of the
// output (global alignment: the images base is 16-byte aligned); an interior
// chunk is two aligned 16-byte loads of the source merged with funnel shifts
// (the misalignment is the same for the whole row) and one streaming 16-byte
// store.  Chunks at the row ends, in the fill region or shared with the next
// row take a per-byte path.
#include "mtb_internal.cuh"

namespace mtb {
namespace {

constexpr int kApplyThreads = 256;

// 16 bytes starting r bytes into the 32 bytes (a, b): funnel shifts of adjacent
// words; r is uniform over a row.
__device__ __forceinline__ uint4 window16(const uint4 &a, const uint4 &b, int r) {
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    const int q = r >> 2;
    const uint32_t sh = 8u * (uint32_t)(r & 3);
    uint32_t o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // q is 0..3: select without dynamic register indexing
        const uint32_t lo = q == 0 ? w[k] : q == 1 ? w[k + 1] : q == 2 ? w[k + 2] : w[k + 3];
        const uint32_t hi = q == 0 ? w[k + 1] : q == 1 ? w[k + 2] : q == 2 ? w[k + 3] : w[k + 4];
        o[k] = __funnelshift_r(lo, hi, sh);
    }
    return make_uint4(o[0], o[1], o[2], o[3]);
}

// One output byte at global byte index g (any row, any exposure).
__device__ __forceinline__ uint8_t apply_byte(const uint8_t *__restrict__ in, const int32_t *__restrict__ shifts,
                                              long long g, int w, int h, int fill) {
    const long long row_bytes = 3ll * w;
    const long long exp_bytes = row_bytes * h;
    const int e = (int)(g / exp_bytes);
    const long long rem = g - (long long)e * exp_bytes;
    const int y = (int)(rem / row_bytes);
    const int c = (int)(rem - (long long)y * row_bytes);
    const int x = c / 3, ch = c - 3 * x;
    long long xs = (long long)x - shifts[2 * e], ys = (long long)y - shifts[2 * e + 1];
    if (xs < 0 || xs >= w || ys < 0 || ys >= h) {
        if (fill == 0) return 0;
        xs = xs < 0 ? 0 : (xs >= w ? w - 1 : xs);
        ys = ys < 0 ? 0 : (ys >= h ? h - 1 : ys);
    }
    return in[(long long)e * exp_bytes + ys * row_bytes + xs * 3 + ch];
}

// A chunk outside the row's interior: all fill (a zero-filled row), or byte by
// byte (the row ends, a chunk shared with the next row, the stack's last bytes).
__device__ __forceinline__ void edge_chunk(const uint8_t *__restrict__ in, const int32_t *__restrict__ shifts, int w,
                                           int h, int fill, uint8_t *__restrict__ out, long long k, long long r0,
                                           long long row_bytes, long long total, bool zero_row) {
    const long long g = k << 4;
    const long long c = g - r0;
    uint4 v;
    if (c + 16 <= row_bytes && zero_row) {
        v = make_uint4(0u, 0u, 0u, 0u);
    } else {
        uint32_t b[4] = {0u, 0u, 0u, 0u};
        for (int j = 0; j < 16 && g + j < total; ++j)
            b[j >> 2] |= (uint32_t)apply_byte(in, shifts, g + j, w, h, fill) << (8 * (j & 3));
        if (g + 16 > total) {  // the stack's last bytes: no store past its end
            for (int j = 0; g + j < total; ++j) out[g + j] = (uint8_t)(b[j >> 2] >> (8 * (j & 3)));
            return;
        }
        v = make_uint4(b[0], b[1], b[2], b[3]);
    }
    __stcs(reinterpret_cast<uint4 *>(out + g), v);
}

// Warp v of the grid takes output rows v, v + (warps in the grid), ... of the
// n*h rows; a row owns the 16-byte chunks whose first byte lies in it, and the
// lanes take its chunks in turn (coalesced 512-byte steps).
__global__ void __launch_bounds__(kApplyThreads)
k_apply_shifts(const uint8_t *__restrict__ in, int n, int w, int h, const int32_t *__restrict__ shifts, int fill,
               uint8_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (kApplyThreads / 32);
    const long long row_bytes = 3ll * w;
    const long long rows = (long long)n * h;
    const long long total = rows * row_bytes;
    for (long long gr = (long long)blockIdx.x * (kApplyThreads / 32) + (threadIdx.x >> 5); gr < rows; gr += warps) {
        const int e = (int)(gr / h);
        const int y = (int)(gr - (long long)e * h);
        const long long sxb = 3ll * shifts[2 * e];
        long long ys = (long long)y - shifts[2 * e + 1];
        const bool row_in = ys >= 0 && ys < h;
        if (!row_in) ys = ys < 0 ? 0 : h - 1;  // used in edge mode only
        const long long r0 = gr * row_bytes;    // first output byte of the row
        const long long k_first = (r0 + 15) >> 4, k_last = (r0 + row_bytes - 1) >> 4;
        // column bytes c whose source column lies inside the source row
        const long long c_lo = sxb > 0 ? sxb : 0;
        const long long c_hi = row_bytes + (sxb < 0 ? sxb : 0);
        // source byte of column byte c (relative to in): src0 + c; its offset
        // within an aligned 16-byte block is the same for every chunk of the row
        const long long src0 = ((long long)e * h + ys) * row_bytes - sxb;
        const int r = (int)((((src0 - r0) % 16) + 16) % 16);
        const bool zero_row = !row_in && fill == 0;
        // chunks whose 16 bytes all come from inside the source row: a
        // branch-free loop with 4 chunks (8 loads) in flight per lane
        long long k_in_lo = k_last + 1, k_in_hi = k_last;  // empty unless set below
        if (!zero_row) {
            const long long c_end = (c_hi < row_bytes ? c_hi : row_bytes) - 16;
            if (c_end >= c_lo) {
                k_in_lo = (r0 + c_lo + 15) >> 4;
                k_in_hi = (r0 + c_end) >> 4;
                if (k_in_lo < k_first) k_in_lo = k_first;
                if (k_in_hi > k_last) k_in_hi = k_last;
                if (k_in_hi < k_in_lo) k_in_lo = k_last + 1, k_in_hi = k_last;
            }
        }
        if (k_in_lo <= k_in_hi) {
            long long k = k_in_lo + lane;
            for (; k + 96 <= k_in_hi; k += 128) {
                uint4 a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long long s = src0 + ((k + 32 * u) << 4) - r0;
                    const uint4 *p = reinterpret_cast<const uint4 *>(in + (s - r));
                    a[u] = __ldcs(p);
                    b[u] = r == 0 ? a[u] : __ldcs(p + 1);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    __stcs(reinterpret_cast<uint4 *>(out + ((k + 32 * u) << 4)), r == 0 ? a[u] : window16(a[u], b[u], r));
            }
            for (; k <= k_in_hi; k += 32) {
                const long long s = src0 + (k << 4) - r0;
                const uint4 *p = reinterpret_cast<const uint4 *>(in + (s - r));
                const uint4 a = __ldcs(p);
                __stcs(reinterpret_cast<uint4 *>(out + (k << 4)), r == 0 ? a : window16(a, __ldcs(p + 1), r));
            }
        }
        // the other chunks (fill, the row ends, chunks shared with the next row):
        // before and after the interior range
        const long long k_mid = k_in_lo < k_last + 1 ? k_in_lo : k_last + 1;
        for (long long k = k_first + lane; k < k_mid; k += 32) edge_chunk(in, shifts, w, h, fill, out, k, r0, row_bytes,
                                                                        total, zero_row);
        for (long long k = (k_in_hi + 1 > k_first ? k_in_hi + 1 : k_first) + lane; k <= k_last; k += 32)
            edge_chunk(in, shifts, w, h, fill, out, k, r0, row_bytes, total, zero_row);
    }
}

int g_apply_blocks_per_sm = 0;

}  // namespace

cudaError_t launch_apply_shifts(const uint8_t *images, int n, int w, int h, const int32_t *shifts, int fill,
                                uint8_t *out, cudaStream_t s) {
    if (g_apply_blocks_per_sm == 0) {
        int v = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_apply_shifts, kApplyThreads, 0);
        if (err != cudaSuccess) return err;
        g_apply_blocks_per_sm = v > 0 ? v : 1;
    }
    const long long warps = ((long long)n * h + kApplyThreads / 32 - 1) / (kApplyThreads / 32);
    const long long cap = (long long)device_sm_count() * g_apply_blocks_per_sm;
    const int grid = (int)(warps < cap ? warps : cap);
    return launch_k(k_apply_shifts, dim3(grid), dim3(kApplyThreads), s, false, images, n, w, h, shifts, fill, out);
}

}  // namespace mtb
