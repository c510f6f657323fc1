// mtb_internal.cuh -- definitions shared by the CUDA translation units of the
// MTB alignment library (never by the CPU oracle).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mtb.h"

namespace mtb {

// ---------------------------------------------------------------------------
// Pyramid pass geometry.  One tile is kTileRows x kTileCols full-resolution
// pixels (widths a multiple of 16 use 32 x 512 units of two 16 x 512 tiles
// instead, mtb_pyramid.cu); because 2^l divides both sides, every pixel of
// levels 1..kTileLog2 has its whole 2^l x 2^l source block inside one tile, so
// a tile builds its part of those levels on chip.  Deeper levels come from the
// bitmap pass.
constexpr int kTileLog2 = 5;
constexpr int kTileRows = 1 << kTileLog2;  // 32
constexpr int kTileCols = 256;
constexpr int kPyrThreads = 256;
constexpr int kPyrWarps = kPyrThreads / 32;
constexpr int kGroupsPerRow = kTileCols / 16 + 1;  // 16-pixel groups touching one tile row

// Bitmap pass: one CTA turns kBitWordsPerCta output words (32 pixels each) of
// one (exposure, level) plane into bits.
constexpr int kBitThreads = 256;
// 2048: about one wave of 5 CTAs per SM on the 4000x3000x3 planes (one-call
// step 80.7 -> 80.0 us against 1024; 512: 84.4 us; 4096: 81.5 us).
constexpr int kBitWordsPerCta = 2048;

// Words one bitmap CTA packs on a stack: twice kBitWordsPerCta once level 0 of
// all exposures has 2^22 words or more, so that its chunks still fill a wave
// (6000x4000x7, 5.3 M words: one-call step 242.9 -> 240.2 us; 4000x3000x3,
// 1.1 M words, keeps 2048: 4096 took its bitmap stage from 17.6 to 18.6 us).
__host__ __device__ inline int bit_chunk_words(const mtb_layout_t &L) {
    const long long words0 = (long long)L.n * L.bits_pitch[0] * L.height[0];
    return words0 >= (1ll << 22) ? 2 * kBitWordsPerCta : kBitWordsPerCta;
}

constexpr int kMaxShiftThreads = 256;

// Coarse search levels: from the deepest level up, every level whose whole
// reachable window (radius R = 2^(levels - l) - 1 <= kMaxTableRadius) costs at
// most kBruteBudget word-candidate evaluations per pair is searched by brute
// force over that window; the coarse-to-fine chain through those levels is
// then walked in the resulting error tables (kTableWords per pair: the windows
// of radius 1, 3, 7 and 15 take 9 + 49 + 225 + 961 = 1244 words).  2M per
// pair: on 4000x3000 and 6000x4000 stacks the radius-15 window (961
// candidates) costs more than one more 9-candidate hop (one-call step 86.0 ->
// 84.9 us and 269 -> 263 us against a budget of 8M).
constexpr int kMaxTableRadius = 15;
constexpr long long kBruteBudget = 2ll << 20;
constexpr int kTableWords = 1280;

// Bound on any device-side wait of the search (the waits always end when the
// kernels are correct; the bound turns a bug into MTB_ERR_TIMEOUT, not a hang).
constexpr unsigned long long kSearchTimeoutNs = 2000000000ull;

// ---------------------------------------------------------------------------
// Readings of the paper's unstated points, restated for the device.

// Sec. III-A gray conversion: BT.601 luma weights in Q14, rounded.
__host__ __device__ __forceinline__ uint32_t luma(uint32_t r, uint32_t g, uint32_t b) {
    return (4899u * r + 9617u * g + 1868u * b + 8192u) >> 14;
}

// Sec. III-A halving: mean of a 2x2 block, rounded half up.
__host__ __device__ __forceinline__ uint32_t box2(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    return (a + b + c + d + 2u) >> 2;
}

// Sec. III-A candidate k of a level: k = 0 is (0,0); k = 1..8 walk the other
// eight offsets with dy outer and dx inner, each over -1, 0, +1.
__host__ __device__ __forceinline__ int cand_dx(int k) {
    int j = k == 0 ? 4 : (k <= 4 ? k - 1 : k);
    return j % 3 - 1;
}
__host__ __device__ __forceinline__ int cand_dy(int k) {
    int j = k == 0 ? 4 : (k <= 4 ? k - 1 : k);
    return j / 3 - 1;
}

// ---------------------------------------------------------------------------
// Workspace accessors.
struct Planes {
    static __device__ __forceinline__ uint8_t *gray(uint8_t *ws, const mtb_layout_t &L, int e, int l) {
        return ws + L.gray_offset[l] + (size_t)e * L.gray_exposure_stride;
    }
    static __device__ __forceinline__ uint2 *bits(uint8_t *ws, const mtb_layout_t &L, int e, int l) {
        return reinterpret_cast<uint2 *>(ws + L.bits_offset[l] + (size_t)e * L.bits_exposure_stride);
    }
    static __device__ __forceinline__ uint32_t *hist(uint8_t *ws, const mtb_layout_t &L, int e, int l) {
        return reinterpret_cast<uint32_t *>(ws + L.hist_offset) + ((size_t)e * L.levels + l) * 256;
    }
    static __device__ __forceinline__ int32_t *median(uint8_t *ws, const mtb_layout_t &L, int e, int l) {
        return reinterpret_cast<int32_t *>(ws + L.median_offset) + (size_t)e * L.levels + l;
    }
    static __device__ __forceinline__ uint32_t *errs(uint8_t *ws, const mtb_layout_t &L, int e, int l) {
        return reinterpret_cast<uint32_t *>(ws + L.errs_offset) + ((size_t)e * L.levels + l) * 9;
    }
    static __device__ __forceinline__ int32_t *base(uint8_t *ws, const mtb_layout_t &L, int e, int l) {
        return reinterpret_cast<int32_t *>(ws + L.base_offset) + ((size_t)e * L.levels + l) * 2;
    }
    static __device__ __forceinline__ int32_t *shift(uint8_t *ws, const mtb_layout_t &L, int e, int l) {
        return reinterpret_cast<int32_t *>(ws + L.shift_offset) + ((size_t)e * L.levels + l) * 2;
    }
};

// ---------------------------------------------------------------------------
// Host-side launchers (each returns a cudaError_t of the launch).
int compute_layout(int n, int w, int h, int levels, mtb_layout_t *L);
int check_stack_args(int n, int w, int h, int levels, int noise_tol, int ref_idx);

// `chained`: the launch directly follows this library's previous stage in the
// same call, so its first kernel may overlap that stage's tail (programmatic
// dependent launch).  A stage called on its own starts after all earlier work.
cudaError_t launch_pyramid(const uint8_t *images, const mtb_layout_t &L, uint8_t *ws, cudaStream_t s);
// The parts of launch_pyramid: clearing the stack's bookkeeping, and the
// pyramid pass over tiles [tile_begin, tile_end) (tile t is tile t % per_exp,
// row-major, of exposure t / per_exp; launch_pyramid covers them all).
cudaError_t launch_clear_stack(const mtb_layout_t &L, uint8_t *ws, cudaStream_t s);
// Tiles of one 32-row tile row (widths a multiple of 16: 32 x 512 units of
// two 16 x 512 tiles; other widths: 32 x 256 tiles), and of one exposure.
int pyramid_tiles_x(const mtb_layout_t &L);
long long pyramid_tiles_per_exposure(const mtb_layout_t &L);
cudaError_t launch_pyramid_range(const uint8_t *images, const mtb_layout_t &L, uint8_t *ws, long long tile_begin,
                                 long long tile_end, cudaStream_t s, bool chained);
cudaError_t launch_bitmaps(const mtb_layout_t &L, int noise_tol, uint8_t *ws, cudaStream_t s, bool chained);
cudaError_t launch_apply_shifts(const uint8_t *images, int n, int w, int h, const int32_t *shifts, int fill,
                                uint8_t *out, cudaStream_t s);
cudaError_t launch_gather_quadrants(const uint8_t *images, int n, int w, int h, uint8_t *out, long long quad_stride,
                                    cudaStream_t s);
cudaError_t launch_quadrant_flags(const int32_t *quad, int n, int rot_tol, int32_t *out, int32_t *flags,
                                  cudaStream_t s);
// budget: word-candidate evaluations per pair allowed to the coarse windows.
int coarse_start_level(const mtb_layout_t &L, long long budget = kBruteBudget);
// Stream s's last-status slot on the current device: its index (-1 if there is
// none, or none may be taken without `create`) and, in *dev_slot, its device
// address.  read_last_status copies a slot's value to the host (synchronous).
int last_status_slot(cudaStream_t s, bool create, int32_t **dev_slot = nullptr);
int read_last_status(int slot, int32_t *out);
// `overlap` (only directly after launch_bitmaps of the same call, on a workspace
// the same call's launch_pyramid cleared): the search starts while the bitmaps
// are being packed and waits per bit plane.  `chain`: each exposure is searched
// against its neighbour towards ref and the shifts are composed.
cudaError_t launch_search(const mtb_layout_t &L, int ref_idx, uint8_t *ws, int32_t *shifts_out,
                          uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s, bool chained,
                          bool overlap = false, bool chain = false);
cudaError_t launch_search_ex(const mtb_layout_t &L, int ref_idx, uint8_t *ws, int32_t *shifts_out,
                             uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s, bool chained,
                             unsigned long long timeout_ns, int withhold_pair, bool overlap = false,
                             bool chain = false);

// Which kernel a search of this stack runs on the current device: 1 the
// staged kernel, 0 the item kernel, -1 on a CUDA error.
int search_kernel_choice(const mtb_layout_t &L, int ref_idx, bool overlap);

int device_sm_count();

// Host memory moved by SM loads and stores instead of copy engines.  A copy
// engine that has been idle for some milliseconds is slow to start its next
// copy (a 504 MB copy: 2.4 ms back to back, p99 19 ms with 20 ms between
// copies, p90 34 ms with 100 ms); SM loads of the same page-locked memory keep
// their pace (p99 2.4 and 4.7 ms) at the same ~210 GB/s.
// The address at which a kernel reaches host buffer p: non-null only for
// page-locked memory seen through unified addressing, 16-byte aligned.
const uint8_t *host_device_view(const void *p);
// dst[0, n) = src[0, n), src from host_device_view, dst device memory, both
// 16-byte aligned: 32 CTAs, enough to keep the host link busy.
cudaError_t launch_copy_in(const uint8_t *src, uint8_t *dst, size_t n, cudaStream_t s);
// dst_a[0, na) = src_a[0, na) and dst_b[0, nb) = src_b[0, nb) (int32 words,
// src in device memory, dst from host_device_view or null when n is 0), then a
// system-scope fence: results handed to the host with no copy engine.
cudaError_t launch_copy_out(const int32_t *src_a, int32_t *dst_a, int na, const int32_t *src_b, int32_t *dst_b,
                            int nb, cudaStream_t s);

// Whole alignment of one stack in one persistent launch (mtb_engine.cu).
cudaError_t launch_engine_single(const mtb_layout_t &L, const uint8_t *images, uint8_t *ws, int tol, int ref,
                                 int32_t *shifts_out, uint32_t *level_errs_out, int32_t *level_shifts_out,
                                 cudaStream_t s);

// Launches kernel<<<grid, block, 0, s>>>(args...).  With `after_previous` the
// launch carries the programmatic-stream-serialization attribute: it may begin
// while the previous kernel in the stream runs, and the kernel orders its
// dependent accesses with pdl_wait().  The first kernel of a call is launched
// without it, so it starts only after all earlier work in the stream.
template <typename... KArgs, typename... Args>
cudaError_t launch_k_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t dyn_smem, cudaStream_t s,
                          bool after_previous, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = dyn_smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = after_previous ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, bool after_previous,
                     Args... args) {
    return launch_k_smem(kernel, grid, block, 0, s, after_previous, args...);
}

}  // namespace mtb
