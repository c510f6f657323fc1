// mtb_api.cu -- the C ABI declared in include/mtb.h: argument checks, the
// workspace layout and the entry points that enqueue the three stages.
#include <cstring>
#include <mutex>

#include "mtb_internal.cuh"

namespace mtb {

namespace {
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int check_dims(int n, int w, int h, int levels) {
    if (n < 2 || n > MTB_MAX_EXPOSURES) return MTB_ERR_INVALID_ARG;
    if (w < 1 || h < 1 || w > MTB_MAX_DIM || h > MTB_MAX_DIM) return MTB_ERR_INVALID_ARG;
    if (levels < 1 || levels > MTB_MAX_LEVELS) return MTB_ERR_INVALID_ARG;
    if ((w >> (levels - 1)) < 1 || (h >> (levels - 1)) < 1) return MTB_ERR_INVALID_ARG;
    return MTB_OK;
}

int g_sm_count[64] = {0};
}  // namespace

int device_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (g_sm_count[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        g_sm_count[dev] = v;
    }
    return g_sm_count[dev];
}

namespace {

constexpr int kCopyCtas = 32, kCopyThreads = 256, kCopyUnroll = 8;  // eight 16-byte loads in flight a thread

__global__ void __launch_bounds__(kCopyThreads) k_copy_in(const uint4 *__restrict__ src, uint4 *__restrict__ dst,
                                                          size_t n) {
    const size_t n16 = n / 16, stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (kCopyUnroll - 1) * stride < n16; i += kCopyUnroll * stride) {
        uint4 v[kCopyUnroll];
#pragma unroll
        for (int k = 0; k < kCopyUnroll; ++k) v[k] = __ldcs(src + i + k * stride);
#pragma unroll
        for (int k = 0; k < kCopyUnroll; ++k) dst[i + k * stride] = v[k];
    }
    for (; i < n16; i += stride) dst[i] = __ldcs(src + i);
    const size_t tail = n - n16 * 16;
    if (blockIdx.x == 0 && threadIdx.x < tail)
        reinterpret_cast<uint8_t *>(dst + n16)[threadIdx.x] = reinterpret_cast<const uint8_t *>(src + n16)[threadIdx.x];
}

__global__ void k_copy_out(const int32_t *__restrict__ src_a, int32_t *dst_a, int na, const int32_t *__restrict__ src_b,
                           int32_t *dst_b, int nb) {
    for (int i = threadIdx.x; i < na; i += blockDim.x) dst_a[i] = __ldcg(src_a + i);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) dst_b[i] = __ldcg(src_b + i);
    __threadfence_system();
}

}  // namespace

const uint8_t *host_device_view(const void *p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || (reinterpret_cast<uintptr_t>(a.devicePointer) & 15))
        return nullptr;
    return static_cast<const uint8_t *>(a.devicePointer);
}

cudaError_t launch_copy_in(const uint8_t *src, uint8_t *dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_copy_in<<<kCopyCtas, kCopyThreads, 0, s>>>(reinterpret_cast<const uint4 *>(src), reinterpret_cast<uint4 *>(dst),
                                                 n);
    return cudaGetLastError();
}

cudaError_t launch_copy_out(const int32_t *src_a, int32_t *dst_a, int na, const int32_t *src_b, int32_t *dst_b,
                            int nb, cudaStream_t s) {
    k_copy_out<<<1, 64, 0, s>>>(src_a, dst_a, na, src_b, dst_b, nb);
    return cudaGetLastError();
}

int check_stack_args(int n, int w, int h, int levels, int noise_tol, int ref_idx) {
    int rc = check_dims(n, w, h, levels);
    if (rc != MTB_OK) return rc;
    if (noise_tol < 0 || noise_tol > 255) return MTB_ERR_INVALID_ARG;
    if (ref_idx < 0 || ref_idx >= n) return MTB_ERR_INVALID_ARG;
    return MTB_OK;
}

int compute_layout(int n, int w, int h, int levels, mtb_layout_t *L) {
    int rc = check_dims(n, w, h, levels);
    if (rc != MTB_OK) return rc;
    std::memset(L, 0, sizeof(*L));
    L->n = n;
    L->w = w;
    L->h = h;
    L->levels = levels;
    L->tile_levels = levels < kTileLog2 + 1 ? levels : kTileLog2 + 1;
    size_t per_exp = 0;
    for (int l = 0; l < levels; ++l) {
        L->width[l] = w >> l;
        L->height[l] = h >> l;
        L->gray_pitch[l] = (int32_t)align_up((size_t)L->width[l], 32);
        // at least 2 zero words end every row: a run of rows copied as it lies
        // has zeros on both sides of each row's data (the search reads past
        // the row ends without checks)
        L->bits_pitch[l] = (int32_t)align_up(((size_t)L->width[l] + 31) / 32 + 2, 2);
        L->gray_offset[l] = per_exp;
        per_exp += align_up((size_t)L->gray_pitch[l] * L->height[l], 256);
    }
    L->gray_exposure_stride = per_exp;
    size_t off = per_exp * n;
    size_t bits_per_exp = 0;
    for (int l = 0; l < levels; ++l) {
        L->bits_offset[l] = off + bits_per_exp;
        bits_per_exp += align_up((size_t)L->bits_pitch[l] * 8 * L->height[l], 256);
    }
    L->bits_exposure_stride = bits_per_exp;
    off += bits_per_exp * n;
    L->hist_offset = off;
    off += (size_t)n * levels * 256 * sizeof(uint32_t);
    L->counter_offset = off;  // right after hist: the pyramid stage clears both in one launch
    off += (size_t)(n * (2 * levels + 4) + 16) * sizeof(int32_t);
    off = align_up(off, 256);
    L->errs_offset = off;
    off += (size_t)n * levels * 9 * sizeof(uint32_t);
    off = align_up(off, 256);
    L->median_offset = off;
    off = align_up(off + (size_t)n * levels * sizeof(int32_t), 256);
    L->base_offset = off;
    off = align_up(off + (size_t)n * levels * 2 * sizeof(int32_t), 256);
    L->shift_offset = off;
    off = align_up(off + (size_t)n * levels * 2 * sizeof(int32_t), 256);
    L->table_offset = off;
    off = align_up(off + (size_t)n * kTableWords * sizeof(uint32_t), 256);
    L->status_offset = off;
    off = align_up(off + 4 * sizeof(int32_t), 256);
    L->total_bytes = off;
    return MTB_OK;
}

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? MTB_OK : MTB_ERR_CUDA; }

int stage_pyramid(const uint8_t *images, const mtb_layout_t &L, uint8_t *ws, cudaStream_t s) {
    return cuda_status(launch_pyramid(images, L, ws, s));
}

// One stack: the three stage kernels chained with programmatic dependent launch
// (lower latency for a single stack than the engine, whose strength is
// overlapping many stacks in a batch).
int run_all(const uint8_t *images, const mtb_layout_t &L, int tol, int ref, uint8_t *ws, int32_t *shifts_out,
            uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s, bool chain = false) {
    int rc = stage_pyramid(images, L, ws, s);
    if (rc != MTB_OK) return rc;
    rc = cuda_status(launch_bitmaps(L, tol, ws, s, true));
    if (rc != MTB_OK) return rc;
    return cuda_status(launch_search(L, ref, ws, shifts_out, level_errs_out, level_shifts_out, s, true, true, chain));
}


// ---- host-buffer entry: the copy in, in row bands, overlapped with the pyramid ----
// The RGB is copied in bands of whole tile rows of one exposure on a copy
// stream the library owns (one per device); after each band's copy the
// pyramid pass over that band's tiles is launched on the caller's stream, so
// only the last band's pyramid, the bitmaps and the search follow the copy.
constexpr int kMaxBands = 32;
constexpr size_t kBandBytes = 16u << 20;  // target bytes per band copy
constexpr size_t kBandMinStack = 8u << 20;  // smaller stacks are copied in one piece

struct CopyPipe {
    std::mutex mu;  // held while a call enqueues (its events are reused by the next call)
    bool ready = false;
    cudaStream_t copy = nullptr;
    cudaEvent_t start = nullptr;
    cudaEvent_t band[kMaxBands] = {};
};
CopyPipe g_pipes[64];
std::mutex g_pipes_mu;

// The calling thread's device's pipe, created on first use; nullptr on error.
CopyPipe *copy_pipe() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    CopyPipe &p = g_pipes[dev];
    std::lock_guard<std::mutex> g(g_pipes_mu);
    if (!p.ready) {
        // all or nothing: a failed setup releases what it made, and the next
        // call tries again from scratch
        cudaStream_t copy = nullptr;
        cudaEvent_t ev[1 + kMaxBands] = {};
        bool ok = cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking) == cudaSuccess;
        for (int k = 0; ok && k <= kMaxBands; ++k)
            ok = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            for (cudaEvent_t e : ev)
                if (e) cudaEventDestroy(e);
            if (copy) cudaStreamDestroy(copy);
            cudaGetLastError();
            return nullptr;
        }
        p.copy = copy;
        p.start = ev[0];
        for (int k = 0; k < kMaxBands; ++k) p.band[k] = ev[1 + k];
        p.ready = true;
    }
    return &p;
}

// Bands of tile rows per exposure: about kBandBytes each, at most kMaxBands in
// all; 0 when the stack is copied in one piece.
int bands_per_exposure(const mtb_layout_t &L, size_t img_bytes) {
    if (img_bytes < kBandMinStack) return 0;
    const long long tile_rows = (L.h + kTileRows - 1) / kTileRows;
    const size_t exp_bytes = img_bytes / L.n;
    long long b = (long long)((exp_bytes + kBandBytes / 2) / kBandBytes);
    if (b < 1) b = 1;
    if (b > tile_rows) b = tile_rows;
    while (b > 1 && b * L.n > kMaxBands) --b;
    return b * L.n > kMaxBands ? 0 : (int)b;
}

// Enqueues the banded copy of host_images into d_img and, on s, the clear and
// the pyramid pass band by band; the bitmaps and search are chained after.  On
// a failure after the first copy, waits for the copies so that the caller may
// release the device buffer.
int enqueue_banded(const uint8_t *host_images, uint8_t *d_img, const mtb_layout_t &L, int bands, uint8_t *ws,
                   cudaStream_t s) {
    CopyPipe *p = copy_pipe();
    if (!p) return MTB_ERR_CUDA;
    std::lock_guard<std::mutex> g(p->mu);
    const long long tile_rows = (L.h + kTileRows - 1) / kTileRows;
    const long long tiles_x = pyramid_tiles_x(L);
    const long long per_exp = pyramid_tiles_per_exposure(L);
    const size_t row_bytes = (size_t)L.w * 3;
    // the copy must not overwrite the device images while earlier work on s
    // (a previous call on the same workspace) may still read them
    if (cudaEventRecord(p->start, s) != cudaSuccess || cudaStreamWaitEvent(p->copy, p->start, 0) != cudaSuccess)
        return MTB_ERR_CUDA;
    auto fail = [&]() {
        cudaStreamSynchronize(p->copy);
        return MTB_ERR_CUDA;
    };
    // the bands go through the copy engine: a copy kernel would wait for SMs
    // held by the previous band's pyramid pass, so the copy and the pyramid
    // would no longer overlap (6000x4000x7 end to end: 2.85 ms with the copy
    // kernel, 2.62 ms with the copy engine)
    int k = 0;
    for (int e = 0; e < L.n; ++e)
        for (int b = 0; b < bands; ++b, ++k) {
            const long long r0 = tile_rows * b / bands, r1 = tile_rows * (b + 1) / bands;
            const size_t y0 = (size_t)r0 * kTileRows, y1 = (size_t)(r1 * kTileRows < L.h ? r1 * kTileRows : L.h);
            const size_t off = ((size_t)e * L.h + y0) * row_bytes, len = (y1 - y0) * row_bytes;
            const cudaError_t err =
                cudaMemcpyAsync(d_img + off, host_images + off, len, cudaMemcpyHostToDevice, p->copy);
            if (err != cudaSuccess || cudaEventRecord(p->band[k], p->copy) != cudaSuccess) return fail();
        }
    if (launch_clear_stack(L, ws, s) != cudaSuccess) return fail();
    k = 0;
    for (int e = 0; e < L.n; ++e)
        for (int b = 0; b < bands; ++b, ++k) {
            const long long r0 = tile_rows * b / bands, r1 = tile_rows * (b + 1) / bands;
            if (cudaStreamWaitEvent(s, p->band[k], 0) != cudaSuccess) return fail();
            const long long t0 = e * per_exp + r0 * tiles_x, t1 = e * per_exp + r1 * tiles_x;
            if (launch_pyramid_range(d_img, L, ws, t0, t1, s, false) != cudaSuccess) return fail();
        }
    return MTB_OK;
}

bool misaligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; }

// Whether the byte ranges [a, a + na) and [b, b + nb) share a byte (a null
// pointer or an empty range shares none).
bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    if (!a || !b || na == 0 || nb == 0) return false;
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

// The outputs of an alignment call must not overlap the images, and a caller
// workspace none of them: the kernels write the workspace and the outputs
// while they read the images.
bool buffers_alias(const uint8_t *images, int n, int w, int h, int levels, const void *shifts_out,
                   const void *level_errs_out, const void *level_shifts_out, const void *workspace,
                   size_t workspace_bytes) {
    const size_t img = (size_t)n * w * h * 3;
    const size_t sh = (size_t)n * 2 * sizeof(int32_t), le = (size_t)n * levels * 9 * sizeof(uint32_t),
                 ls = (size_t)n * levels * 2 * sizeof(int32_t);
    const void *outs[3] = {shifts_out, level_errs_out, level_shifts_out};
    const size_t sizes[3] = {sh, le, ls};
    for (int k = 0; k < 3; ++k) {
        if (overlaps(outs[k], sizes[k], images, img) || overlaps(outs[k], sizes[k], workspace, workspace_bytes))
            return true;
        for (int j = k + 1; j < 3; ++j)
            if (overlaps(outs[k], sizes[k], outs[j], sizes[j])) return true;
    }
    return overlaps(workspace, workspace_bytes, images, img);
}

// Caller workspace if given (checked), else a stream-ordered allocation.
int acquire(void *given, size_t given_bytes, size_t need, cudaStream_t s, uint8_t **ws, bool *owned) {
    *owned = false;
    if (given) {
        if (given_bytes < need || misaligned(given, 256)) return MTB_ERR_INVALID_ARG;
        *ws = static_cast<uint8_t *>(given);
        return MTB_OK;
    }
    void *p = nullptr;
    if (cudaMallocAsync(&p, need, s) != cudaSuccess) {
        cudaGetLastError();
        return MTB_ERR_OOM;
    }
    *ws = static_cast<uint8_t *>(p);
    *owned = true;
    return MTB_OK;
}

int release(uint8_t *ws, bool owned, cudaStream_t s, int rc) {
    if (owned && cudaFreeAsync(ws, s) != cudaSuccess && rc == MTB_OK) rc = MTB_ERR_CUDA;
    return rc;
}

}  // namespace
}  // namespace mtb

using namespace mtb;

extern "C" {

const char *mtb_status_string(int status) {
    switch (status) {
        case MTB_OK: return "ok";
        case MTB_ERR_INVALID_ARG: return "invalid argument";
        case MTB_ERR_OOM: return "out of memory";
        case MTB_ERR_CUDA: return "CUDA error";
        case MTB_ERR_TIMEOUT: return "device wait timed out";
        case MTB_ERR_BUSY: return "over budget";
        default: return "unknown status";
    }
}

int mtb_abi_version(void) { return 1; }

int mtb_get_last_status(void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return MTB_ERR_CUDA;
    const int slot = last_status_slot(s, false);
    if (slot < 0) return MTB_OK;  // no search was ever launched on this stream
    int32_t v = MTB_OK;
    if (read_last_status(slot, &v) != MTB_OK) return MTB_ERR_CUDA;
    return v;
}

size_t mtb_workspace_bytes(int n_exposures, int w, int h, int levels) {
    mtb_layout_t L;
    if (compute_layout(n_exposures, w, h, levels, &L) != MTB_OK) return 0;
    return L.total_bytes;
}

int mtb_workspace_layout(int n_exposures, int w, int h, int levels, mtb_layout_t *out) {
    if (!out) return MTB_ERR_INVALID_ARG;
    return compute_layout(n_exposures, w, h, levels, out);
}

int mtb_align_stack_ex(const uint8_t *images, int n_exposures, int w, int h, int levels, int noise_tol,
                       int ref_idx, int32_t *shifts_out, uint32_t *level_errs_out, int32_t *level_shifts_out,
                       void *workspace, size_t workspace_bytes, void *stream) {
    int rc = check_stack_args(n_exposures, w, h, levels, noise_tol, ref_idx);
    if (rc != MTB_OK) return rc;
    if (!images || !shifts_out || misaligned(images, 16)) return MTB_ERR_INVALID_ARG;
    if (buffers_alias(images, n_exposures, w, h, levels, shifts_out, level_errs_out, level_shifts_out, workspace,
                      workspace_bytes))
        return MTB_ERR_INVALID_ARG;
    mtb_layout_t L;
    compute_layout(n_exposures, w, h, levels, &L);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *ws = nullptr;
    bool owned = false;
    rc = acquire(workspace, workspace_bytes, L.total_bytes, s, &ws, &owned);
    if (rc != MTB_OK) return rc;
    rc = run_all(images, L, noise_tol, ref_idx, ws, shifts_out, level_errs_out, level_shifts_out, s);
    return release(ws, owned, s, rc);
}

int mtb_align_stack_chain(const uint8_t *images, int n_exposures, int w, int h, int levels, int noise_tol,
                          int ref_idx, int32_t *shifts_out, uint32_t *level_errs_out, int32_t *level_shifts_out,
                          void *workspace, size_t workspace_bytes, void *stream) {
    int rc = check_stack_args(n_exposures, w, h, levels, noise_tol, ref_idx);
    if (rc != MTB_OK) return rc;
    if (!images || !shifts_out || misaligned(images, 16)) return MTB_ERR_INVALID_ARG;
    if (buffers_alias(images, n_exposures, w, h, levels, shifts_out, level_errs_out, level_shifts_out, workspace,
                      workspace_bytes))
        return MTB_ERR_INVALID_ARG;
    mtb_layout_t L;
    compute_layout(n_exposures, w, h, levels, &L);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *ws = nullptr;
    bool owned = false;
    rc = acquire(workspace, workspace_bytes, L.total_bytes, s, &ws, &owned);
    if (rc != MTB_OK) return rc;
    rc = run_all(images, L, noise_tol, ref_idx, ws, shifts_out, level_errs_out, level_shifts_out, s, true);
    return release(ws, owned, s, rc);
}

int mtb_align_stack(const uint8_t *images, int n_exposures, int w, int h, int levels, int noise_tol, int ref_idx,
                    int32_t *shifts_out, void *stream) {
    return mtb_align_stack_ex(images, n_exposures, w, h, levels, noise_tol, ref_idx, shifts_out, nullptr, nullptr,
                              nullptr, 0, stream);
}

int mtb_build_pyramids(const uint8_t *images, int n_exposures, int w, int h, int levels, void *workspace,
                       size_t workspace_bytes, void *stream) {
    mtb_layout_t L;
    int rc = compute_layout(n_exposures, w, h, levels, &L);
    if (rc != MTB_OK) return rc;
    if (!images || misaligned(images, 16) || !workspace || workspace_bytes < L.total_bytes ||
        misaligned(workspace, 256))
        return MTB_ERR_INVALID_ARG;
    if (overlaps(workspace, workspace_bytes, images, (size_t)n_exposures * w * h * 3)) return MTB_ERR_INVALID_ARG;
    return stage_pyramid(images, L, static_cast<uint8_t *>(workspace), static_cast<cudaStream_t>(stream));
}

int mtb_build_bitmaps(int n_exposures, int w, int h, int levels, int noise_tol, void *workspace,
                      size_t workspace_bytes, void *stream) {
    mtb_layout_t L;
    int rc = compute_layout(n_exposures, w, h, levels, &L);
    if (rc != MTB_OK) return rc;
    if (noise_tol < 0 || noise_tol > 255) return MTB_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < L.total_bytes || misaligned(workspace, 256)) return MTB_ERR_INVALID_ARG;
    return cuda_status(launch_bitmaps(L, noise_tol, static_cast<uint8_t *>(workspace),
                                      static_cast<cudaStream_t>(stream), false));
}

int mtb_search_shifts(int n_exposures, int w, int h, int levels, int ref_idx, void *workspace,
                      size_t workspace_bytes, int32_t *shifts_out, uint32_t *level_errs_out,
                      int32_t *level_shifts_out, void *stream) {
    mtb_layout_t L;
    int rc = compute_layout(n_exposures, w, h, levels, &L);
    if (rc != MTB_OK) return rc;
    if (ref_idx < 0 || ref_idx >= n_exposures) return MTB_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < L.total_bytes || misaligned(workspace, 256)) return MTB_ERR_INVALID_ARG;
    if (buffers_alias(nullptr, n_exposures, w, h, levels, shifts_out, level_errs_out, level_shifts_out, workspace,
                      workspace_bytes))
        return MTB_ERR_INVALID_ARG;
    return cuda_status(launch_search(L, ref_idx, static_cast<uint8_t *>(workspace), shifts_out, level_errs_out,
                                     level_shifts_out, static_cast<cudaStream_t>(stream), false));
}

int mtb_workspace_status(const void *workspace, size_t workspace_bytes, int n_exposures, int w, int h, int levels,
                         void *stream) {
    mtb_layout_t L;
    int rc = compute_layout(n_exposures, w, h, levels, &L);
    if (rc != MTB_OK) return rc;
    if (!workspace || workspace_bytes < L.total_bytes || misaligned(workspace, 256)) return MTB_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return MTB_ERR_CUDA;
    int32_t status = 0;
    if (cudaMemcpy(&status, static_cast<const uint8_t *>(workspace) + L.status_offset, sizeof(status),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return MTB_ERR_CUDA;
    return status;
}

int mtb_search_kernel(int n_exposures, int w, int h, int levels, int ref_idx, int chained) {
    const int rc = check_stack_args(n_exposures, w, h, levels, 0, ref_idx);
    if (rc != MTB_OK) return rc;
    mtb_layout_t L;
    compute_layout(n_exposures, w, h, levels, &L);
    const int k = search_kernel_choice(L, ref_idx, chained != 0);
    return k < 0 ? MTB_ERR_CUDA : k;
}

int mtb_debug_search_withheld(int n_exposures, int w, int h, int levels, int ref_idx, void *workspace,
                              size_t workspace_bytes, long long timeout_ns, void *stream) {
    mtb_layout_t L;
    int rc = compute_layout(n_exposures, w, h, levels, &L);
    if (rc != MTB_OK) return rc;
    if (ref_idx < 0 || ref_idx >= n_exposures || timeout_ns <= 0 || timeout_ns > 1000000000LL)
        return MTB_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < L.total_bytes || misaligned(workspace, 256)) return MTB_ERR_INVALID_ARG;
    if (coarse_start_level(L) >= L.levels) return MTB_ERR_INVALID_ARG;  // no resolve item to withhold
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = cuda_status(launch_search_ex(L, ref_idx, static_cast<uint8_t *>(workspace), nullptr, nullptr, nullptr, s,
                                      false, (unsigned long long)timeout_ns, 0));
    if (rc != MTB_OK) return rc;
    return mtb_workspace_status(workspace, workspace_bytes, n_exposures, w, h, levels, stream);
}

size_t mtb_host_workspace_bytes(int n_exposures, int w, int h, int levels) {
    mtb_layout_t L;
    if (compute_layout(n_exposures, w, h, levels, &L) != MTB_OK) return 0;
    const size_t img = align_up((size_t)n_exposures * w * h * 3, 256);
    return img + L.total_bytes + align_up((size_t)n_exposures * 2 * sizeof(int32_t), 256);
}

int mtb_align_stack_host(const uint8_t *host_images, int n_exposures, int w, int h, int levels, int noise_tol,
                         int ref_idx, int32_t *host_shifts_out, void *device_workspace,
                         size_t device_workspace_bytes, void *stream) {
    int rc = check_stack_args(n_exposures, w, h, levels, noise_tol, ref_idx);
    if (rc != MTB_OK) return rc;
    if (!host_images || !host_shifts_out) return MTB_ERR_INVALID_ARG;
    mtb_layout_t L;
    compute_layout(n_exposures, w, h, levels, &L);
    const size_t img_bytes = (size_t)n_exposures * w * h * 3;
    const size_t need = mtb_host_workspace_bytes(n_exposures, w, h, levels);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *base = nullptr;
    bool owned = false;
    rc = acquire(device_workspace, device_workspace_bytes, need, s, &base, &owned);
    if (rc != MTB_OK) return rc;
    uint8_t *d_img = base;
    uint8_t *ws = base + align_up(img_bytes, 256);
    int32_t *d_shifts = reinterpret_cast<int32_t *>(ws + L.total_bytes);
    const int bands = bands_per_exposure(L, img_bytes);
    if (bands > 0) {
        rc = enqueue_banded(host_images, d_img, L, bands, ws, s);
        if (rc == MTB_OK) rc = cuda_status(launch_bitmaps(L, noise_tol, ws, s, true));
        if (rc == MTB_OK)
            rc = cuda_status(launch_search(L, ref_idx, ws, d_shifts, nullptr, nullptr, s, true, true, false));
    } else {
        const uint8_t *view = host_device_view(host_images);
        rc = cuda_status(view ? launch_copy_in(view, d_img, img_bytes, s)
                              : cudaMemcpyAsync(d_img, host_images, img_bytes, cudaMemcpyHostToDevice, s));
        if (rc == MTB_OK) rc = run_all(d_img, L, noise_tol, ref_idx, ws, d_shifts, nullptr, nullptr, s);
    }
    if (rc == MTB_OK) {
        // page-locked output is written by SM stores, like the input
        int32_t *out_view = reinterpret_cast<int32_t *>(const_cast<uint8_t *>(host_device_view(host_shifts_out)));
        rc = cuda_status(out_view ? launch_copy_out(d_shifts, out_view, n_exposures * 2, nullptr, nullptr, 0, s)
                                  : cudaMemcpyAsync(host_shifts_out, d_shifts,
                                                    (size_t)n_exposures * 2 * sizeof(int32_t),
                                                    cudaMemcpyDeviceToHost, s));
    }
    rc = release(base, owned, s, rc);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == MTB_OK) rc = MTB_ERR_CUDA;
    return rc;
}

// Quadrant workspace: the four quadrant stacks, one alignment workspace used by
// the four alignments in turn, and their shifts [4][n][2].
static int quadrant_layout(int n, int w, int h, int levels, mtb_layout_t *Lq, size_t *quad_stride,
                           size_t *ws_offset, size_t *shifts_offset, size_t *total) {
    const int wq = w / 2, hq = h / 2;
    int rc = compute_layout(n, wq, hq, levels, Lq);
    if (rc != MTB_OK) return rc;
    *quad_stride = align_up((size_t)n * wq * hq * 3, 256);
    *ws_offset = 4 * *quad_stride;
    *shifts_offset = *ws_offset + align_up(Lq->total_bytes, 256);
    *total = *shifts_offset + align_up((size_t)4 * n * 2 * sizeof(int32_t), 256);
    return MTB_OK;
}

size_t mtb_quadrant_workspace_bytes(int n_exposures, int w, int h, int levels) {
    mtb_layout_t Lq;
    size_t stride, wso, so, total;
    if (w < 2 || h < 2 || quadrant_layout(n_exposures, w, h, levels, &Lq, &stride, &wso, &so, &total) != MTB_OK)
        return 0;
    return total;
}

int mtb_align_quadrants(const uint8_t *images, int n_exposures, int w, int h, int levels, int noise_tol, int ref_idx,
                        int rot_tol, int32_t *quad_shifts_out, int32_t *flags_out, void *workspace,
                        size_t workspace_bytes, void *stream) {
    if (w < 2 || h < 2 || w > MTB_MAX_DIM || h > MTB_MAX_DIM || rot_tol < 0) return MTB_ERR_INVALID_ARG;
    int rc = check_stack_args(n_exposures, w / 2, h / 2, levels, noise_tol, ref_idx);
    if (rc != MTB_OK) return rc;
    if (!images || !quad_shifts_out || misaligned(images, 16)) return MTB_ERR_INVALID_ARG;
    mtb_layout_t Lq;
    size_t stride, wso, so, total;
    quadrant_layout(n_exposures, w, h, levels, &Lq, &stride, &wso, &so, &total);
    {
        const size_t img = (size_t)n_exposures * w * h * 3, qs = (size_t)n_exposures * 4 * 2 * sizeof(int32_t),
                     fl = (size_t)n_exposures * sizeof(int32_t);
        if (overlaps(workspace, workspace_bytes, images, img) || overlaps(quad_shifts_out, qs, images, img) ||
            overlaps(quad_shifts_out, qs, workspace, workspace_bytes) || overlaps(flags_out, fl, images, img) ||
            overlaps(flags_out, fl, workspace, workspace_bytes) || overlaps(flags_out, fl, quad_shifts_out, qs))
            return MTB_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *base = nullptr;
    bool owned = false;
    rc = acquire(workspace, workspace_bytes, total, s, &base, &owned);
    if (rc != MTB_OK) return rc;
    int32_t *quad = reinterpret_cast<int32_t *>(base + so);
    rc = cuda_status(launch_gather_quadrants(images, n_exposures, w, h, base, (long long)stride, s));
    for (int q = 0; q < 4 && rc == MTB_OK; ++q)
        rc = run_all(base + q * stride, Lq, noise_tol, ref_idx, base + wso, quad + (size_t)q * n_exposures * 2,
                     nullptr, nullptr, s);
    if (rc == MTB_OK)
        rc = cuda_status(launch_quadrant_flags(quad, n_exposures, rot_tol, quad_shifts_out, flags_out, s));
    return release(base, owned, s, rc);
}

int mtb_apply_shifts(const uint8_t *images, int n_exposures, int w, int h, const int32_t *shifts, int fill,
                     uint8_t *out, void *stream) {
    if (n_exposures < 1 || n_exposures > MTB_MAX_EXPOSURES || w < 1 || h < 1 || w > MTB_MAX_DIM ||
        h > MTB_MAX_DIM || (fill != MTB_FILL_ZERO && fill != MTB_FILL_EDGE))
        return MTB_ERR_INVALID_ARG;
    if (!images || !shifts || !out || misaligned(images, 16) || misaligned(out, 16) || misaligned(shifts, 4))
        return MTB_ERR_INVALID_ARG;
    const uintptr_t bytes = (uintptr_t)n_exposures * w * h * 3;
    const uintptr_t a = reinterpret_cast<uintptr_t>(images), b = reinterpret_cast<uintptr_t>(out);
    if (a < b + bytes && b < a + bytes) return MTB_ERR_INVALID_ARG;  // overlapping buffers
    return cuda_status(launch_apply_shifts(images, n_exposures, w, h, shifts, fill, out,
                                           static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
