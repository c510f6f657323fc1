// mtb_noalloc.cu -- an alignment entry point that allocates no memory.
//
// Who needs it: callers that may not allocate device memory while they align.
// Examples are a per-frame video or camera loop with a hard deadline (an
// allocation can synchronise the device or wait on the memory pool), a plug-in
// whose host application owns every allocation, and code running under a fixed
// device-memory budget where an allocation might fail halfway through a job.
// mtb_align_stack allocates its workspace stream-ordered, and
// mtb_align_stack_ex needs the caller to have allocated one; this entry point
// needs neither.
//
// How: the workspace is the fixed array g_noalloc_scratch below, of
// MTB_NOALLOC_SCRATCH_BYTES.  The CUDA runtime creates it on each device where
// this module is loaded (with lazy module loading: on the first call on that
// device) and keeps it until the process exits.  Host code cannot use the
// array's name as a device address, so the first call on a device looks the
// address up with cudaGetSymbolAddress while that device is current and keeps it
// for later calls.  That first call therefore has to happen before any CUDA
// stream capture that would include a later call.
//
// Sharing: every call on a device uses the same array, which keeps whatever the
// previous call left in it.  The pipeline clears the parts that must start at
// zero (histograms, error counters) and overwrites everything else before
// reading it.  Two calls whose work overlaps on the GPU -- on different streams,
// or from different host threads -- race on the array and give wrong results;
// callers must order such calls (same stream, or events).
#include <mutex>

#include "mtb_internal.cuh"

static __device__ __align__(256) uint8_t g_noalloc_scratch[MTB_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once.
int scratch_on_current_device(uint8_t **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return MTB_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return MTB_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<uint8_t *>(g_scratch_addr[dev]);
    return MTB_OK;
}

}  // namespace

extern "C" int mtb_align_stack_noalloc(const uint8_t *images, int n_exposures, int w, int h, int levels,
                                       int noise_tol, int ref_idx, int32_t *shifts_out, uint32_t *level_errs_out,
                                       int32_t *level_shifts_out, void *stream) {
    int rc = mtb::check_stack_args(n_exposures, w, h, levels, noise_tol, ref_idx);
    if (rc != MTB_OK) return rc;
    if (!images || !shifts_out || (reinterpret_cast<uintptr_t>(images) & 15u) != 0) return MTB_ERR_INVALID_ARG;
    if (mtb_workspace_bytes(n_exposures, w, h, levels) > (size_t)MTB_NOALLOC_SCRATCH_BYTES)
        return MTB_ERR_INVALID_ARG;  // the stack does not fit in the fixed scratch array
    uint8_t *scratch = nullptr;
    rc = scratch_on_current_device(&scratch);
    if (rc != MTB_OK) return rc;
    return mtb_align_stack_ex(images, n_exposures, w, h, levels, noise_tol, ref_idx, shifts_out, level_errs_out,
                              level_shifts_out, scratch, (size_t)MTB_NOALLOC_SCRATCH_BYTES, stream);
}
