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
// for later calls, together with the identity of the context it belongs to.  A
// context destroyed and created again (cudaDeviceReset) loads the module again
// and may place the array elsewhere, so a call that finds another context
// current looks the address up again.  The first call on a device, and the
// first call after such a reset, therefore has to happen before any CUDA stream
// capture that would include a later call.
//
// Sharing: every call on a device uses the same array, which keeps whatever the
// previous call left in it.  The pipeline clears the parts that must start at
// zero (histograms, error counters) and overwrites everything else before
// reading it.  Two calls whose work overlaps on the GPU -- on different streams,
// or from different host threads -- race on the array and give wrong results;
// callers must order such calls (same stream, or events).
#include <cuda.h>  // CUcontext and CUresult only: the driver calls are fetched through the runtime

#include <mutex>

#include "mtb_internal.cuh"

static __device__ __align__(256) uint8_t g_noalloc_scratch[MTB_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
struct ScratchAddr {
    unsigned long long ctx_id = 0;  // context the address was looked up in (0: none yet)
    void *addr = nullptr;
};
std::mutex g_scratch_mutex;
ScratchAddr g_scratch_addr[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Driver id of the calling thread's current context (ids are never reused in a
// process), or 0 if it cannot be read, in which case every call looks the
// address up again.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_noalloc_scratch in the current context, looked up once
// per context.
int scratch_on_current_device(uint8_t **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return MTB_ERR_CUDA;
    }
    // cudaGetDevice does not create the context; the lookup below does, so the
    // id is read again after it
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchAddr &c = g_scratch_addr[dev];
    if (c.addr == nullptr || id == 0 || c.ctx_id != id) {
        void *p = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            c = ScratchAddr{};
            return MTB_ERR_CUDA;
        }
        c.addr = p;
        c.ctx_id = current_context_id();
    }
    *out = static_cast<uint8_t *>(c.addr);
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
