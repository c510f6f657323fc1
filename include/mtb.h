/*
 * mtb.h -- C ABI of the GB300 median-threshold-bitmap (MTB) alignment library.
 *
 * The library aligns the exposures of an HDR stack by a global integer
 * translation, following Ward's MTB method as Alpay, Aydemir & Temizel,
 * "Accelerating Translational Image Registration for HDR Images on GPU"
 * (arXiv 2007.06483), describe it:
 *   Sec. III-A  gray conversion, per-level histogram and median, the threshold
 *               bitmap (pixel <= median -> 0, else 1), a pyramid made by halving
 *               both dimensions, and a coarse-to-fine search testing +-1 pixel in
 *               x and y (9 candidates) per level, the offset doubled per level;
 *   Sec. III-B  the exclusion bitmap (pixels within +-tol of the median removed),
 *               the error of a candidate = number of pixels set in
 *               (MTB_ref XOR MTB_shifted) AND EB_ref AND EB_shifted, and pairwise
 *               alignment of a stack whose pyramids are built once.
 *
 * Readings fixed where the paper is silent (the CUDA code states each again):
 *   gray      (4899 R + 9617 G + 1868 B + 8192) >> 14, channels in R,G,B order
 *   shrink    2x2 mean rounded half up; level l is floor(w/2^l) x floor(h/2^l)
 *   levels    number of pyramid images, full resolution included
 *   median    lower median (smallest v with cumulative count >= ceil(N/2))
 *   bitmaps   tb = [g > m], eb = [g < m - tol or g > m + tol]
 *   shift     exposure i's maps move by (sx, sy): S(b)(x,y) = b(x-sx, y-sy),
 *             0 outside the image; the reference is never moved
 *   order     candidate k: 0 = (0,0), then (dx,dy) with dy outer and dx inner
 *             over -1,0,+1 skipping (0,0); the first minimum in k order wins
 *   pairs     every exposure i != ref_idx is aligned directly to ref_idx
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA device (or managed) addresses on the current
 *     device; host pointers are ordinary (preferably pinned) host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device entry points only enqueue work and return; results are valid once
 *     the stream has reached them.  Host entry points return when done.
 *   - Images are [n][h][w][3] uint8, RGB interleaved, row pitch 3*w bytes, the
 *     exposures back to back, base address 16-byte aligned.
 *   - Shifts are int32 (sx, sy) pairs: the translation to apply to exposure i so
 *     that it lines up with exposure ref_idx; the ref_idx row is (0, 0).
 *   - The caller owns every buffer it passes.  Between calls the library keeps
 *     only per-device state made on first use and held until the process exits
 *     (the copy stream and events of mtb_align_stack_host, the last-status
 *     array of mtb_get_last_status, the scratch array of
 *     mtb_align_stack_noalloc), besides buffers it allocated and frees
 *     stream-ordered on the caller's stream.
 *   - Return value: MTB_OK or one of the negative MTB_ERR_* codes.  Arguments are
 *     checked before anything is enqueued; an invalid call enqueues nothing.
 */
#ifndef MTB_H_
#define MTB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MTB_OK 0
#define MTB_ERR_INVALID_ARG (-1) /* a size, index, tolerance or pointer is out of range */
#define MTB_ERR_OOM (-2)         /* device or host memory could not be allocated */
#define MTB_ERR_CUDA (-3)        /* a CUDA call or kernel launch failed */
#define MTB_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up */
#define MTB_ERR_BUSY (-5)        /* a server could not admit work within its budget */

#define MTB_MAX_LEVELS 16
#define MTB_MAX_EXPOSURES 4096
#define MTB_MAX_DIM 65535

/* Workspace layout of one stack, in bytes from the workspace base.  Per level l
 * (0 = full resolution):
 *   gray plane   uint8 [height[l]][gray_pitch[l]], at gray_offset[l] +
 *                e * gray_exposure_stride for exposure e
 *   bit plane    uint32 pairs (tb word, eb word) [height[l]][bits_pitch[l]], at
 *                bits_offset[l] + e * bits_exposure_stride; bit b of word q of a
 *                row is pixel 32*q + b; bits at x >= width[l] are 0, and the
 *                last 2 words of every row hold no pixel
 *   hist         uint32 [n][levels][256]
 *   median       int32  [n][levels]
 *   errs         uint32 [n][levels][9]   (candidate errors, reference row 0)
 *   base         int32  [n][levels][2]   (search offset each level starts from)
 *   shift        int32  [n][levels][2]   (best shift chosen at each level)
 *   table        uint32 [n][1280]         (candidate errors of whole search windows
 *                                         at the coarsest levels, per pair)
 *   counters     int32  [n * (2 * levels + 4) + 16] (completion counters of the kernels)
 *   status       int32 [4]               (device status words) */
typedef struct mtb_layout {
    int32_t n, w, h, levels;
    int32_t tile_levels; /* levels 0..tile_levels-1 come from the pyramid pass */
    int32_t width[MTB_MAX_LEVELS];
    int32_t height[MTB_MAX_LEVELS];
    int32_t gray_pitch[MTB_MAX_LEVELS]; /* bytes per gray row (multiple of 32) */
    int32_t bits_pitch[MTB_MAX_LEVELS]; /* 8-byte (tb, eb) words per row (even) */
    uint64_t gray_offset[MTB_MAX_LEVELS];
    uint64_t gray_exposure_stride;
    uint64_t bits_offset[MTB_MAX_LEVELS];
    uint64_t bits_exposure_stride;
    uint64_t hist_offset;
    uint64_t median_offset;
    uint64_t errs_offset;
    uint64_t base_offset;
    uint64_t shift_offset;
    uint64_t table_offset;
    uint64_t counter_offset;
    uint64_t status_offset;
    uint64_t total_bytes;
} mtb_layout_t;

/* Text for a status code (static storage; never NULL). */
const char *mtb_status_string(int status);

/* ABI version of this header: 1. */
int mtb_abi_version(void);

/* Bytes of device workspace one stack needs (0 if the sizes are invalid).
 * Host only; enqueues nothing. */
size_t mtb_workspace_bytes(int n_exposures, int w, int h, int levels);

/* Fill *out with the workspace layout of a stack.  Host only. */
int mtb_workspace_layout(int n_exposures, int w, int h, int levels, mtb_layout_t *out);

/* Align a stack (Sec. III-A, III-B).  images: device [n][h][w][3] uint8;
 * shifts_out: device int32 [n][2].  The workspace is allocated and freed
 * stream-ordered (cudaMallocAsync / cudaFreeAsync) on `stream`.
 * Requires 2 <= n <= MTB_MAX_EXPOSURES, 1 <= w, h <= MTB_MAX_DIM,
 * 1 <= levels <= MTB_MAX_LEVELS with (w >> (levels-1)) >= 1 and
 * (h >> (levels-1)) >= 1, 0 <= noise_tol <= 255, 0 <= ref_idx < n. */
int mtb_align_stack(const uint8_t *images, int n_exposures, int w, int h, int levels,
                    int noise_tol, int ref_idx, int32_t *shifts_out, void *stream);

/* As mtb_align_stack, plus optional per-level outputs and a caller workspace.
 * level_errs_out: device uint32 [n][levels][9] or NULL -- the 9 candidate errors
 *   of every level (Sec. III-A: 9 tests per level), reference row 0.
 * level_shifts_out: device int32 [n][levels][2] or NULL -- the shift chosen at
 *   every level; level 0 equals shifts_out.
 * workspace: device, 256-byte aligned, >= mtb_workspace_bytes(...) bytes, or
 *   NULL to allocate stream-ordered.  The call overwrites it entirely. */
int mtb_align_stack_ex(const uint8_t *images, int n_exposures, int w, int h, int levels,
                       int noise_tol, int ref_idx, int32_t *shifts_out,
                       uint32_t *level_errs_out, int32_t *level_shifts_out,
                       void *workspace, size_t workspace_bytes, void *stream);

/* Consecutive-chain alignment.  Sec. II recalls that each exposure can be
 * compared with its neighbours; Sec. III-B still takes n - 1 pair alignments.
 * Here exposure i != ref_idx is searched against its neighbour towards ref_idx
 * (i + 1 below it, i - 1 above it) and the translations add up along the chain:
 * shifts_out[i] = the pair's shift + shifts_out[neighbour], shifts_out[ref] =
 * (0, 0).  level_errs_out / level_shifts_out rows hold the pair (neighbour, i)
 * values (level 0 of level_shifts_out is the pair's own shift).  Arguments,
 * workspace and errors as in mtb_align_stack_ex. */
int mtb_align_stack_chain(const uint8_t *images, int n_exposures, int w, int h, int levels,
                          int noise_tol, int ref_idx, int32_t *shifts_out,
                          uint32_t *level_errs_out, int32_t *level_shifts_out,
                          void *workspace, size_t workspace_bytes, void *stream);

/* Stage 1 (Sec. III-A gray conversion and pyramid, Sec. III-B histograms):
 * clears every area after the bit planes (histograms, counters, errors,
 * medians, bases, shifts, window tables, status), then writes the gray planes,
 * histograms and medians of levels 0..tile_levels-1 into the workspace. */
int mtb_build_pyramids(const uint8_t *images, int n_exposures, int w, int h, int levels,
                       void *workspace, size_t workspace_bytes, void *stream);

/* Stage 2 (Sec. III-A median and MTB, Sec. III-B exclusion bitmap): needs
 * stage 1 in the same workspace.  Writes both bit planes of every level, and
 * the gray planes, histograms and medians of levels tile_levels..levels-1. */
int mtb_build_bitmaps(int n_exposures, int w, int h, int levels, int noise_tol,
                      void *workspace, size_t workspace_bytes, void *stream);

/* Stage 3 (Sec. III-A coarse-to-fine search, Sec. III-B error count): needs
 * stage 2 in the same workspace.  Outputs as in mtb_align_stack_ex (each may be
 * NULL); overwrites the error, base and shift areas. */
int mtb_search_shifts(int n_exposures, int w, int h, int levels, int ref_idx,
                      void *workspace, size_t workspace_bytes, int32_t *shifts_out,
                      uint32_t *level_errs_out, int32_t *level_shifts_out, void *stream);

/* Status of the device-side work of the last search enqueued on `stream` (by
 * any entry point that runs the shift search on a stream; batches report
 * through mtb_batch_status): MTB_OK, or MTB_ERR_TIMEOUT if a bounded
 * device-side wait gave up.  Waits for `stream` first.  MTB_OK if no search
 * was ever enqueued on `stream`; MTB_ERR_CUDA if the wait fails.  Unlike
 * mtb_workspace_status it needs no workspace, so it also serves calls whose
 * workspace the library allocated and has freed.  The library keeps the
 * status of the 256 most recent streams per device in a static device array;
 * it allocates nothing. */
int mtb_get_last_status(void *stream);

/* Status word of the last search run in `workspace` (sizes as when it ran):
 * MTB_OK, or MTB_ERR_TIMEOUT if a bounded device-side wait gave up.  Waits for
 * `stream` first, then copies 4 bytes to the host.  Device-side waits only end
 * by timeout if the library has a bug; the results of such a run are invalid. */
int mtb_workspace_status(const void *workspace, size_t workspace_bytes, int n_exposures, int w, int h, int levels,
                         void *stream);

/* Which of the library's two search kernels a search of this stack runs on the
 * calling thread's current device: 1 the staged kernel (bit planes staged in
 * shared memory, coarse levels on thread-block clusters), 0 the item kernel
 * (persistent work queue).  chained != 0: the search of a whole-stack call
 * (mtb_align_stack*), which starts while the bitmaps are still being packed;
 * 0: mtb_search_shifts on its own.  Both compute the same result (Sec. III-A,
 * III-B); the paper has one search, so this query has no counterpart in it.
 * Returns MTB_ERR_INVALID_ARG for an invalid stack, MTB_ERR_CUDA if the device
 * cannot be queried.  Host only; enqueues nothing. */
int mtb_search_kernel(int n_exposures, int w, int h, int levels, int ref_idx, int chained);

/* Test hook with no counterpart in the paper: runs the search of stage 3 with
 * pair 0's coarse-level work withholding its completion signal, so the work that
 * depends on it waits until timeout_ns (1 ns .. 1 s) runs out.  Returns the
 * status afterwards: MTB_ERR_TIMEOUT shows that the bounded waits end and
 * report instead of hanging.  Needs stage 2 in the workspace and at least one
 * coarse level (MTB_ERR_INVALID_ARG otherwise); outputs nothing. */
int mtb_debug_search_withheld(int n_exposures, int w, int h, int levels, int ref_idx, void *workspace,
                              size_t workspace_bytes, long long timeout_ns, void *stream);

/* Bytes of device memory mtb_align_stack_host needs: the images, the
 * workspace and the shifts (0 if the sizes are invalid).  Host only. */
size_t mtb_host_workspace_bytes(int n_exposures, int w, int h, int levels);

/* Align a stack held in HOST memory (Sec. III-B: the exposures are copied to the
 * device once).  host_images: host [n][h][w][3] uint8 (pinned memory lets the
 * copy run asynchronously); host_shifts_out: host int32 [n][2].  Stacks of 8 MB
 * or more are copied in bands of whole 32-row tile rows of one exposure (about
 * 16 MB each) on a copy stream the library owns, one per device; the pyramid
 * pass over each band runs on `stream` as soon as the band has landed, after
 * work enqueued earlier on `stream`.  Smaller stacks are copied in one piece on
 * `stream`, by a copy kernel when host_images is page-locked and 16-byte
 * aligned (a copy engine idle for some milliseconds is slow to start), else by
 * cudaMemcpyAsync; page-locked host_shifts_out is written by SM stores.  The
 * alignment and the copy out are enqueued on `stream`, and the
 * call returns after synchronising it.  device_workspace: device, 256-byte
 * aligned, >= mtb_host_workspace_bytes(...) bytes, or NULL to allocate
 * stream-ordered.  Thread-safe; calls from several threads share the copy
 * stream, so their copies run one after another. */
int mtb_align_stack_host(const uint8_t *host_images, int n_exposures, int w, int h, int levels,
                         int noise_tol, int ref_idx, int32_t *host_shifts_out,
                         void *device_workspace, size_t device_workspace_bytes, void *stream);

/* ---- Batches: many stacks of any sizes in one persistent launch ----------
 * Sec. III-B aligns one stack's pairs with each exposure's pyramid built once;
 * a batch does that for many stacks together.  Every step of every stack runs
 * as work items of one persistent kernel (after one small clearing kernel),
 * queued in topological order with per-item completion counters, so the
 * latency-bound coarse-to-fine searches of some stacks overlap the
 * bandwidth-bound pyramid and bitmap work of others.  Results are exactly those
 * of mtb_align_stack_ex for each stack. */
typedef struct mtb_stack_desc {
    const uint8_t *images;      /* device [n][h][w][3] uint8, 16-byte aligned */
    int n_exposures, w, h, levels, noise_tol, ref_idx;  /* as for mtb_align_stack */
    int32_t *shifts_out;        /* device int32 [n][2] */
    uint32_t *level_errs_out;   /* device uint32 [n][levels][9] or NULL */
    int32_t *level_shifts_out;  /* device int32 [n][levels][2] or NULL */
} mtb_stack_desc_t;

typedef struct mtb_batch mtb_batch_t;

/* Device workspace a batch of these stacks needs (0 if a stack is invalid). */
size_t mtb_batch_workspace_bytes(const mtb_stack_desc_t *stacks, int count);

/* Plans a batch: checks every stack (MTB_ERR_INVALID_ARG on the first invalid
 * one), lays the stacks out in `workspace` (device, 256-byte aligned, >=
 * mtb_batch_workspace_bytes; NULL to let the batch cudaMalloc its own), uploads
 * the work tables and captures the launch in a CUDA graph.  Synchronous; the
 * descriptors are copied, the buffers they point to must stay valid while the
 * batch is used.  *out receives the batch. */
int mtb_batch_create(const mtb_stack_desc_t *stacks, int count, void *workspace, size_t workspace_bytes,
                     mtb_batch_t **out);

/* Enqueues one run of the batch on `stream` (aligns every stack from the
 * current contents of its image buffer). */
int mtb_batch_run(mtb_batch_t *batch, void *stream);

/* Autotuner: times `reps` runs of the batch for each candidate setting and
 * keeps the fastest, coordinate by coordinate:
 *   - runs of pyramid tiles per CTA: 1, 2, 4;
 *   - words per bitmap chunk: 512, 1024, 2048, 4096;
 *   - search chunks per level: 1, 2, 4;
 *   - the coarse-window budget: 0, 256 or 2048 units of 1024 word-candidates
 *     per pair.
 * The window budget trades the brute-force windows of the coarse levels
 * (Sec. III-B's search, counted for every candidate of the reachable window at
 * once) against one 9-candidate hop per level; results are the same either
 * way.  Synchronous.  No run of the batch may still be in flight on another
 * stream: the tables a run reads are rewritten.  If a timing fails, the best
 * setting found so far is rebuilt and the error returned. */
int mtb_batch_tune(mtb_batch_t *batch, int reps, void *stream);

/* The batch's settings:
 *   - values[0]: pyramid runs per CTA;
 *   - values[1]: words per bitmap chunk;
 *   - values[2]: search chunks per level (x CTAs / stacks);
 *   - values[3]: 1 if the launch is a CUDA graph;
 *   - values[4] (written if n_values >= 5): the coarse-window budget in units
 *     of 1024 word-candidates per pair.
 * n_values >= 4. */
int mtb_batch_config(const mtb_batch_t *batch, int *values, int n_values);

/* Sets the batch's settings in the layout of mtb_batch_config.  values[3] is
 * ignored.  Each other value must be one of the autotuner's candidates
 * (MTB_ERR_INVALID_ARG otherwise).  n_values >= 5.  Replans the batch and
 * recaptures its graph; on an error the previous settings stay.  As for
 * mtb_batch_tune, no run of the batch may be in flight. */
int mtb_batch_set_config(mtb_batch_t *batch, const int *values, int n_values);

/* Waits for `stream`, then returns MTB_OK or the first stack's non-zero status
 * word (MTB_ERR_TIMEOUT if a bounded device wait gave up). */
int mtb_batch_status(mtb_batch_t *batch, void *stream);

/* Frees the batch (and its workspace if it allocated it) once its runs are
 * complete.  NULL is ignored. */
void mtb_batch_destroy(mtb_batch_t *batch);

/* Size of the fixed device scratch array used by mtb_align_stack_noalloc:
 * 32 MiB, enough for a stack of five 3.7 MP exposures at 6 levels. */
#define MTB_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* mtb_align_stack_ex for callers that cannot allocate device memory when they
 * align (a per-frame loop with a deadline, a plug-in whose host owns all
 * allocations, a fixed memory budget).  The paper has no counterpart; this is a
 * property of the library.  Arguments and outputs as in mtb_align_stack_ex
 * (level_errs_out and level_shifts_out may be NULL); no cudaMalloc, cudaFree or
 * other allocating call is made.  The workspace is a fixed device array of
 * MTB_NOALLOC_SCRATCH_BYTES that each device holds from the first call on it
 * until the process exits.
 * - A stack whose mtb_workspace_bytes() exceeds MTB_NOALLOC_SCRATCH_BYTES is
 *   rejected with MTB_ERR_INVALID_ARG before anything is enqueued.
 * - The first call on a device looks the array's address up (cudaGetSymbolAddress)
 *   with that device current and keeps it for that device's context; a call
 *   that finds another context current (after cudaDeviceReset) looks it up
 *   again.  Make the first call, and the first call after a reset, before any
 *   stream capture.
 * - All calls on a device share the array.  Calls whose GPU work overlaps (other
 *   streams, other host threads) race and give wrong results: order them. */
int mtb_align_stack_noalloc(const uint8_t *images, int n_exposures, int w, int h, int levels,
                            int noise_tol, int ref_idx, int32_t *shifts_out,
                            uint32_t *level_errs_out, int32_t *level_shifts_out, void *stream);

/* ---- After the alignment: moving the exposures ----------------------------
 * The search's operator S (Sec. III-B moves the second image's maps by
 * (sx, sy), 0 outside the image) applied to the RGB exposures themselves:
 * out_i(x, y) = in_i(x - sx_i, y - sy_i), per channel.  Where the source lies
 * outside the image the pixel is 0 (MTB_FILL_ZERO) or the nearest edge pixel
 * (MTB_FILL_EDGE).  The paper stops at the shifts; this is the step after. */
#define MTB_FILL_ZERO 0
#define MTB_FILL_EDGE 1

/* images: device [n][h][w][3] uint8, 16-byte aligned; shifts: device int32
 * [n][2] (e.g. the shifts_out of an alignment on the same stream); out: device
 * [n][h][w][3] uint8, 16-byte aligned, not overlapping images.  Requires
 * 1 <= n <= MTB_MAX_EXPOSURES, 1 <= w, h <= MTB_MAX_DIM, fill 0 or 1; any int32
 * shift is valid (beyond the image the whole exposure is fill).  Enqueues one
 * kernel on `stream`. */
int mtb_apply_shifts(const uint8_t *images, int n_exposures, int w, int h, const int32_t *shifts, int fill,
                     uint8_t *out, void *stream);

/* ---- Rotation test by quadrants --------------------------------------------
 * Sec. II recalls Ward's test for a rotation between exposures: split each
 * exposure into four quadrants and align every quadrant stack on its own; a
 * pure translation moves the four alike.  Quadrant q = 2*qy + qx (top-left,
 * top-right, bottom-left, bottom-right) is the floor(w/2) x floor(h/2) block at
 * (qx*floor(w/2), qy*floor(h/2)); each quadrant stack is aligned directly to
 * ref_idx exactly as mtb_align_stack would align it. */

/* Device workspace of mtb_align_quadrants (0 if the sizes are invalid). */
size_t mtb_quadrant_workspace_bytes(int n_exposures, int w, int h, int levels);

/* images: device [n][h][w][3] uint8 (16-byte aligned); `levels` must be valid
 * for the floor(w/2) x floor(h/2) quadrants (other arguments as for
 * mtb_align_stack).  quad_shifts_out: device int32 [n][4][2]; flags_out: device
 * int32 [n] or NULL -- 1 where the four quadrant shifts of an exposure spread by
 * more than rot_tol (>= 0) pixels in x or in y, else 0.  workspace: device,
 * 256-byte aligned, >= mtb_quadrant_workspace_bytes(...), or NULL to allocate
 * stream-ordered. */
int mtb_align_quadrants(const uint8_t *images, int n_exposures, int w, int h, int levels, int noise_tol,
                        int ref_idx, int rot_tol, int32_t *quad_shifts_out, int32_t *flags_out,
                        void *workspace, size_t workspace_bytes, void *stream);

/* ---- Serving: continuous admission of jobs under a device-memory budget ----
 * Sec. III-B copies each exposure of a stack to the GPU once and aligns it
 * there; a server does that for a stream of independent stacks held in host
 * memory.  It owns one device arena of budget_bytes, `slots` compute streams
 * and `copy_streams` copy streams, and one worker thread.  A submitted job
 * waits in arrival order until a slot is free and the arena can hold the job's
 * images, workspace and shifts (mtb_job_bytes); it is then admitted -- also
 * while other jobs are still on the GPU -- and its copy in (split over the copy
 * streams, in admission order), alignment and copy out are enqueued.  Jobs on
 * different slots overlap on the GPU; each job's pyramids and bitmaps stay in
 * the arena until its shifts are out, and its memory then returns to the arena.
 * Every job's shifts are exactly those of mtb_align_stack_ex on the same
 * stack, whatever else runs beside it. */
#define MTB_SERVER_MAX_SLOTS 64
#define MTB_SERVER_MAX_COPY_STREAMS 8
#define MTB_SERVER_STATS 9

typedef struct mtb_server_config {
    size_t budget_bytes;  /* device arena, >= 1 MiB (allocated by mtb_server_create) */
    int slots;            /* jobs on the GPU at most, 1..MTB_SERVER_MAX_SLOTS */
    int copy_streams;     /* streams each job's copy in is split over, 1..MTB_SERVER_MAX_COPY_STREAMS */
    int max_pending;      /* jobs waiting for admission at most (0 = no limit) */
} mtb_server_config_t;

typedef struct mtb_job {
    const uint8_t *host_images;  /* host [n][h][w][3] uint8, valid until the job completes.
                                    Page-locked (pinned) memory, 16-byte aligned, is read
                                    by a copy kernel over the host link; other memory is
                                    copied by cudaMemcpyAsync */
    int n_exposures, w, h, levels, noise_tol, ref_idx;  /* as for mtb_align_stack */
    int32_t *host_shifts_out;    /* host int32 [n][2], written when the job completes */
} mtb_job_t;

typedef struct mtb_server mtb_server_t;

/* Device bytes a job is charged against the budget: its images, workspace and
 * shifts (= mtb_host_workspace_bytes); 0 if the job is invalid.  Host only. */
size_t mtb_job_bytes(const mtb_job_t *job);

/* Checks the configuration (MTB_ERR_INVALID_ARG before any CUDA call), then
 * allocates the arena on the current device (MTB_ERR_OOM if it cannot), the
 * streams and a pinned result area per slot, and starts the worker.  After
 * this call the server allocates nothing on the host per job beyond the job's
 * record in mtb_server_submit (MTB_ERR_OOM if that fails). */
int mtb_server_create(const mtb_server_config_t *config, mtb_server_t **out);

/* Queues a job; *job_id receives its id.  MTB_ERR_INVALID_ARG for an invalid
 * job; MTB_ERR_BUSY if the job is larger than the whole budget or max_pending
 * jobs are already waiting (back-pressure: nothing is queued). */
int mtb_server_submit(mtb_server_t *server, const mtb_job_t *job, uint64_t *job_id);

/* 1 while the job waits or runs, else its final status (MTB_OK, or an
 * MTB_ERR_* code such as MTB_ERR_TIMEOUT from the device-side waits);
 * MTB_ERR_INVALID_ARG for an unknown id.  Does not block. */
int mtb_server_poll(mtb_server_t *server, uint64_t job_id);

/* Blocks until the job completes, returns its final status and forgets the id.
 * times_ms (NULL or double[2]) receives the latency from submission to the
 * shifts being in host_shifts_out, and the part of it spent waiting for
 * admission. */
int mtb_server_wait(mtb_server_t *server, uint64_t job_id, double *times_ms);

/* As mtb_server_wait, with the latency split into its phases (host clock,
 * milliseconds): times_ms (NULL or double[5]) receives [0] submission to the
 * shifts being in host_shifts_out, [1] waiting for admission, [2] enqueueing
 * the job's copies and kernels, [3] from then to the completion callback
 * (the copy in, the alignment, the copy out and the callback's dispatch), [4]
 * the callback itself.  No counterpart in the paper (serving is this
 * library's addition). */
int mtb_server_wait_phases(mtb_server_t *server, uint64_t job_id, double *times_ms);

/* Holds (paused != 0) or resumes admission; queued jobs stay queued. */
int mtb_server_pause(mtb_server_t *server, int paused);

/* values[0..8]: jobs admitted, completed, refused, failed; jobs waiting now,
 * running now; arena bytes in use now; peak arena bytes in use; peak jobs
 * running at once.  n_values >= MTB_SERVER_STATS. */
int mtb_server_stats(mtb_server_t *server, uint64_t *values, int n_values);

/* Resumes admission, waits until every submitted job has completed, then
 * stops the worker and frees everything.  NULL is ignored. */
void mtb_server_destroy(mtb_server_t *server);

#ifdef __cplusplus
}
#endif

#endif /* MTB_H_ */
