// mtb_engine.cu -- whole alignments in one persistent launch.
//
// The engine runs every step of Sec. III-A / III-B -- gray pyramid with
// histograms and medians, threshold and exclusion bitmaps, and the
// coarse-to-fine search -- for one stack or for a batch of stacks of any sizes,
// as work items of one persistent kernel.  Items are queued in topological
// order, phase by phase over all stacks:
//   PYR     a run of 32x256 pyramid tiles of one exposure (levels 0..5, their
//           histograms; the run that finishes an exposure computes its medians)
//   BIT_HI  bitmap chunks of levels 1..5 of an exposure, and the deep levels
//   BIT_L0* level-0 bitmap chunks, when level 0 is itself a window level
//   WIN     window items of the coarsest levels (see mtb_search_dev.cuh)
//   RES     resolve items: the chain through the window tables
//   BIT_L0  level-0 bitmap chunks (after the window work, so that the
//           latency-bound coarse search overlaps this bandwidth-bound pass)
//   SHIFT   search chunks, level by level from coarse to fine
//   FINAL   the shifts and per-level outputs of a stack
// An item waits (one thread, bounded) on the completion counters of the items
// it reads, which always come earlier in the queue; CTAs take items in queue
// order, so every wait ends.  Data produced inside the launch is read with
// weak or L2-only loads after the acquire of its counter, never through the
// non-coherent path.
#include <new>
#include <vector>

#include "mtb_bitmaps_dev.cuh"
#include "mtb_pyramid_dev.cuh"
#include "mtb_search_dev.cuh"

namespace mtb {

enum EnginePhase : int {
    kPhPyr = 0,
    kPhBitHi,
    kPhBitL0First,
    kPhWin,
    kPhRes,
    kPhBitL0,
    kPhShift,                            // + (MTB_MAX_LEVELS - 1 - l) for level l
    kPhFinal = kPhShift + MTB_MAX_LEVELS,
    kPhases
};

struct StackDesc {
    mtb_layout_t L;
    const uint8_t *images;
    uint8_t *ws;
    int tol;
    int aligned;          // width is a multiple of 16
    int tiles_x, tiles_per_exp;
    int pyr_chunk;        // tiles per PYR item
    int pyr_items;        // PYR items per exposure
    int bit_hi_items;     // BIT_HI items per exposure (levels 1..5, plus 1 for the deep levels)
    int bit_l0_items;     // level-0 bitmap chunks per exposure
    int bit_chunk_words;  // words per bitmap chunk
    int l0_first;         // level 0 is a window level
    SearchPlan sp;
    int count[kPhases];   // items of this stack in each phase
};

struct EngineArgs {
    StackDesc single;          // the stack, when the launch has one
    const StackDesc *stacks;   // device table, when it has several
    const int *stack_first;    // [kPhases][n_stacks + 1] first item of each stack within a phase
    int n_stacks;
    int phase_first[kPhases + 1];
    int total_items;
    int32_t *queue;            // work-queue head
};

namespace {

constexpr int kEngineThreads = 256;
static_assert(kEngineThreads == kPyrThreads && kEngineThreads == kBitThreads && kEngineThreads == kSearchThreads,
              "items share one CTA shape");

struct EngineShared {
    PyrShared pyr;
    SearchShared search;
    uint32_t hist[256];
    mtb_layout_t L;  // the layout of the stack a pyramid item works on
    int med;
    int stack, phase, local, ok;
};

// Exposure of the j-th group of PYR items: the reference first, then the
// others in order, so that the first pair's search can start early.
__device__ __forceinline__ int pyr_exposure(const StackDesc &d, int j) {
    return j == 0 ? d.sp.ref : (j <= d.sp.ref ? j - 1 : j);
}

static_assert(sizeof(mtb_layout_t) % 4 == 0, "the layout is copied to shared memory as 32-bit words");

__device__ __noinline__ void pyr_item(const StackDesc &d, int k, EngineShared &sm) {
    // the stack's layout in shared memory: the tile functions read its fields
    // for every tile and level
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&d.L);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sm.L);
        for (int v = threadIdx.x; v < (int)(sizeof(mtb_layout_t) / 4); v += kEngineThreads) dst[v] = src[v];
        __syncthreads();
    }
    const mtb_layout_t &L = sm.L;
    const int e = pyr_exposure(d, k / d.pyr_items);
    const int t0 = (k % d.pyr_items) * d.pyr_chunk;
    const int t1 = min(d.tiles_per_exp, t0 + d.pyr_chunk);
    const int K = L.tile_levels - 1;
    const int tiles_x = d.tiles_x, aligned = d.aligned;
    const uint8_t *images = d.images;
    uint8_t *ws = d.ws;
    int ty = t0 / tiles_x, tx = t0 - ty * tiles_x;
    if (aligned) {
        // levels 0..2 from registers, one barrier, levels 3..5 by the half of
        // the warps that alternates with the tile (the stage kernel's path
        // without its prefetch: the engine runs at 4 CTAs per SM)
        uint8_t *ebase = ws + (size_t)e * L.gray_exposure_stride;
        for (int t = t0; t < t1; ++t) {
            const int y0 = ty * kTileRows, x0 = tx * kTileCols;
            const int rows = min(kTileRows, L.h - y0), cols = min(kTileCols, L.w - x0);
            if (++tx == tiles_x) {
                tx = 0;
                ++ty;
            }
            const bool full = rows == kTileRows && cols == kTileCols;
            uint8_t *lv2 = sm.pyr.lv + ((t - t0) & 1) * kLv2Bytes;
            TileRgb rgb;
            tile_load_rgb(images, L, e, y0, x0, rows, cols, rgb);
            uint4 v[2];
            if (full) tile_level0<true>(rgb, L, ebase, y0, x0, rows, cols, sm.pyr, v);
            else tile_level0<false>(rgb, L, ebase, y0, x0, rows, cols, sm.pyr, v);
            if (K >= 1) {
                if (full) tile_levels12_pair<true>(v, L, ebase, y0, x0, K, sm.pyr, lv2);
                else tile_levels12_pair<false>(v, L, ebase, y0, x0, K, sm.pyr, lv2);
            }
            __syncthreads();
            const int a = (threadIdx.x >> 5) - (((t - t0) & 1) ? 4 : 0);
            if (K >= 3 && a >= 0 && a < 4) {
                if (full) tile_tail<true>(L, ebase, y0, x0, K, sm.pyr, lv2, a);
                else tile_tail<false>(L, ebase, y0, x0, K, sm.pyr, lv2, a);
            }
        }
    } else {
        for (int t = t0; t < t1; ++t) {
            const int y0 = ty * kTileRows, x0 = tx * kTileCols;
            const int rows = min(kTileRows, L.h - y0), cols = min(kTileCols, L.w - x0);
            if (++tx == tiles_x) {
                tx = 0;
                ++ty;
            }
            tile_level0_general(images, L, ws, e, y0, x0, rows, cols, sm.pyr);
            __syncthreads();
            tile_store_level0(L, ws, e, y0, x0, rows, cols, sm.pyr);
            if (K >= 1) tile_levels12(L, ws, e, y0, x0, K, sm.pyr);
            __syncthreads();
            if (K >= 3) tile_block_tail(L, ws, e, y0, x0, K, sm.pyr);
        }
    }
    flush_exposure(L, ws, e, t1 - t0, d.tiles_per_exp, K, sm.pyr);
}

// Waits (thread 0) for exposure e's pyramid pass; false if the wait gave up.
__device__ bool wait_pyramid(const StackDesc &d, int e, EngineShared &sm) {
    if (threadIdx.x == 0)
        sm.ok = wait_at_least(Ctr::pyr_ready(d.ws, d.L, e), 1, status_word(d.ws, d.L), d.sp.timeout_ns);
    __syncthreads();
    return sm.ok;
}

__device__ __noinline__ void bit_hi_item(const StackDesc &d, int k, EngineShared &sm) {
    const mtb_layout_t &L = d.L;
    const int je = k / d.bit_hi_items;
    const int e = pyr_exposure(d, je);
    const int j = k - je * d.bit_hi_items;
    if (!wait_pyramid(d, e, sm)) return;
    if (L.levels > L.tile_levels && j == d.bit_hi_items - 1) {
        deep_levels(L, d.ws, d.tol, e, sm.hist, &sm.med);
        return;
    }
    int l, c;
    bitmap_chunk_of(L, j + bitmap_chunks(L, 0, d.bit_chunk_words), d.bit_chunk_words, &l, &c);  // past level 0
    bitmap_chunk(L, d.ws, d.tol, e, l, c, d.bit_chunk_words, &sm.med);
}

__device__ __noinline__ void bit_l0_item(const StackDesc &d, int k, EngineShared &sm) {
    const int j = k / d.bit_l0_items;
    const int e = pyr_exposure(d, j);
    if (!wait_pyramid(d, e, sm)) return;
    bitmap_chunk(d.L, d.ws, d.tol, e, 0, k - j * d.bit_l0_items, d.bit_chunk_words, &sm.med);
}

// Search items as separate (not inlined) functions: each gets its own register
// allocation instead of the union of all item types.
__device__ __noinline__ void win_item(const StackDesc &d, int k, SearchShared &sm) {
    window_item<true>(d.L, d.ws, d.sp, k, sm);
}
__device__ __noinline__ void res_item(const StackDesc &d, int k, SearchShared &sm) {
    resolve_item(d.L, d.ws, d.sp, k, sm);
}
__device__ __noinline__ void sh_item(const StackDesc &d, int p, int l, int c, SearchShared &sm) {
    shift_item<true>(d.L, d.ws, d.sp, p, l, c, sm);
}
__device__ __noinline__ void fin_item(const StackDesc &d, SearchShared &sm) { final_item(d.L, d.ws, d.sp, sm); }

__device__ void run_item(const StackDesc &d, int phase, int k, EngineShared &sm) {
    const SearchPlan &P = d.sp;
    if (phase == kPhPyr) {
        pyr_item(d, k, sm);
    } else if (phase == kPhBitHi) {
        bit_hi_item(d, k, sm);
    } else if (phase == kPhBitL0First || phase == kPhBitL0) {
        bit_l0_item(d, k, sm);
    } else if (phase == kPhWin) {
        win_item(d, k, sm.search);
    } else if (phase == kPhRes) {
        res_item(d, k, sm.search);
    } else if (phase == kPhFinal) {
        fin_item(d, sm.search);
    } else {
        const int l = MTB_MAX_LEVELS - 1 - (phase - kPhShift);
        sh_item(d, k / P.chunks[l], l, k % P.chunks[l], sm.search);
    }
}

template <bool kBatch>
__global__ void __launch_bounds__(kEngineThreads, 4) k_engine(const EngineArgs A) {
    __shared__ EngineShared sm;
    const int tid = threadIdx.x;
    for (int v = tid; v < 2 * kPyrWarps * 256; v += kEngineThreads) (&sm.pyr.h01[0][0][0])[v] = 0;
    for (int v = tid; v < (kTileLog2 - 1) * 256; v += kEngineThreads) (&sm.pyr.hs[0][0])[v] = 0;
    pdl_trigger();
    pdl_wait();  // counters and histograms were cleared by the previous launch
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            const int it = atomicAdd(A.queue, 1);
            int ph = -1, s = 0, k = 0;
            if (it < A.total_items) {
                ph = 0;
                while (it >= A.phase_first[ph + 1]) ++ph;
                k = it - A.phase_first[ph];
                if (kBatch) {  // stack of the item: binary search in this phase's prefix table
                    const int *f = A.stack_first + ph * (A.n_stacks + 1);
                    int lo = 0, hi = A.n_stacks - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (__ldg(f + mid) <= k) lo = mid;
                        else hi = mid - 1;
                    }
                    s = lo;
                    k -= __ldg(f + s);
                }
            }
            sm.phase = ph;
            sm.stack = s;
            sm.local = k;
        }
        __syncthreads();
        const int ph = sm.phase, s = sm.stack, k = sm.local;
        __syncthreads();
        if (ph < 0) break;
        run_item(kBatch ? A.stacks[s] : A.single, ph, k, sm);
        __syncthreads();
    }
}

// Clears, for every stack, the histograms, counters, error counters, window
// tables and status word, and the reference's base and shift rows; then the
// engine's queue head.  One CTA per stack.
template <bool kBatch>
__global__ void k_engine_clear(const EngineArgs A) {
    pdl_trigger();  // k_engine waits (griddepcontrol.wait) before it touches anything cleared here
    const StackDesc &d = kBatch ? A.stacks[blockIdx.x] : A.single;
    const mtb_layout_t &L = d.L;
    uint8_t *ws = d.ws;
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.hist_offset);
    const int hist_words = (int)((L.counter_offset - L.hist_offset) / 4) + pyramid_counter_words(L) +
                           search_counter_words(L);  // histograms and the whole counter area
    for (int k = threadIdx.x; k < hist_words; k += blockDim.x) hist[k] = 0;
    uint32_t *errs = reinterpret_cast<uint32_t *>(ws + L.errs_offset);
    for (int k = threadIdx.x; k < L.n * L.levels * 9; k += blockDim.x) errs[k] = 0;
    uint32_t *tab = reinterpret_cast<uint32_t *>(ws + L.table_offset);
    for (int k = threadIdx.x; k < L.n * kTableWords; k += blockDim.x) tab[k] = 0;
    for (int k = threadIdx.x; k < L.levels * 2; k += blockDim.x) {
        Planes::base(ws, L, d.sp.ref, 0)[k] = 0;
        Planes::shift(ws, L, d.sp.ref, 0)[k] = 0;
    }
    if (threadIdx.x == 0) *status_word(ws, L) = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.queue = 0;
}

int g_engine_blocks_per_sm[2] = {0, 0};

}  // namespace

// CTAs an engine launch uses: every SM at the engine's occupancy.
long long engine_capacity(bool batch) {
    int &nb = g_engine_blocks_per_sm[batch ? 1 : 0];
    if (nb == 0) {
        int v = 0;
        const cudaError_t err =
            batch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_engine<true>, kEngineThreads, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_engine<false>, kEngineThreads, 0);
        if (err != cudaSuccess) return -1;
        nb = v > 0 ? v : 1;
    }
    return (long long)device_sm_count() * nb;
}

// The engine's tile shapes; the batch autotuner searches over them.
struct EngineTuning {
    int pyr_runs_per_cta;  // PYR items per CTA of the launch (tiles per item follow from it)
    int bit_chunk_words;   // words per bitmap chunk
    int search_waves;      // search chunks per larger level: about search_waves * CTAs / stacks
    int window_kwords;     // coarse-window budget, 1024 word-candidates per pair (0: no windows)
};
constexpr EngineTuning kDefaultTuning = {1, 1024, 1, (int)(kBruteBudget >> 10)};
// The autotuner's candidates, which mtb_batch_set_config also accepts.  Many
// stacks in flight favour fewer coarse windows than one stack alone: their
// 9-candidate hops overlap each other's work.
constexpr int kRunsCand[] = {1, 2, 4};
constexpr int kWordsCand[] = {512, 1024, 2048, 4096};
constexpr int kWavesCand[] = {1, 2, 4};
constexpr int kWindowCand[] = {0, 256, 2048};
template <int N>
bool one_of(int v, const int (&c)[N]) {
    for (int k = 0; k < N; ++k)
        if (v == c[k]) return true;
    return false;
}

// Fills the item plan of one stack.  total_tiles: pyramid tiles of the whole
// launch (all stacks), n_stacks: stacks in the launch.
int plan_stack(const mtb_layout_t &L, const uint8_t *images, uint8_t *ws, int tol, int ref, int32_t *shifts_out,
               uint32_t *level_errs_out, int32_t *level_shifts_out, long long cap, long long total_tiles,
               int n_stacks, const EngineTuning &tun, unsigned long long timeout_ns, StackDesc *d) {
    *d = StackDesc{};
    d->L = L;
    d->images = images;
    d->ws = ws;
    d->tol = tol;
    d->aligned = (L.w % 16) == 0;
    d->tiles_x = (L.w + kTileCols - 1) / kTileCols;
    d->tiles_per_exp = d->tiles_x * ((L.h + kTileRows - 1) / kTileRows);
    // each run of tiles ends with a histogram flush: about pyr_runs_per_cta runs per CTA
    const long long runs = (cap > 0 ? cap : 1) * (tun.pyr_runs_per_cta > 0 ? tun.pyr_runs_per_cta : 1);
    long long chunk = (total_tiles + runs - 1) / runs;
    chunk = chunk < 1 ? 1 : (chunk > 64 ? 64 : chunk);
    d->pyr_chunk = (int)chunk;
    d->pyr_items = (d->tiles_per_exp + d->pyr_chunk - 1) / d->pyr_chunk;
    d->bit_chunk_words = tun.bit_chunk_words;
    d->bit_hi_items = 0;
    for (int l = 1; l < L.tile_levels; ++l) d->bit_hi_items += bitmap_chunks(L, l, d->bit_chunk_words);
    if (L.levels > L.tile_levels) d->bit_hi_items += 1;
    d->bit_l0_items = bitmap_chunks(L, 0, d->bit_chunk_words);
    long long search_cap = cap * (tun.search_waves > 0 ? tun.search_waves : 1) / (n_stacks > 0 ? n_stacks : 1);
    if (search_cap < 1) search_cap = 1;
    plan_search(L, ref, search_cap, shifts_out, level_errs_out, level_shifts_out, timeout_ns, -1, &d->sp, 0,
                (long long)tun.window_kwords << 10);
    if (d->sp.total_items < 0) return MTB_ERR_INVALID_ARG;
    d->sp.bit_chunk_words = d->bit_chunk_words;
    const SearchPlan &P = d->sp;
    d->l0_first = P.lc == 0;
    d->count[kPhPyr] = L.n * d->pyr_items;
    d->count[kPhBitHi] = L.n * d->bit_hi_items;
    d->count[kPhBitL0First] = d->l0_first ? L.n * d->bit_l0_items : 0;
    d->count[kPhWin] = P.pairs * P.window_items;
    d->count[kPhRes] = P.pairs;
    d->count[kPhBitL0] = d->l0_first ? 0 : L.n * d->bit_l0_items;
    for (int l = 0; l < MTB_MAX_LEVELS; ++l)
        d->count[kPhShift + MTB_MAX_LEVELS - 1 - l] = l < P.lc ? P.pairs * P.chunks[l] : 0;
    d->count[kPhFinal] = 1;
    return MTB_OK;
}

long long stack_tiles(const mtb_layout_t &L) {
    return (long long)((L.w + kTileCols - 1) / kTileCols) * ((L.h + kTileRows - 1) / kTileRows) * L.n;
}

// One stack through the engine: clear, then the persistent launch.
cudaError_t launch_engine_single(const mtb_layout_t &L, const uint8_t *images, uint8_t *ws, int tol, int ref,
                                 int32_t *shifts_out, uint32_t *level_errs_out, int32_t *level_shifts_out,
                                 cudaStream_t s) {
    const long long cap = engine_capacity(false);
    if (cap <= 0) return cudaErrorInvalidValue;
    EngineArgs A = {};
    if (plan_stack(L, images, ws, tol, ref, shifts_out, level_errs_out, level_shifts_out, cap, stack_tiles(L), 1,
                   kDefaultTuning, kSearchTimeoutNs, &A.single) != MTB_OK)
        return cudaErrorInvalidValue;
    long long first = 0;
    for (int ph = 0; ph < kPhases; ++ph) {
        A.phase_first[ph] = (int)first;
        first += A.single.count[ph];
    }
    if (first > 0x7fffffffLL) return cudaErrorInvalidValue;
    A.phase_first[kPhases] = (int)first;
    A.total_items = (int)first;
    A.n_stacks = 1;
    A.queue = Ctr::queue_host(ws, L);
    cudaError_t err = launch_k(k_engine_clear<false>, dim3(1), dim3(1024), s, false, A);
    if (err != cudaSuccess) return err;
    const int grid = (int)(A.total_items < cap ? A.total_items : cap);
    return launch_k(k_engine<false>, dim3(grid), dim3(kEngineThreads), s, true, A);
}

}  // namespace mtb

// ---------------------------------------------------------------------------
// Batches (mtb.h): many stacks of any sizes in one persistent launch, captured
// in a CUDA graph.
using namespace mtb;

struct mtb_batch {
    int count = 0;
    std::vector<mtb_stack_desc_t> user;
    std::vector<mtb_layout_t> layouts;
    std::vector<size_t> ws_offset;
    uint8_t *workspace = nullptr;
    size_t workspace_bytes = 0;
    bool own_workspace = false;
    uint8_t *tables = nullptr;  // device: StackDesc[count], stack_first[kPhases][count + 1], queue
    EngineArgs args = {};
    EngineTuning tuning = kDefaultTuning;
    long long cap = 0;
    cudaGraphExec_t graph = nullptr;
};

namespace {

int stack_layout(const mtb_stack_desc_t &sd, mtb_layout_t *L) {
    int rc = check_stack_args(sd.n_exposures, sd.w, sd.h, sd.levels, sd.noise_tol, sd.ref_idx);
    if (rc != MTB_OK) return rc;
    if (!sd.images || !sd.shifts_out || (reinterpret_cast<uintptr_t>(sd.images) & 15u)) return MTB_ERR_INVALID_ARG;
    return compute_layout(sd.n_exposures, sd.w, sd.h, sd.levels, L);
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Plans all stacks with b->tuning, uploads the tables and captures the graph.
// A plan that fails (MTB_ERR_INVALID_ARG) leaves the batch as it was; a failed
// upload leaves it refusing to run (MTB_ERR_CUDA from batch_launch).
int batch_build_tables(mtb_batch *b) {
    const int n = b->count;
    long long total_tiles = 0;
    for (int s = 0; s < n; ++s) total_tiles += stack_tiles(b->layouts[s]);
    std::vector<StackDesc> descs(n);
    for (int s = 0; s < n; ++s) {
        const mtb_stack_desc_t &u = b->user[s];
        if (plan_stack(b->layouts[s], u.images, b->workspace + b->ws_offset[s], u.noise_tol, u.ref_idx, u.shifts_out,
                       u.level_errs_out, u.level_shifts_out, b->cap, total_tiles, n, b->tuning, kSearchTimeoutNs,
                       &descs[s]) != MTB_OK)
            return MTB_ERR_INVALID_ARG;
    }
    // phase-major queue: phase_first over all stacks, stack_first within each phase
    std::vector<int> stack_first((size_t)kPhases * (n + 1));
    long long first = 0;
    EngineArgs A = b->args;
    for (int ph = 0; ph < kPhases; ++ph) {
        A.phase_first[ph] = (int)first;
        long long within = 0;
        for (int s = 0; s < n; ++s) {
            stack_first[(size_t)ph * (n + 1) + s] = (int)within;
            within += descs[s].count[ph];
        }
        stack_first[(size_t)ph * (n + 1) + n] = (int)within;
        first += within;
        if (first > 0x7fffffffLL) return MTB_ERR_INVALID_ARG;
    }
    A.phase_first[kPhases] = (int)first;
    A.total_items = (int)first;
    A.n_stacks = n;
    const size_t desc_bytes = align256(sizeof(StackDesc) * n);
    const size_t first_bytes = align256(sizeof(int) * stack_first.size());
    // the plan holds; from here on the batch's old graph and tables go
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (cudaMemcpy(b->tables, descs.data(), sizeof(StackDesc) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tables + desc_bytes, stack_first.data(), sizeof(int) * stack_first.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        b->args.total_items = 0;
        return MTB_ERR_CUDA;
    }
    A.stacks = reinterpret_cast<const StackDesc *>(b->tables);
    A.stack_first = reinterpret_cast<const int *>(b->tables + desc_bytes);
    A.queue = reinterpret_cast<int32_t *>(b->tables + desc_bytes + first_bytes);
    b->args = A;
    // capture clear + engine in a graph (run without one if capture is refused)
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MTB_ERR_CUDA;
    const int grid = (int)(A.total_items < b->cap ? A.total_items : b->cap);
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        ok = launch_k(k_engine_clear<true>, dim3(n), dim3(1024), cs, false, A) == cudaSuccess &&
             launch_k(k_engine<true>, dim3(grid), dim3(kEngineThreads), cs, true, A) == cudaSuccess;
        ok = (cudaStreamEndCapture(cs, &g) == cudaSuccess) && ok && g != nullptr;
    }
    if (ok && cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) b->graph = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    cudaStreamDestroy(cs);
    return MTB_OK;
}

// batch_build_tables with a failed host allocation reported as MTB_ERR_OOM (no
// C++ exception leaves the library).  The host vectors are all allocated before
// the graph capture begins, so no capture is left open.
int batch_build(mtb_batch *b) {
    try {
        return batch_build_tables(b);
    } catch (...) {
        return MTB_ERR_OOM;
    }
}

int batch_launch(mtb_batch *b, cudaStream_t s) {
    if (b->graph) return cudaGraphLaunch(b->graph, s) == cudaSuccess ? MTB_OK : MTB_ERR_CUDA;
    const EngineArgs &A = b->args;
    if (A.total_items <= 0) return MTB_ERR_CUDA;  // the last table upload failed
    const int grid = (int)(A.total_items < b->cap ? A.total_items : b->cap);
    if (launch_k(k_engine_clear<true>, dim3(b->count), dim3(1024), s, false, A) != cudaSuccess) return MTB_ERR_CUDA;
    if (launch_k(k_engine<true>, dim3(grid), dim3(kEngineThreads), s, true, A) != cudaSuccess) return MTB_ERR_CUDA;
    return MTB_OK;
}

}  // namespace

extern "C" {

size_t mtb_batch_workspace_bytes(const mtb_stack_desc_t *stacks, int count) {
    if (!stacks || count < 1) return 0;
    size_t total = 0;
    for (int s = 0; s < count; ++s) {
        mtb_layout_t L;
        if (stack_layout(stacks[s], &L) != MTB_OK) return 0;
        total += align256(L.total_bytes);
    }
    return total;
}

int mtb_batch_create(const mtb_stack_desc_t *stacks, int count, void *workspace, size_t workspace_bytes,
                     mtb_batch_t **out) {
    if (!out || !stacks || count < 1 || count > (1 << 20)) return MTB_ERR_INVALID_ARG;
    *out = nullptr;
    mtb_batch *b = new (std::nothrow) mtb_batch();
    if (!b) return MTB_ERR_OOM;
    b->count = count;
    try {
        b->user.assign(stacks, stacks + count);
        b->layouts.resize(count);
        b->ws_offset.resize(count);
    } catch (...) {
        delete b;
        return MTB_ERR_OOM;
    }
    size_t total = 0;
    int rc = MTB_OK;
    for (int s = 0; s < count && rc == MTB_OK; ++s) {
        rc = stack_layout(stacks[s], &b->layouts[s]);
        b->ws_offset[s] = total;
        total += align256(b->layouts[s].total_bytes);
    }
    if (rc == MTB_OK) {
        if (workspace) {
            if (workspace_bytes < total || (reinterpret_cast<uintptr_t>(workspace) & 255u)) rc = MTB_ERR_INVALID_ARG;
            b->workspace = static_cast<uint8_t *>(workspace);
        } else if (cudaMalloc(&b->workspace, total) != cudaSuccess) {
            cudaGetLastError();
            rc = MTB_ERR_OOM;
        } else {
            b->own_workspace = true;
        }
        b->workspace_bytes = total;
    }
    if (rc == MTB_OK) {
        const size_t tbytes = align256(sizeof(StackDesc) * count) + align256(sizeof(int) * kPhases * (count + 1)) + 256;
        if (cudaMalloc(&b->tables, tbytes) != cudaSuccess) {
            cudaGetLastError();
            rc = MTB_ERR_OOM;
        }
    }
    if (rc == MTB_OK) {
        b->cap = engine_capacity(true);
        if (b->cap <= 0) rc = MTB_ERR_CUDA;
    }
    if (rc == MTB_OK) rc = batch_build(b);
    if (rc != MTB_OK) {
        mtb_batch_destroy(b);
        return rc;
    }
    *out = b;
    return MTB_OK;
}

int mtb_batch_run(mtb_batch_t *b, void *stream) {
    if (!b) return MTB_ERR_INVALID_ARG;
    return batch_launch(b, static_cast<cudaStream_t>(stream));
}

int mtb_batch_tune(mtb_batch_t *b, int reps, void *stream) {
    if (!b || reps < 1 || reps > 100) return MTB_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return MTB_ERR_CUDA;
    }
    auto time_config = [&](float *ms) -> int {
        int rc = batch_build(b);
        if (rc != MTB_OK) return rc;
        if ((rc = batch_launch(b, s)) != MTB_OK) return rc;  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && rc == MTB_OK; ++r) rc = batch_launch(b, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return MTB_ERR_CUDA;
        cudaEventElapsedTime(ms, e0, e1);
        return rc;
    };
    // coordinate descent over the four knobs
    EngineTuning best = b->tuning;
    float best_ms = 0;
    int rc = time_config(&best_ms);
    for (int knob = 0; knob < 4 && rc == MTB_OK; ++knob) {
        const int *cand = knob == 0 ? kRunsCand : knob == 1 ? kWordsCand : knob == 2 ? kWavesCand : kWindowCand;
        const int nc = knob == 1 ? 4 : 3;
        for (int c = 0; c < nc && rc == MTB_OK; ++c) {
            EngineTuning t = best;
            int &field = knob == 0   ? t.pyr_runs_per_cta
                         : knob == 1 ? t.bit_chunk_words
                         : knob == 2 ? t.search_waves
                                     : t.window_kwords;
            if (field == cand[c]) continue;
            field = cand[c];
            b->tuning = t;
            float ms = 0;
            rc = time_config(&ms);
            if (rc == MTB_OK && ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    }
    // the best setting found (the starting one if the first timing failed) is
    // rebuilt even after a failure, so the batch stays runnable as before
    b->tuning = best;
    const int rc_build = batch_build(b);
    if (rc == MTB_OK) rc = rc_build;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int mtb_batch_config(const mtb_batch_t *b, int *values, int n_values) {
    if (!b || !values || n_values < 4) return MTB_ERR_INVALID_ARG;
    values[0] = b->tuning.pyr_runs_per_cta;
    values[1] = b->tuning.bit_chunk_words;
    values[2] = b->tuning.search_waves;
    values[3] = b->graph != nullptr;
    if (n_values >= 5) values[4] = b->tuning.window_kwords;
    return MTB_OK;
}

int mtb_batch_set_config(mtb_batch_t *b, const int *values, int n_values) {
    if (!b || !values || n_values < 5) return MTB_ERR_INVALID_ARG;
    if (!one_of(values[0], kRunsCand) || !one_of(values[1], kWordsCand) || !one_of(values[2], kWavesCand) ||
        !one_of(values[4], kWindowCand))
        return MTB_ERR_INVALID_ARG;
    const EngineTuning old = b->tuning;
    b->tuning = EngineTuning{values[0], values[1], values[2], values[4]};
    const int rc = batch_build(b);
    if (rc != MTB_OK) {
        b->tuning = old;
        batch_build(b);
    }
    return rc;
}

int mtb_batch_status(mtb_batch_t *b, void *stream) {
    if (!b) return MTB_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return MTB_ERR_CUDA;
    for (int s = 0; s < b->count; ++s) {
        int32_t v = 0;
        const uint8_t *ws = b->workspace + b->ws_offset[s];
        if (cudaMemcpy(&v, ws + b->layouts[s].status_offset, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
            return MTB_ERR_CUDA;
        if (v != 0) return v;
    }
    return MTB_OK;
}

void mtb_batch_destroy(mtb_batch_t *b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->tables) cudaFree(b->tables);
    if (b->own_workspace && b->workspace) cudaFree(b->workspace);
    delete b;
}

}  // extern "C"
