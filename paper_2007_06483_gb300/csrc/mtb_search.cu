// mtb_search.cu -- coarse-to-fine shift search.
//
// Sec. III-A: starting at the deepest level with offset (0,0), the 9 candidates
// offset + (dx, dy), dx, dy in {-1, 0, +1}, are tested; the best is doubled and
// the next finer level searched around it.  Sec. III-B: the error of a
// candidate is the number of pixels set in
//     (tb_ref XOR S(tb_i)) AND eb_ref AND S(eb_i),
// S = move by the candidate with 0 outside the image.
//
// Arithmetic: the moved words of exposure i come from funnel shifts of three
// neighbouring words (the 3 x offsets of a row share them); a candidate is then
// XOR, AND, AND, popc on a 32-pixel word.  Counts are summed per warp with
// __reduce_add_sync and per CTA in shared memory.
//
// Two kernels carry it:
//   - k_search_staged (mtb_search_staged.cuh): bit planes staged in shared
//     memory by bulk copies ahead of the level that reads them; each pair's deep
//     levels on one thread-block cluster, the largest levels spread over the
//     whole grid.  Used whenever a level's rows fit the staging buffers.
//   - k_search_items, the fallback for rows too wide to stage (beyond about
//     12 K words): one persistent kernel fed by a work queue in topological
//     order:
//   1. window items: at the coarsest levels the whole reachable search window
//      (all shifts within +-(2^(levels-l) - 1) at level l) is cheap, so every
//      candidate of it is counted, one window row per item, with no dependency
//      between items;
//   2. one resolve item per pair: walks the coarse-to-fine chain through those
//      error tables (Sec. III-A's rule, unchanged: the counts at the candidates
//      it picks are the same counts);
//   3. for each larger level, coarse to fine, chunks of (word columns x rows)
//      for every pair; a chunk waits until all chunks of its pair's level
//      below are done, reads their 9 counters once (one thread, broadcast
//      through shared memory), searches, and adds its counts;
//   4. one final item that writes the shifts and the per-level outputs.
// CTAs take items in queue order, so every item waits only on items taken
// earlier by running CTAs: the waits always end.  Each wait is still bounded
// by a timeout that sets the workspace status word instead of hanging.
#include <cstdlib>
#include <mutex>

#include "mtb_search_staged.cuh"

static __device__ int32_t g_last_status[256];  // see last_status_slot

namespace mtb {
namespace {

// kOverlap: the launch directly follows the bitmap pass of the same call, whose
// clearing was done by the pyramid stage; the search then starts while the
// bitmaps are still being packed, and every item waits for the planes it reads
// (their completion counters, acquired; weak loads afterwards) instead of for
// the whole previous launch.  Its words that the call's clearing kernel zeroes
// (queue head, counters, status) are clear by the time it launches: the bitmap
// pass lets it launch only after its own wait on the pyramid pass, which
// completes only after the clearing kernel.
template <bool kOverlap>
// 3 CTAs per SM: 80 registers and no spills.  At 4 (64 registers) the item
// functions spilled 124 bytes and the 4000x3000x3 one-call step took 85.1 us
// instead of 80.8 us; at 2 it took 82.1 us.
__global__ void __launch_bounds__(kSearchThreads, 3)
k_search_items(const mtb_layout_t L, uint8_t *__restrict__ ws, const SearchPlan P) {
    __shared__ SearchShared sm;
    const int tid = threadIdx.x;
    pdl_trigger();
    if (!kOverlap) pdl_wait();  // bit planes and cleared counters come from the previous launches
    int32_t *head = Ctr::queue(ws, L);
    for (;;) {
        if (tid == 0) sm.item = atomicAdd(head, 1);
        __syncthreads();
        const int it = sm.item;
        __syncthreads();
        if (it >= P.total_items) break;
        const int n_window = P.pairs * P.window_items;
        if (it < n_window) {
            window_item<kOverlap>(L, ws, P, it, sm);
        } else if (it < n_window + P.pairs) {
            resolve_item(L, ws, P, it - n_window, sm);
        } else if (it == P.total_items - 1) {
            final_item(L, ws, P, sm);
        } else {
            int l = P.lc - 1;
            while (l > 0 && it >= P.first_item[l - 1]) --l;
            const int rel = it - P.first_item[l];
            shift_item<kOverlap>(L, ws, P, rel / P.chunks[l], l, rel % P.chunks[l], sm);
        }
    }
}

// Clears the error counters, the queue head, the done counters and the status
// word of a search.  Launched chained behind whatever the stream ran before, so
// its launch overlaps that kernel's end; it waits for that kernel before it
// writes anything (a previous search on the same workspace may still be
// running), and lets the search launch at once: the search waits for it in
// turn, so it also sees the bit planes complete.
__global__ void k_clear_search(const mtb_layout_t L, uint8_t *__restrict__ ws, int ref) {
    pdl_trigger();
    pdl_wait();
    uint32_t *errs = reinterpret_cast<uint32_t *>(ws + L.errs_offset);
    for (int k = threadIdx.x; k < L.n * L.levels * 9; k += blockDim.x) errs[k] = 0;
    for (int k = threadIdx.x; k < L.levels * 2; k += blockDim.x) {  // the reference's rows are zero
        Planes::base(ws, L, ref, 0)[k] = 0;
        Planes::shift(ws, L, ref, 0)[k] = 0;
    }
    int32_t *ctr = Ctr::queue(ws, L);
    for (int k = threadIdx.x; k < search_counter_words(L); k += blockDim.x) ctr[k] = 0;
    uint32_t *tab = reinterpret_cast<uint32_t *>(ws + L.table_offset);
    for (int k = threadIdx.x; k < L.n * kTableWords; k += blockDim.x) tab[k] = 0;
    if (threadIdx.x == 0) *status_word(ws, L) = 0;
}

// The staged search (mtb_search_staged.cuh).  kOverlap as for k_search_items.
// One CTA per SM: 768 threads and the staging buffers in shared memory.
template <bool kOverlap>
__global__ void __launch_bounds__(kStThreads, 1)
k_search_staged(const mtb_layout_t Lp, uint8_t *__restrict__ ws, const StagedPlan Pp) {
    extern __shared__ __align__(128) uint8_t st_dyn[];
    __shared__ StagedShared s;
    // the layout and the plan in shared memory: the chain reads their
    // per-level fields at every level, by a level index only known at run time
    __shared__ mtb_layout_t L;
    __shared__ StagedPlan P;
    static_assert(sizeof(mtb_layout_t) % 4 == 0 && sizeof(StagedPlan) % 4 == 0, "copied as 32-bit words");
    const int tid = threadIdx.x;
    for (int v = tid; v < (int)(sizeof(mtb_layout_t) / 4); v += kStThreads)
        reinterpret_cast<uint32_t *>(&L)[v] = reinterpret_cast<const uint32_t *>(&Lp)[v];
    for (int v = tid; v < (int)(sizeof(StagedPlan) / 4); v += kStThreads)
        reinterpret_cast<uint32_t *>(&P)[v] = reinterpret_cast<const uint32_t *>(&Pp)[v];
    if (tid == 0) {
        for (int k = 0; k < kMbCount; ++k)
            mbar_init_n(smem_addr(&s.mbar[k]), k == kMbCounted || k == kMbCounted + 1 ? kStCountWarps : 1);
        for (int k = 0; k < 9; ++k) s.acc[0][k] = s.acc[1][k] = s.prev[0][k] = s.prev[1][k] = 0;
        s.arrived[0] = s.arrived[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_trigger();
    if (!kOverlap) pdl_wait();  // bit planes and cleared counters come from the previous launches
    if (tid == 0) fence_proxy_global();
    cg::cluster_group cluster = cg::this_cluster();
    uint32_t ph = 0;  // parity of the current phase of each mbarrier this thread waits on
    int lv = 0;       // levels this CTA's cluster has searched (the exchange barriers' sequence)
    int32_t *pair_head = Ctr::queue(ws, L) + 1;
    for (;;) {
        // the cluster takes the next pair: rank 0 draws it, every rank reads it
        if (cluster.block_rank() == 0 && tid == 0) s.task = atomicAdd(pair_head, 1);
        cluster.sync();
        const int p = *cluster.map_shared_rank(&s.task, 0);
        if (p >= P.pairs) {
            cluster.sync();  // rank 0's word is read by all before any CTA moves on
            break;
        }
        // (the pair's first cluster barrier orders this read before rank 0's next draw)
        st_pair<kOverlap>(L, ws, P, p, s, st_dyn, ph, lv, cluster);
    }
    st_grid<kOverlap>(L, ws, P, s, st_dyn, ph);
}

int g_search_blocks_per_sm[2] = {0, 0};

// Last-status slots: one int32 per (device, stream) in a static device array,
// written by the final item of every search launched on the stream.  The
// runtime creates the array with the module: taking a slot allocates nothing.
constexpr int kStatusSlots = 256;
struct StatusSlots {
    int32_t *dev = nullptr;  // g_last_status on this device
    cudaStream_t key[kStatusSlots] = {};
    bool used[kStatusSlots] = {};
    int next = 0;  // slot to take when all are used (oldest first)
};
StatusSlots g_status[64];
std::mutex g_status_mu;

}  // namespace

int last_status_slot(cudaStream_t s, bool create, int32_t **dev_slot) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    std::lock_guard<std::mutex> g(g_status_mu);
    StatusSlots &t = g_status[dev];
    if (!t.dev) {
        void *a = nullptr;
        if (cudaGetSymbolAddress(&a, g_last_status) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        t.dev = static_cast<int32_t *>(a);
    }
    int k = 0;
    while (k < kStatusSlots && !(t.used[k] && t.key[k] == s)) ++k;
    if (k == kStatusSlots) {
        if (!create) return -1;
        k = 0;
        while (k < kStatusSlots && t.used[k]) ++k;
        if (k == kStatusSlots) {  // every slot taken: reuse the oldest
            k = t.next;
            t.next = (t.next + 1) % kStatusSlots;
        }
        t.used[k] = true;
        t.key[k] = s;
    }
    if (dev_slot) *dev_slot = t.dev + k;
    return k;
}

int read_last_status(int slot, int32_t *out) {
    return cudaMemcpyFromSymbol(out, g_last_status, sizeof(int32_t), (size_t)slot * sizeof(int32_t),
                                cudaMemcpyDeviceToHost) == cudaSuccess
               ? MTB_OK
               : MTB_ERR_CUDA;
}

// Levels at or above lc are searched by whole windows (see kBruteBudget).
int coarse_start_level(const mtb_layout_t &L, long long budget) {
    int lc = L.levels;
    while (lc > 0) {
        const int l = lc - 1;
        const long long R = (1ll << (L.levels - l)) - 1;
        if (R > kMaxTableRadius) break;
        const long long words = (long long)L.bits_pitch[l] * L.height[l];
        if (words * (2 * R + 1) * (2 * R + 1) > budget) break;
        --lc;
    }
    return lc;
}

void plan_search(const mtb_layout_t &L, int ref_idx, long long cap, int32_t *shifts_out, uint32_t *level_errs_out,
                 int32_t *level_shifts_out, unsigned long long timeout_ns, int withhold_pair, SearchPlan *out,
                 int chain, long long brute_budget) {
    SearchPlan &P = *out;
    P = SearchPlan{};
    P.ref = ref_idx;
    P.chain = chain;
    P.pairs = L.n - 1;
    P.lc = coarse_start_level(L, brute_budget);
    P.shifts_out = shifts_out;
    P.level_errs_out = level_errs_out;
    P.level_shifts_out = level_shifts_out;
    P.timeout_ns = timeout_ns;
    P.withhold_pair = withhold_pair;
    P.bit_chunk_words = bit_chunk_words(L);
    P.window_items = 0;
    for (int l = L.levels - 1; l >= P.lc; --l) {
        const long long words = (long long)L.bits_pitch[l] * L.height[l];
        const int R = (1 << (L.levels - l)) - 1;
        P.window_items += (int)((2 * R + 1) * window_parts(R) * ((words + kWindowChunk - 1) / kWindowChunk));
    }
    // each larger level is one wave: about cap / pairs chunks per pair, a chunk being
    // tx word columns x ty thread rows x rows_per_thread image rows
    long long item = (long long)P.pairs * (P.window_items + 1);  // window items, resolve items
    const long long per_pair = cap / P.pairs > 0 ? cap / P.pairs : 1;
    for (int l = P.lc - 1; l >= 0; --l) {
        const int bp = L.bits_pitch[l], hl = L.height[l];
        const int tx = bp >= 64 ? 64 : ((bp + 31) / 32) * 32;
        const int ty = kSearchThreads / tx;
        const int col_blocks = (bp + tx - 1) / tx;
        long long row_blocks = per_pair / col_blocks;
        const long long max_row_blocks = (hl + ty * kRowBatch - 1) / (ty * kRowBatch);
        row_blocks = row_blocks < 1 ? 1 : (row_blocks > max_row_blocks ? max_row_blocks : row_blocks);
        const int rpt = (int)((hl + ty * row_blocks - 1) / (ty * row_blocks));
        P.tx[l] = tx;
        P.ty[l] = ty;
        P.col_blocks[l] = col_blocks;
        P.rows_per_thread[l] = rpt;
        P.chunks[l] = (int)(col_blocks * ((hl + ty * rpt - 1) / (ty * rpt)));
        P.first_item[l] = (int)item;
        item += (long long)P.pairs * P.chunks[l];
    }
    item += 1;  // final item
    P.total_items = item > 0x7fffffffLL ? -1 : (int)item;
}

namespace {

// Cluster shape of the staged search on one device: CTAs per cluster and the
// clusters that fit at once (one CTA per SM).  The largest cluster whose
// co-resident clusters still cover most SMs is taken: a bigger cluster gives a
// pair more SMs for its deep levels, more clusters give the grid levels more
// CTAs.
struct ClusterShape {
    int cluster = 0, clusters = 0;
};
ClusterShape g_shape[64][2];
std::mutex g_shape_mu;

template <bool kOverlap>
cudaError_t query_shape(int cluster, int *clusters) {
    cudaError_t e = cudaFuncSetAttribute(k_search_staged<kOverlap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kStSmemBytes);
    if (e != cudaSuccess) return e;
    if (cluster > 8) {
        e = cudaFuncSetAttribute(k_search_staged<kOverlap>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(kStThreads);
    cfg.dynamicSmemBytes = kStSmemBytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, k_search_staged<kOverlap>, &cfg);
}

int env_int(const char *name, int fallback) {
    const char *v = std::getenv(name);
    if (!v || !*v) return fallback;
    char *end = nullptr;
    const long x = std::strtol(v, &end, 10);
    return (end && *end == 0) ? (int)x : fallback;
}

// MTB_SEARCH_CLUSTER (CTAs per cluster) overrides the choice, for tuning.
cudaError_t cluster_shape(bool overlap, ClusterShape *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int forced = env_int("MTB_SEARCH_CLUSTER", 0);
    std::lock_guard<std::mutex> g(g_shape_mu);
    ClusterShape &c = g_shape[dev][overlap ? 1 : 0];
    if (c.cluster == 0 || (forced > 0 && forced != c.cluster)) {
        const int sms = device_sm_count();
        ClusterShape best;
        const int sizes[] = {8, 4, 2, 1};
        for (int k : sizes) {
            if (forced > 0 && k != forced) continue;
            int n = 0;
            const cudaError_t e = overlap ? query_shape<true>(k, &n) : query_shape<false>(k, &n);
            if (e != cudaSuccess || n < 1) {
                cudaGetLastError();
                continue;
            }
            if (best.cluster == 0 || k * n > best.cluster * best.clusters) best = ClusterShape{k, n};
            if (k * n >= (sms * 5) / 6) break;  // the largest cluster that covers most SMs
        }
        if (best.cluster == 0) return cudaErrorInvalidConfiguration;
        c = best;
    }
    *out = c;
    return cudaSuccess;
}

// Cost of one grid-wide dependency hop in word-rows of counting per SM (about
// 2 us at ~1.8 word-rows per clock per SM): a level goes to the grid only when
// counting it there plus one more hop is cheaper than counting it on the
// pair's cluster.
constexpr long long kGridHopWords = 8192;

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// Rows one thread walks when a band of `rows` rows x bp words is counted by
// `threads` threads (one word column and a run of rows each).
int seg_rows(int rows, int bp, int threads) {
    const int runs = bp >= threads ? 1 : threads / bp;
    const int seg = (int)ceil_div(rows, runs);
    return seg > 0 ? seg : 1;
}

}  // namespace

int plan_staged_search(const mtb_layout_t &L, int ref_idx, int cluster, int clusters, int32_t *shifts_out,
                       uint32_t *level_errs_out, int32_t *level_shifts_out, unsigned long long timeout_ns,
                       int withhold_pair, int chain, int split, StagedPlan *out) {
    StagedPlan &P = *out;
    P = StagedPlan{};
    P.ref = ref_idx;
    P.chain = chain;
    P.pairs = L.n - 1;
    P.cluster = cluster;
    P.shifts_out = shifts_out;
    P.level_errs_out = level_errs_out;
    P.level_shifts_out = level_shifts_out;
    P.timeout_ns = timeout_ns;
    P.withhold_pair = withhold_pair;
    P.bit_chunk_words = bit_chunk_words(L);
    P.status_out = nullptr;
    if (cluster < 1 || cluster > kStMaxCluster || clusters < 1 || P.pairs < 1) return MTB_ERR_INVALID_ARG;
    const int top = L.levels - 1;
    const long long ctas = (long long)cluster * clusters;
    const long long rounds = ceil_div(P.pairs, clusters);  // pairs per cluster
    auto row_bytes = [&](int l) { return (long long)L.bits_pitch[l] * 8; };
    auto cl_band = [&](int l) { return (int)ceil_div(L.height[l], cluster); };
    // a cluster level fits when one CTA's reference band and the predicted
    // exposure rows fit a staging buffer (the deepest level's rows are exact)
    auto cl_fits = [&](int l) {
        const int halo = l == top ? 1 : kStHalo;
        return (2ll * cl_band(l) + 2 * halo) * row_bytes(l) + kStGuard <= kStBufBytes;
    };
    // deep levels: both planes copied whole at the pair's start
    int ld = L.levels;
    long long deep = 0;
    while (ld > 0) {
        const int l = ld - 1;
        const long long bytes = 2ll * L.height[l] * row_bytes(l);
        if (deep + bytes > kStDeepBytes) break;
        P.deep_off[l] = (int)deep;
        deep += bytes;
        --ld;
    }
    if (ld == L.levels && !cl_fits(top)) return MTB_ERR_INVALID_ARG;  // nothing to run the deepest level in
    int ls = top;
    while (ls > 0) {
        const int l = ls - 1;
        if (split >= 0) {
            if (l < split) break;
        } else {
            const long long words = (long long)L.bits_pitch[l] * L.height[l];
            const long long t_cluster = ceil_div(words * rounds, cluster);
            const long long t_grid = ceil_div(words * P.pairs, ctas) + kGridHopWords;
            if (t_cluster > t_grid) break;
        }
        if (l < ld && !cl_fits(l)) break;
        --ls;
    }
    P.ls = ls;
    P.ld = ld < ls ? ls : ld;
    for (int l = ls; l < L.levels; ++l) {
        P.band[l] = l >= P.ld ? L.height[l] : cl_band(l);
        P.seg[l] = seg_rows(P.band[l], L.bits_pitch[l], l >= P.ld ? kStSoloThreads : kStThreads);
    }
    // grid levels: bands of one pair's rows; the first grid level is sized so
    // that the CTAs not running a pair hold all of it, two tasks each
    const long long busy = (long long)(P.pairs < clusters ? P.pairs : clusters) * cluster;
    long long task = 0;
    for (int g = ls - 1; g >= 0; --g) {
        const long long cap = ((kStBufBytes - kStGuard) / row_bytes(g) - 2 * kStHalo) / 2;
        if (cap < 1) return MTB_ERR_INVALID_ARG;  // rows too wide to stage
        const long long holders = (g == ls - 1 && ctas > busy) ? ctas - busy : ctas;
        long long band = ceil_div((long long)L.height[g] * P.pairs, 2 * holders);
        if (band > cap) band = cap;
        if (band < 1) band = 1;
        P.band[g] = (int)band;
        P.seg[g] = seg_rows(P.band[g], L.bits_pitch[g], kStCounters);
        P.tasks[g] = (int)ceil_div(L.height[g], band);
        P.first_task[g] = (int)task;
        task += (long long)P.pairs * P.tasks[g];
        if (task > 0x3fffffffLL) return MTB_ERR_INVALID_ARG;
    }
    P.total_tasks = (int)task + 1;  // the final task
    return MTB_OK;
}

namespace {

cudaError_t launch_items(const mtb_layout_t &L, int ref_idx, uint8_t *ws, int32_t *shifts_out,
                         uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s, bool chained,
                         unsigned long long timeout_ns, int withhold_pair, bool overlap, bool chain) {
    int &nb = g_search_blocks_per_sm[overlap ? 1 : 0];
    if (nb == 0) {
        int v = 0;
        cudaError_t err =
            overlap ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_search_items<true>, kSearchThreads, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_search_items<false>, kSearchThreads, 0);
        if (err != cudaSuccess) return err;
        nb = v > 0 ? v : 1;
    }
    const long long cap = (long long)device_sm_count() * nb;
    SearchPlan P;
    plan_search(L, ref_idx, cap, shifts_out, level_errs_out, level_shifts_out, timeout_ns, withhold_pair, &P,
                chain ? 1 : 0);
    if (P.total_items < 0) return cudaErrorInvalidValue;
    P.status_out = nullptr;
    last_status_slot(s, true, &P.status_out);
    const int grid = (int)(P.total_items < cap ? P.total_items : cap);
    if (overlap)  // the pyramid stage of the same call cleared the search's areas
        return launch_k(k_search_items<true>, dim3(grid), dim3(kSearchThreads), s, true, L, ws, P);
    cudaError_t err = launch_k(k_clear_search, dim3(1), dim3(1024), s, true, L, ws, ref_idx);
    if (err != cudaSuccess) return err;
    return launch_k(k_search_items<false>, dim3(grid), dim3(kSearchThreads), s, true, L, ws, P);
}

}  // namespace

namespace {

// Whether a search of this stack runs the staged kernel (else the item kernel).
// The staged kernel needs whole SMs (one CTA each) in clusters: right behind
// the bitmap pass it starts only once bitmap CTAs have left whole SMs, and the
// item kernel, whose CTAs fit beside them, overlaps that pass about as well
// (6000x4000x7 one-call step: 242.4 us with the item kernel, 240.7 us with the
// staged one; 4000x3000x3: 78.3 against 85.4 us).  On its own the staged
// kernel wins from about 64 M pair-pixels at level 0 (6000x4000x7: 59.3
// against 69.6 us; 4000x3000x3: 41.7 against 40.7 us).  MTB_SEARCH_ITEMS=1
// (0) forces the item (staged) kernel, for comparisons and tests.
bool wants_staged(const mtb_layout_t &L, bool overlap) {
    const long long pair_pixels = (long long)L.w * L.h * (L.n - 1);
    const int forced = env_int("MTB_SEARCH_ITEMS", -1);
    return forced == 0 || (forced != 1 && !overlap && pair_pixels >= (64ll << 20));
}

}  // namespace

int search_kernel_choice(const mtb_layout_t &L, int ref_idx, bool overlap) {
    if (!wants_staged(L, overlap)) return 0;
    ClusterShape shape;
    if (cluster_shape(overlap, &shape) != cudaSuccess) return -1;
    StagedPlan P;
    return plan_staged_search(L, ref_idx, shape.cluster, shape.clusters, nullptr, nullptr, nullptr, 1, -1, 0,
                              env_int("MTB_SEARCH_SPLIT", -1), &P) == MTB_OK
               ? 1
               : 0;
}

cudaError_t launch_search_ex(const mtb_layout_t &L, int ref_idx, uint8_t *ws, int32_t *shifts_out,
                             uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s, bool chained,
                             unsigned long long timeout_ns, int withhold_pair, bool overlap, bool chain) {
    ClusterShape shape;
    cudaError_t err = cluster_shape(overlap, &shape);
    if (err != cudaSuccess) return err;
    // MTB_SEARCH_SPLIT (the finest level the clusters search) overrides the
    // planner's choice, for tuning
    StagedPlan P;
    if (!wants_staged(L, overlap) ||
        plan_staged_search(L, ref_idx, shape.cluster, shape.clusters, shifts_out, level_errs_out, level_shifts_out,
                           timeout_ns, withhold_pair, chain ? 1 : 0, env_int("MTB_SEARCH_SPLIT", -1),
                           &P) != MTB_OK)
        return launch_items(L, ref_idx, ws, shifts_out, level_errs_out, level_shifts_out, s, chained, timeout_ns,
                            withhold_pair, overlap, chain);
    last_status_slot(s, true, &P.status_out);
    if (!overlap) {
        err = launch_k(k_clear_search, dim3(1), dim3(1024), s, true, L, ws, ref_idx);
        if (err != cudaSuccess) return err;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(shape.cluster * shape.clusters);
    cfg.blockDim = dim3(kStThreads);
    cfg.dynamicSmemBytes = kStSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = shape.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;  // the search always follows its stage's previous kernel (bitmaps or clearing)
    return overlap ? cudaLaunchKernelEx(&cfg, k_search_staged<true>, L, ws, P)
                   : cudaLaunchKernelEx(&cfg, k_search_staged<false>, L, ws, P);
}

cudaError_t launch_search(const mtb_layout_t &L, int ref_idx, uint8_t *ws, int32_t *shifts_out,
                          uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s, bool chained,
                          bool overlap, bool chain) {
    return launch_search_ex(L, ref_idx, ws, shifts_out, level_errs_out, level_shifts_out, s, chained,
                            kSearchTimeoutNs, -1, overlap, chain);
}

}  // namespace mtb
