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
// Scheduling: the search is latency-bound (each level needs the argmin of the
// level below), so all of it runs in one persistent kernel fed by a work queue
// in topological order:
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
#include <mutex>

#include "mtb_search_dev.cuh"

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
k_search(const mtb_layout_t L, uint8_t *__restrict__ ws, const SearchPlan P) {
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
// word of a search, then waits for the previous launch, so that the search
// launched after it also sees the bit planes complete.
__global__ void k_clear_search(const mtb_layout_t L, uint8_t *__restrict__ ws, int ref) {
    pdl_trigger();
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
    pdl_wait();
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
    P.bit_chunk_words = kBitWordsPerCta;
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

cudaError_t launch_search_ex(const mtb_layout_t &L, int ref_idx, uint8_t *ws, int32_t *shifts_out,
                             uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s, bool chained,
                             unsigned long long timeout_ns, int withhold_pair, bool overlap, bool chain) {
    int &nb = g_search_blocks_per_sm[overlap ? 1 : 0];
    if (nb == 0) {
        int v = 0;
        cudaError_t err = overlap
                              ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_search<true>, kSearchThreads, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_search<false>, kSearchThreads, 0);
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
        return launch_k(k_search<true>, dim3(grid), dim3(kSearchThreads), s, true, L, ws, P);
    cudaError_t err = launch_k(k_clear_search, dim3(1), dim3(1024), s, chained, L, ws, ref_idx);
    if (err != cudaSuccess) return err;
    return launch_k(k_search<false>, dim3(grid), dim3(kSearchThreads), s, true, L, ws, P);
}

cudaError_t launch_search(const mtb_layout_t &L, int ref_idx, uint8_t *ws, int32_t *shifts_out,
                          uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s, bool chained,
                          bool overlap, bool chain) {
    return launch_search_ex(L, ref_idx, ws, shifts_out, level_errs_out, level_shifts_out, s, chained,
                            kSearchTimeoutNs, -1, overlap, chain);
}

}  // namespace mtb
