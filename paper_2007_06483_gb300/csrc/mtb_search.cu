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
#include "mtb_device.cuh"

namespace mtb {
namespace {

constexpr int kSearchThreads = 256;
constexpr int kRowBatch = 4;       // rows whose loads a thread issues together
constexpr int kWindowChunk = 1024;  // reference words per window item

// Moved (tb, eb) words of one exposure-i row for x offsets dx = +1, 0, -1
// (index j = 1 - dx).
struct Moved {
    uint32_t t[3], e[3];
};

// Words q, q+1, q+2 of row yi (0 outside the plane); the j-th result is the 32
// bits starting at bit o + j of word q.  Bit planes are read through L1: they
// come from the bitmap pass, an earlier launch.
__device__ __forceinline__ Moved moved_row(const uint2 *plane, int bp, int hl, int yi, int q, int o) {
    uint2 a = make_uint2(0u, 0u), b = a, c = a;
    if (yi >= 0 && yi < hl) {
        const uint2 *row = plane + (size_t)yi * bp;
        if (q >= 0 && q < bp) a = __ldg(row + q);
        if (q + 1 >= 0 && q + 1 < bp) b = __ldg(row + q + 1);
        if (q + 2 >= 0 && q + 2 < bp) c = __ldg(row + q + 2);
    }
    Moved m;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int off = o + j;
        const bool low = off < 32;
        m.t[j] = __funnelshift_r(low ? a.x : b.x, low ? b.x : c.x, off & 31);
        m.e[j] = __funnelshift_r(low ? a.y : b.y, low ? b.y : c.y, off & 31);
    }
    return m;
}

__device__ __forceinline__ uint32_t cand_err(uint2 r, const Moved &m, int j) {
    return __popc((r.x ^ m.t[j]) & r.y & m.e[j]);
}

// Adds the 9 candidate errors of reference word r given the moved rows for
// dy = +1 (rm), 0 (r0), -1 (rp).  Candidate order: (0,0), (-1,-1), (0,-1),
// (1,-1), (-1,0), (1,0), (-1,1), (0,1), (1,1).
__device__ __forceinline__ void add_candidates(uint32_t (&cnt)[9], uint2 r, const Moved &rm, const Moved &r0,
                                               const Moved &rp) {
    cnt[0] += cand_err(r, r0, 1);
    cnt[1] += cand_err(r, rp, 2);
    cnt[2] += cand_err(r, rp, 1);
    cnt[3] += cand_err(r, rp, 0);
    cnt[4] += cand_err(r, r0, 2);
    cnt[5] += cand_err(r, r0, 0);
    cnt[6] += cand_err(r, rm, 2);
    cnt[7] += cand_err(r, rm, 1);
    cnt[8] += cand_err(r, rm, 0);
}

struct SearchShared {
    uint32_t red[kSearchThreads / 32][2 * kMaxTableRadius + 1];
    uint32_t cnt[2 * kMaxTableRadius + 1];
    uint32_t table[kTableWords];
    int item;
    int bx, by;
    int ok;
};

// Sum of cnt over the CTA into sm.cnt; all threads must call it.
__device__ __forceinline__ void block_sum9(const uint32_t (&cnt)[9], SearchShared &sm) {
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[k]);
        if (lane == 0) sm.red[warp][k] = v;
    }
    __syncthreads();
    if (t < 9) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < kSearchThreads / 32; ++w) sum += sm.red[w][t];
        sm.cnt[t] = sum;
    }
    __syncthreads();
}

__device__ __forceinline__ int first_min9(const uint32_t *e) {
    int kb = 0;
    uint32_t best = e[0];
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        const uint32_t v = e[k];
        if (v < best) {
            best = v;
            kb = k;
        }
    }
    return kb;
}

// Geometry and queue layout of one search; filled on the host.
struct SearchPlan {
    int ref, lc, pairs, total_items;
    int window_items;  // window items (row of a level's window x word chunk) of one pair
    int32_t *shifts_out;
    uint32_t *level_errs_out;
    int32_t *level_shifts_out;
    unsigned long long timeout_ns;
    int withhold_pair;  // test hook: this pair's resolve item never reports completion (-1: none)
    int tx[MTB_MAX_LEVELS], ty[MTB_MAX_LEVELS], col_blocks[MTB_MAX_LEVELS], chunks[MTB_MAX_LEVELS];
    int rows_per_thread[MTB_MAX_LEVELS];
    int first_item[MTB_MAX_LEVELS];  // queue index of pair 0, chunk 0 of level l (l < lc)
};

__device__ __forceinline__ int32_t *done_ctr(uint8_t *ws, const mtb_layout_t &L, int p, int l) {
    return counters(ws, L) + L.n + kCtrDone + p * L.levels + l;
}
__device__ __forceinline__ int32_t *window_ctr(uint8_t *ws, const mtb_layout_t &L, int p) {
    return counters(ws, L) + L.n + kCtrDone + L.n * L.levels + p;
}

// Window radius of coarse level l, and the offset of its table in a pair's
// table area (the tables of the deeper levels come first).
__device__ __forceinline__ int window_radius(const mtb_layout_t &L, int l) { return (1 << (L.levels - l)) - 1; }
__device__ __forceinline__ int table_offset_of(const mtb_layout_t &L, int l) {
    int off = 0;
    for (int k = L.levels - 1; k > l; --k) {
        const int d = 2 * window_radius(L, k) + 1;
        off += d * d;
    }
    return off;
}
__device__ __forceinline__ uint32_t *pair_table(uint8_t *ws, const mtb_layout_t &L, int p) {
    return reinterpret_cast<uint32_t *>(ws + L.table_offset) + (size_t)p * kTableWords;
}

// Chunks of level l a pair must finish before level l - 1 may start.
__device__ __forceinline__ int level_target(const SearchPlan &P, int l) { return l >= P.lc ? 1 : P.chunks[l]; }

// Final shift of exposure i (level 0's best) and the per-level outputs; the
// reference gets zeros.  Reads go through L2: other CTAs wrote them.
__device__ void finalize_exposure(const mtb_layout_t &L, uint8_t *ws, const SearchPlan &P, int i) {
    int sx = 0, sy = 0;
    if (i != P.ref) {
        uint32_t e0[9];
        const uint32_t *ep = Planes::errs(ws, L, i, 0);
#pragma unroll
        for (int k = 0; k < 9; ++k) e0[k] = __ldcg(ep + k);
        const int kb = first_min9(e0);
        const int32_t *b0 = Planes::base(ws, L, i, 0);
        sx = __ldcg(b0) + cand_dx(kb);
        sy = __ldcg(b0 + 1) + cand_dy(kb);
    }
    int32_t *s0 = Planes::shift(ws, L, i, 0);
    s0[0] = sx;
    s0[1] = sy;
    if (P.shifts_out) {
        P.shifts_out[2 * i] = sx;
        P.shifts_out[2 * i + 1] = sy;
    }
    for (int l = 0; l < L.levels; ++l) {
        if (P.level_shifts_out) {
            const int32_t *sl = Planes::shift(ws, L, i, l);
            P.level_shifts_out[((size_t)i * L.levels + l) * 2] = l == 0 ? sx : __ldcg(sl);
            P.level_shifts_out[((size_t)i * L.levels + l) * 2 + 1] = l == 0 ? sy : __ldcg(sl + 1);
        }
        if (P.level_errs_out) {
            const uint32_t *el = Planes::errs(ws, L, i, l);
            for (int k = 0; k < 9; ++k) P.level_errs_out[((size_t)i * L.levels + l) * 9 + k] = __ldcg(el + k);
        }
    }
}

// Window item: row sy of the whole window of coarse level l of pair p -- the
// errors of all candidates (sx, sy), |sx| <= R, over the level.  With R <= 15
// the bits of exposure i that land on reference word w come from its words
// w-1, w, w+1 of row y - sy.
template <int R>
__device__ void window_row(const mtb_layout_t &L, uint8_t *ws, const SearchPlan &P, int p, int l, int sy,
                           int chunk, SearchShared &sm) {
    constexpr int D = 2 * R + 1;
    const int tid = threadIdx.x;
    const int i = p < P.ref ? p : p + 1;
    const int hl = L.height[l], bp = L.bits_pitch[l];
    const uint2 *pr = Planes::bits(ws, L, P.ref, l);
    const uint2 *pi = Planes::bits(ws, L, i, l);
    uint32_t cnt[D];
#pragma unroll
    for (int k = 0; k < D; ++k) cnt[k] = 0;
    const int idx_end = min(bp * hl, (chunk + 1) * kWindowChunk);
#pragma unroll 2
    for (int idx = chunk * kWindowChunk + tid; idx < idx_end; idx += kSearchThreads) {
        const int y = idx / bp, w = idx - y * bp;
        const uint2 r = __ldg(pr + idx);
        const int yi = y - sy;
        uint2 a = make_uint2(0u, 0u), b = a, c = a;
        if (yi >= 0 && yi < hl) {
            const uint2 *row = pi + (size_t)yi * bp;
            if (w >= 1) a = __ldg(row + w - 1);
            b = __ldg(row + w);
            if (w + 1 < bp) c = __ldg(row + w + 1);
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int sh = 32 + R - k;  // bit of the (a, b, c) window where word w's pixels start, sx = k - R
            const uint32_t t = sh < 32 ? __funnelshift_r(a.x, b.x, sh & 31) : __funnelshift_r(b.x, c.x, sh & 31);
            const uint32_t e = sh < 32 ? __funnelshift_r(a.y, b.y, sh & 31) : __funnelshift_r(b.y, c.y, sh & 31);
            cnt[k] += __popc((r.x ^ t) & r.y & e);
        }
    }
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[k]);
        if (lane == 0) sm.red[warp][k] = v;
    }
    __syncthreads();
    if (tid < D) {
        uint32_t sum = 0;
#pragma unroll
        for (int wi = 0; wi < kSearchThreads / 32; ++wi) sum += sm.red[wi][tid];
        if (sum) atomicAdd(pair_table(ws, L, p) + table_offset_of(L, l) + (sy + R) * D + tid, sum);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(window_ctr(ws, L, p), 1);
}

__device__ void window_item(const mtb_layout_t &L, uint8_t *ws, const SearchPlan &P, int it, SearchShared &sm) {
    const int p = it / P.window_items;
    int rem = it - p * P.window_items;
    int l = L.levels - 1;
    int nchunks = 1;
    for (;; --l) {
        const int d = 2 * window_radius(L, l) + 1;
        nchunks = (L.bits_pitch[l] * L.height[l] + kWindowChunk - 1) / kWindowChunk;
        if (rem < d * nchunks) break;
        rem -= d * nchunks;
    }
    const int R = window_radius(L, l);
    const int sy = rem / nchunks - R;
    const int chunk = rem % nchunks;
    switch (R) {
        case 1: window_row<1>(L, ws, P, p, l, sy, chunk, sm); break;
        case 3: window_row<3>(L, ws, P, p, l, sy, chunk, sm); break;
        case 7: window_row<7>(L, ws, P, p, l, sy, chunk, sm); break;
        default: window_row<15>(L, ws, P, p, l, sy, chunk, sm); break;
    }
}

// Resolve item: the coarse-to-fine walk of pair p through its window tables,
// levels levels-1 .. lc, writing each level's 9 errors, base and shift.
__device__ void resolve_item(const mtb_layout_t &L, uint8_t *ws, const SearchPlan &P, int p, SearchShared &sm) {
    const int tid = threadIdx.x;
    const int i = p < P.ref ? p : p + 1;
    if (tid == 0) {
        sm.ok = wait_at_least(window_ctr(ws, L, p), P.window_items, status_word(ws, L), P.timeout_ns);
        __threadfence();
    }
    __syncthreads();
    if (!sm.ok) return;
    const int words = table_offset_of(L, P.lc - 1);
    const uint32_t *tab = pair_table(ws, L, p);
    for (int k = tid; k < words; k += kSearchThreads) sm.table[k] = __ldcg(tab + k);
    __syncthreads();
    if (tid == 0) {
        int bx = 0, by = 0;
        for (int l = L.levels - 1; l >= P.lc; --l) {
            const int R = window_radius(L, l), D = 2 * R + 1;
            const uint32_t *t = sm.table + table_offset_of(L, l);
            uint32_t e[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) e[k] = t[(by + cand_dy(k) + R) * D + (bx + cand_dx(k) + R)];
            const int kb = first_min9(e);
            const int sx = bx + cand_dx(kb), sy = by + cand_dy(kb);
            uint32_t *el = Planes::errs(ws, L, i, l);
#pragma unroll
            for (int k = 0; k < 9; ++k) el[k] = e[k];
            int32_t *b = Planes::base(ws, L, i, l);
            int32_t *s = Planes::shift(ws, L, i, l);
            b[0] = bx;
            b[1] = by;
            s[0] = sx;
            s[1] = sy;
            bx = 2 * sx;
            by = 2 * sy;
        }
        __threadfence();
        if (p != P.withhold_pair && P.lc < L.levels) atomicAdd(done_ctr(ws, L, p, P.lc), 1);
    }
    __syncthreads();
}

// Chunk c of level l of pair p.
__device__ void shift_item(const mtb_layout_t &L, uint8_t *ws, const SearchPlan &P, int p, int l, int c,
                           SearchShared &sm) {
    const int tid = threadIdx.x;
    const int i = p < P.ref ? p : p + 1;
    if (tid == 0) {
        int bx = 0, by = 0, ok = 1;
        if (l + 1 < L.levels) {
            ok = wait_at_least(done_ctr(ws, L, p, l + 1), level_target(P, l + 1), status_word(ws, L), P.timeout_ns);
            if (ok) {
                uint32_t e1[9];
                const uint32_t *ep = Planes::errs(ws, L, i, l + 1);
#pragma unroll
                for (int k = 0; k < 9; ++k) e1[k] = __ldcg(ep + k);
                const int kb = first_min9(e1);
                const int32_t *b1 = Planes::base(ws, L, i, l + 1);
                const int psx = __ldcg(b1) + cand_dx(kb), psy = __ldcg(b1 + 1) + cand_dy(kb);
                bx = 2 * psx;
                by = 2 * psy;
                if (c == 0) {
                    int32_t *s1 = Planes::shift(ws, L, i, l + 1);
                    s1[0] = psx;
                    s1[1] = psy;
                }
            }
        }
        if (ok && c == 0) {
            int32_t *b0 = Planes::base(ws, L, i, l);
            b0[0] = bx;
            b0[1] = by;
        }
        sm.bx = bx;
        sm.by = by;
        sm.ok = ok;
    }
    __syncthreads();
    if (!sm.ok) return;
    const int bx = sm.bx, by = sm.by;
    const int hl = L.height[l], bp = L.bits_pitch[l];
    const int tx = P.tx[l], ty = P.ty[l], rpt = P.rows_per_thread[l];
    const int cb = c % P.col_blocks[l], rb = c / P.col_blocks[l];
    const int x = tid % tx, yb = tid / tx;
    const bool active = yb < ty;
    const uint2 *pr = Planes::bits(ws, L, P.ref, l);
    const uint2 *pi = Planes::bits(ws, L, i, l);
    const int w = cb * tx + x;
    const int t = -bx - 1;
    const int q = w + (t >> 5);
    const int o = t & 31;
    const int y0 = (rb * ty + yb) * rpt;
    const int y1 = min(hl, y0 + rpt);
    uint32_t cnt[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (active && w < bp && y0 < y1) {
        // moved rows of exposure i: row y - by - 1 + j serves reference row y for dy = 1 - j
        Moved m0 = moved_row(pi, bp, hl, y0 - by - 1, q, o);
        Moved m1 = moved_row(pi, bp, hl, y0 - by, q, o);
        for (int y = y0; y < y1; y += kRowBatch) {
            uint2 r[kRowBatch];
            Moved mn[kRowBatch];
#pragma unroll
            for (int j = 0; j < kRowBatch; ++j) {
                r[j] = y + j < y1 ? __ldg(pr + (size_t)(y + j) * bp + w) : make_uint2(0u, 0u);
                mn[j] = moved_row(pi, bp, hl, y + j - by + 1, q, o);
            }
#pragma unroll
            for (int j = 0; j < kRowBatch; ++j) {
                add_candidates(cnt, r[j], m0, m1, mn[j]);
                m0 = m1;
                m1 = mn[j];
            }
        }
    }
    block_sum9(cnt, sm);
    if (tid < 9 && sm.cnt[tid]) atomicAdd(Planes::errs(ws, L, i, l) + tid, sm.cnt[tid]);
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(done_ctr(ws, L, p, l), 1);
}

// Final item: waits for level 0 of every pair, then writes the outputs.
__device__ void final_item(const mtb_layout_t &L, uint8_t *ws, const SearchPlan &P, SearchShared &sm) {
    if (threadIdx.x == 0) {
        int ok = 1;
        for (int p = 0; p < P.pairs && ok; ++p)
            ok = wait_at_least(done_ctr(ws, L, p, 0), level_target(P, 0), status_word(ws, L), P.timeout_ns);
        sm.ok = ok;
        __threadfence();
    }
    __syncthreads();
    if (!sm.ok) return;
    for (int e = threadIdx.x; e < L.n; e += kSearchThreads) finalize_exposure(L, ws, P, e);
}

__global__ void __launch_bounds__(kSearchThreads, 3)
k_search(const mtb_layout_t L, uint8_t *__restrict__ ws, const SearchPlan P) {
    __shared__ SearchShared sm;
    const int tid = threadIdx.x;
    pdl_trigger();
    pdl_wait();  // bit planes and cleared counters come from the previous launches
    int32_t *head = counters(ws, L) + L.n + kCtrQueue;
    for (;;) {
        if (tid == 0) sm.item = atomicAdd(head, 1);
        __syncthreads();
        const int it = sm.item;
        __syncthreads();
        if (it >= P.total_items) break;
        const int n_window = P.pairs * P.window_items;
        if (it < n_window) {
            window_item(L, ws, P, it, sm);
        } else if (it < n_window + P.pairs) {
            resolve_item(L, ws, P, it - n_window, sm);
        } else if (it == P.total_items - 1) {
            final_item(L, ws, P, sm);
        } else {
            int l = P.lc - 1;
            while (l > 0 && it >= P.first_item[l - 1]) --l;
            const int rel = it - P.first_item[l];
            shift_item(L, ws, P, rel / P.chunks[l], l, rel % P.chunks[l], sm);
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
    int32_t *ctr = counters(ws, L) + L.n;
    for (int k = threadIdx.x; k < kCtrDone + L.n * L.levels + L.n; k += blockDim.x) ctr[k] = 0;
    uint32_t *tab = reinterpret_cast<uint32_t *>(ws + L.table_offset);
    for (int k = threadIdx.x; k < L.n * kTableWords; k += blockDim.x) tab[k] = 0;
    if (threadIdx.x == 0) *status_word(ws, L) = 0;
    pdl_wait();
}

int g_search_blocks_per_sm = 0;

}  // namespace

// Levels at or above lc are searched by whole windows (see kBruteBudget).
int coarse_start_level(const mtb_layout_t &L) {
    int lc = L.levels;
    while (lc > 0) {
        const int l = lc - 1;
        const long long R = (1ll << (L.levels - l)) - 1;
        if (R > kMaxTableRadius) break;
        const long long words = (long long)L.bits_pitch[l] * L.height[l];
        if (words * (2 * R + 1) * (2 * R + 1) > kBruteBudget) break;
        --lc;
    }
    return lc;
}

cudaError_t launch_search_ex(const mtb_layout_t &L, int ref_idx, uint8_t *ws, int32_t *shifts_out,
                             uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s, bool chained,
                             unsigned long long timeout_ns, int withhold_pair) {
    SearchPlan P = {};
    P.ref = ref_idx;
    P.pairs = L.n - 1;
    P.lc = coarse_start_level(L);
    P.shifts_out = shifts_out;
    P.level_errs_out = level_errs_out;
    P.level_shifts_out = level_shifts_out;
    P.timeout_ns = timeout_ns;
    P.withhold_pair = withhold_pair;
    P.window_items = 0;
    for (int l = L.levels - 1; l >= P.lc; --l) {
        const long long words = (long long)L.bits_pitch[l] * L.height[l];
        P.window_items += (int)((2 * ((1 << (L.levels - l)) - 1) + 1) * ((words + kWindowChunk - 1) / kWindowChunk));
    }
    if (g_search_blocks_per_sm == 0) {
        int v = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_search, kSearchThreads, 0);
        if (err != cudaSuccess) return err;
        g_search_blocks_per_sm = v > 0 ? v : 1;
    }
    const long long cap = (long long)device_sm_count() * g_search_blocks_per_sm;
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
    if (item > 0x7fffffffLL) return cudaErrorInvalidValue;
    P.total_items = (int)item;
    const int grid = (int)(P.total_items < cap ? P.total_items : cap);
    cudaError_t err = launch_k(k_clear_search, dim3(1), dim3(1024), s, chained, L, ws, ref_idx);
    if (err != cudaSuccess) return err;
    return launch_k(k_search, dim3(grid), dim3(kSearchThreads), s, true, L, ws, P);
}

cudaError_t launch_search(const mtb_layout_t &L, int ref_idx, uint8_t *ws, int32_t *shifts_out,
                          uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s, bool chained) {
    return launch_search_ex(L, ref_idx, ws, shifts_out, level_errs_out, level_shifts_out, s, chained,
                            kSearchTimeoutNs, -1);
}

}  // namespace mtb
