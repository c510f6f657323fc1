// mtb_search_dev.cuh -- device functions of the shift search (window, resolve,
// chunk and final items), shared by the stage kernel and the engine.
#pragma once

#include "mtb_device.cuh"

namespace mtb {

// Geometry and queue layout of one search; filled on the host.
struct SearchPlan {
    int ref, lc, pairs, total_items;
    int chain;         // 0: every exposure against ref; 1: against its neighbour towards ref
    int window_items;  // window items (row of a level's window x word chunk) of one pair
    int32_t *shifts_out;
    uint32_t *level_errs_out;
    int32_t *level_shifts_out;
    unsigned long long timeout_ns;
    int withhold_pair;  // test hook: this pair's resolve item never reports completion (-1: none)
    int32_t *status_out;  // the launching stream's last-status slot (host-mapped; may be null)
    int tx[MTB_MAX_LEVELS], ty[MTB_MAX_LEVELS], col_blocks[MTB_MAX_LEVELS], chunks[MTB_MAX_LEVELS];
    int rows_per_thread[MTB_MAX_LEVELS];
    int bit_chunk_words;  // words per bitmap chunk (the engine waits for all chunks of a level)
    int first_item[MTB_MAX_LEVELS];  // queue index of pair 0, chunk 0 of level l (l < lc)
};

// brute_budget: word-candidate evaluations per pair allowed to the coarse
// windows (0: every level is a 9-candidate hop).
void plan_search(const mtb_layout_t &L, int ref_idx, long long cap, int32_t *shifts_out, uint32_t *level_errs_out,
                 int32_t *level_shifts_out, unsigned long long timeout_ns, int withhold_pair, SearchPlan *out,
                 int chain = 0, long long brute_budget = kBruteBudget);

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
template <bool kEng>
__device__ __forceinline__ Moved moved_row(const uint2 *plane, int bp, int hl, int yi, int q, int o) {
    uint2 a = make_uint2(0u, 0u), b = a, c = a;
    if (yi >= 0 && yi < hl) {
        const uint2 *row = plane + (size_t)yi * bp;
        if (q >= 0 && q < bp) a = kEng ? ld_weak(row + q) : __ldg(row + q);
        if (q + 1 >= 0 && q + 1 < bp) b = kEng ? ld_weak(row + q + 1) : __ldg(row + q + 1);
        if (q + 2 >= 0 && q + 2 < bp) c = kEng ? ld_weak(row + q + 2) : __ldg(row + q + 2);
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

__device__ __forceinline__ int32_t *done_ctr(uint8_t *ws, const mtb_layout_t &L, int p, int l) {
    return Ctr::done(ws, L, p, l);
}
__device__ __forceinline__ int32_t *window_ctr(uint8_t *ws, const mtb_layout_t &L, int p) {
    return Ctr::window(ws, L, p);
}

// Bit-plane loads.  The search stage reads planes an earlier launch wrote
// (non-coherent path, ld.global.nc); inside the engine the planes come from the
// same launch, so the loads are weak ld.global, made safe by the acquire of the
// planes' completion counters (kEng).
template <bool kEng>
__device__ __forceinline__ uint2 bit_load(const uint2 *p) {
    return kEng ? ld_weak(p) : __ldg(p);
}

// The exposure that moving exposure i is searched against: ref itself, or in
// chain mode its neighbour towards ref.
__device__ __forceinline__ int pair_ref(const SearchPlan &P, int i) {
    return P.chain ? (i < P.ref ? i + 1 : i - 1) : P.ref;
}

// Engine and overlapped search: thread 0 waits until level l of exposure i and
// of the exposure it is searched against is packed.
template <bool kEng>
__device__ __forceinline__ bool wait_bits(uint8_t *ws, const mtb_layout_t &L, const SearchPlan &P, int i, int l) {
    if (!kEng) return true;
    const int target = bitmap_target(L, l, P.bit_chunk_words);
    return wait_at_least(Ctr::bit_done(ws, L, pair_ref(P, i), l), target, status_word(ws, L), P.timeout_ns) &&
           wait_at_least(Ctr::bit_done(ws, L, i, l), target, status_word(ws, L), P.timeout_ns);
}

// Window items a row of a radius-R window is split into (by candidate columns).
__host__ __device__ __forceinline__ int window_parts(int R) { return R > 7 ? 2 : 1; }

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
    if (P.shifts_out && !P.chain) {
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
// Candidates sx = k - R for k in [K0, K0 + N) of the row (the radius-15 rows are
// split in two halves to bound the registers a thread needs).
template <bool kEng, int R, int K0, int N>
__device__ void window_row(const mtb_layout_t &L, uint8_t *ws, const SearchPlan &P, int p, int l, int sy,
                           int chunk, SearchShared &sm) {
    constexpr int D = 2 * R + 1;
    const int tid = threadIdx.x;
    const int i = p < P.ref ? p : p + 1;
    if (kEng) {
        if (tid == 0) sm.ok = wait_bits<kEng>(ws, L, P, i, l);
        __syncthreads();
        if (!sm.ok) return;
    }
    const int hl = L.height[l], bp = L.bits_pitch[l];
    const uint2 *pr = Planes::bits(ws, L, pair_ref(P, i), l);
    const uint2 *pi = Planes::bits(ws, L, i, l);
    uint32_t cnt[N];
#pragma unroll
    for (int k = 0; k < N; ++k) cnt[k] = 0;
    const int idx_end = min(bp * hl, (chunk + 1) * kWindowChunk);
#pragma unroll 2
    for (int idx = chunk * kWindowChunk + tid; idx < idx_end; idx += kSearchThreads) {
        const int y = idx / bp, w = idx - y * bp;
        const uint2 r = bit_load<kEng>(pr + idx);
        const int yi = y - sy;
        uint2 a = make_uint2(0u, 0u), b = a, c = a;
        if (yi >= 0 && yi < hl) {
            const uint2 *row = pi + (size_t)yi * bp;
            if (w >= 1) a = bit_load<kEng>(row + w - 1);
            b = bit_load<kEng>(row + w);
            if (w + 1 < bp) c = bit_load<kEng>(row + w + 1);
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int k = K0 + j;
            const int sh = 32 + R - k;  // bit of the (a, b, c) window where word w's pixels start, sx = k - R
            const uint32_t t = sh < 32 ? __funnelshift_r(a.x, b.x, sh & 31) : __funnelshift_r(b.x, c.x, sh & 31);
            const uint32_t e = sh < 32 ? __funnelshift_r(a.y, b.y, sh & 31) : __funnelshift_r(b.y, c.y, sh & 31);
            cnt[j] += __popc((r.x ^ t) & r.y & e);
        }
    }
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[j]);
        if (lane == 0) sm.red[warp][j] = v;
    }
    __syncthreads();
    if (tid < N) {
        uint32_t sum = 0;
#pragma unroll
        for (int wi = 0; wi < kSearchThreads / 32; ++wi) sum += sm.red[wi][tid];
        if (sum) atomicAdd(pair_table(ws, L, p) + table_offset_of(L, l) + (sy + R) * D + K0 + tid, sum);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(window_ctr(ws, L, p), 1);
}

template <bool kEng>
__device__ void window_item(const mtb_layout_t &L, uint8_t *ws, const SearchPlan &P, int it, SearchShared &sm) {
    const int p = it / P.window_items;
    int rem = it - p * P.window_items;
    int l = L.levels - 1;
    int nchunks = 1, parts = 1;
    for (;; --l) {
        const int R = window_radius(L, l);
        const int d = 2 * R + 1;
        parts = window_parts(R);
        nchunks = (L.bits_pitch[l] * L.height[l] + kWindowChunk - 1) / kWindowChunk;
        if (rem < d * nchunks * parts) break;
        rem -= d * nchunks * parts;
    }
    const int R = window_radius(L, l);
    const int part = rem % parts;
    rem /= parts;
    const int sy = rem / nchunks - R;
    const int chunk = rem % nchunks;
    switch (R) {
        case 1: window_row<kEng, 1, 0, 3>(L, ws, P, p, l, sy, chunk, sm); break;
        case 3: window_row<kEng, 3, 0, 7>(L, ws, P, p, l, sy, chunk, sm); break;
        case 7: window_row<kEng, 7, 0, 15>(L, ws, P, p, l, sy, chunk, sm); break;
        default:
            if (part == 0) window_row<kEng, 15, 0, 16>(L, ws, P, p, l, sy, chunk, sm);
            else window_row<kEng, 15, 16, 15>(L, ws, P, p, l, sy, chunk, sm);
            break;
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
template <bool kEng>
__device__ void shift_item(const mtb_layout_t &L, uint8_t *ws, const SearchPlan &P, int p, int l, int c,
                           SearchShared &sm) {
    const int tid = threadIdx.x;
    const int i = p < P.ref ? p : p + 1;
    if (tid == 0) {
        int bx = 0, by = 0;
        // the planes first: they are usually ready before the level below is
        int ok = wait_bits<kEng>(ws, L, P, i, l);
        if (ok && l + 1 < L.levels) {
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
    const uint2 *pr = Planes::bits(ws, L, pair_ref(P, i), l);
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
        Moved m0 = moved_row<kEng>(pi, bp, hl, y0 - by - 1, q, o);
        Moved m1 = moved_row<kEng>(pi, bp, hl, y0 - by, q, o);
        for (int y = y0; y < y1; y += kRowBatch) {
            uint2 r[kRowBatch];
            Moved mn[kRowBatch];
#pragma unroll
            for (int j = 0; j < kRowBatch; ++j) {
                r[j] = y + j < y1 ? bit_load<kEng>(pr + (size_t)(y + j) * bp + w) : make_uint2(0u, 0u);
                mn[j] = moved_row<kEng>(pi, bp, hl, y + j - by + 1, q, o);
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
// Every way out of it leaves the search's status word (MTB_OK or
// MTB_ERR_TIMEOUT) in the stream's last-status slot.
__device__ void final_item(const mtb_layout_t &L, uint8_t *ws, const SearchPlan &P, SearchShared &sm) {
    if (threadIdx.x == 0) {
        int ok = 1;
        for (int p = 0; p < P.pairs && ok; ++p)
            ok = wait_at_least(done_ctr(ws, L, p, 0), level_target(P, 0), status_word(ws, L), P.timeout_ns);
        sm.ok = ok;
        __threadfence();
        if (P.status_out) {
            // the other items' waits that gave up have set the word by now or
            // set it after this one: a timeout is seen here or by ok == 0
            const int st = ld_acquire(status_word(ws, L));
            *reinterpret_cast<volatile int32_t *>(P.status_out) = st != 0 ? st : (ok ? MTB_OK : MTB_ERR_TIMEOUT);
        }
    }
    __syncthreads();
    if (!sm.ok) return;
    for (int e = threadIdx.x; e < L.n; e += kSearchThreads) finalize_exposure(L, ws, P, e);
    if (!P.chain || !P.shifts_out) return;
    // chain mode: the shift of exposure e is the sum of the pair shifts along its
    // chain to ref (the level-0 shift rows hold the pairs' own shifts)
    __syncthreads();
    for (int e = threadIdx.x; e < L.n; e += kSearchThreads) {
        int sx = 0, sy = 0;
        for (int j = e; j != P.ref; j += e < P.ref ? 1 : -1) {
            const int32_t *sj = Planes::shift(ws, L, j, 0);
            sx += sj[0];
            sy += sj[1];
        }
        P.shifts_out[2 * e] = sx;
        P.shifts_out[2 * e + 1] = sy;
    }
}

}  // namespace
}  // namespace mtb
