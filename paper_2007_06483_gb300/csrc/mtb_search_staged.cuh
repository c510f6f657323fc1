// mtb_search_staged.cuh -- the shift search with its bit planes staged in
// shared memory by bulk copies.
//
// Sec. III-A: the search runs from the deepest level to level 0; at each level
// the 9 candidates base + (dx, dy), dx, dy in {-1, 0, +1}, are scored and the
// best one, doubled, is the next level's base.  Sec. III-B: the score of a
// candidate is the number of pixels set in
//     (tb_ref XOR S(tb_i)) AND eb_ref AND S(eb_i),
// S = move by the candidate with 0 outside the image.
//
// The levels form a chain: level l needs the argmin of level l + 1.  What the
// chain costs is the latency of each hop, so the design keeps the data of a
// level in shared memory before the level's base is known:
//   - base_l = 2 s_(l+1) = 4 s_(l+2) + 2d, d in {-1, 0, 1}, so once s_(l+2) is
//     known, the rows of exposure i that level l can touch lie within 3 rows of
//     4 s_(l+2) away from the reference rows.  That superset is copied into
//     shared memory (one bulk copy of whole rows, completion on an mbarrier)
//     while level l + 1 is still being counted.
//   - Every pair's coarse levels run on one thread-block cluster.  At a cluster
//     level each CTA counts one band of reference rows, pushes its 9 partial
//     counts into every CTA of the cluster (distributed shared memory) and
//     meets the others at the cluster barrier; every CTA then takes the same
//     argmin, so nothing needs broadcasting.  The deepest levels (a few KB) are
//     copied whole at the pair's start and counted whole by every CTA of the
//     cluster, with a reduction inside the CTA: the same counts, hence the
//     same argmin, in every CTA with no exchange between them.  Only the first
//     kStSoloWarps warps run them; the others wait for their base at the first
//     cluster level.
//   - The largest levels are spread over every CTA of the grid as tasks (one
//     band of reference rows of one pair) taken from a queue in level order.
//     A CTA holds two tasks, one per staging buffer: the second one's rows are
//     copied while the first is counted.  A task waits for the level above
//     through a completion counter in global memory.
// Every wait is on work held by running CTAs (pairs and tasks are taken from
// queues by CTAs that are already running, in dependency order) or on the
// bitmap pass, so the waits always end; each is still bounded by a timeout
// that sets the workspace status word instead of hanging.
#pragma once

#include <cooperative_groups.h>

#include "mtb_search_dev.cuh"

namespace mtb {

constexpr int kStThreads = 768;  // one CTA per SM (shared memory), 84 registers at most
constexpr int kStWarps = kStThreads / 32;
// the deep levels run on the first kStSoloWarps warps only (named barrier 1):
// a level of a few KB has too little work for 24 warps, and every warp that
// takes part runs the level's reduction and argmin
constexpr int kStSoloWarps = 8;
constexpr int kStSoloThreads = kStSoloWarps * 32;
constexpr int kStMaxCluster = 16;
constexpr int kStBufBytes = 98 * 1024;  // each of the two staging buffers
constexpr int kStDeepBytes = 24 * 1024;  // the deep levels of one pair
constexpr int kStSmemBytes = 2 * kStBufBytes + kStDeepBytes;
constexpr int kStHalo = 3;  // rows of a predicted exposure band beyond the reference band, each side
// A staging buffer holds the reference rows, then 16 zero bytes (the guard),
// then the exposure rows.  Every bit-plane row ends in at least 2 zero words,
// so with the guard a word index of -2 .. pitch - 1 relative to any staged
// exposure row reads either data or a zero that lies outside the image.
constexpr int kStGuard = 16;
__host__ __device__ __forceinline__ size_t st_exp_offset(int ref_rows, int bp) {
    return (size_t)ref_rows * bp * 8 + kStGuard;
}

// Geometry and queues of one staged search; filled on the host.
struct StagedPlan {
    int ref, pairs, chain;
    int cluster;  // CTAs per cluster
    int ls;       // levels >= ls run on the pair's cluster, levels < ls on the grid
    int ld;       // levels >= ld (the deep levels) are copied whole at the pair's start and
                  // counted whole by every CTA of the cluster
    // per level: reference rows of one band (cluster levels: one CTA's band;
    // deep levels: the whole level; grid levels: one task's band) and the rows
    // one thread walks
    int band[MTB_MAX_LEVELS], seg[MTB_MAX_LEVELS];
    int tasks[MTB_MAX_LEVELS];       // grid levels: tasks (bands) per pair
    int first_task[MTB_MAX_LEVELS];  // grid levels: queue index of pair 0's band 0
    int deep_off[MTB_MAX_LEVELS];    // deep levels: byte offset in the deep area (the whole plane of ref, then of i)
    int total_tasks;                 // grid tasks plus the final task
    int bit_chunk_words;
    int withhold_pair;  // test hook: this pair's cluster work never reports completion (-1: none)
    unsigned long long timeout_ns;
    int32_t *shifts_out;
    uint32_t *level_errs_out;
    int32_t *level_shifts_out;
    int32_t *status_out;
};

namespace {

namespace cg = cooperative_groups;

// mbarriers.  Cluster levels: 0, 1 the reference rows of buffers 0, 1; 2, 3
// the exposure rows of buffers 0, 1; 4 the deep area; 11, 12 the partial
// counts of a level from every rank (by level parity: the bytes of all ranks'
// remote stores plus the own thread 0's arrival).  Grid tasks: 5, 6 buffer b
// full (the producer's one arrival plus the bytes of both copies); 7, 8 buffer
// b counted (one arrival per counting warp); 9, 10 buffer b released (the
// publisher has taken its counts).
constexpr int kMbRef = 0, kMbExp = 2, kMbDeep = 4, kMbFull = 5, kMbCounted = 7, kMbReleased = 9, kMbLvl = 11,
              kMbCount = 13;
// grid tasks: warp 0 stages (the producer), warp 1 publishes, the others count
constexpr int kStCountWarps = kStWarps - 2;
constexpr int kStCounters = kStCountWarps * 32;
constexpr int kStCache = 32;  // the producer's cache of (pair, level) choices

// A grid task as the producer hands it to the counting warps.
struct StagedTask {
    int t, g, p, band, ok, bx, by, ea, ne;
};

struct StagedShared {
    unsigned long long mbar[kMbCount];
    // cluster levels, by level parity: the CTA's running sums of the 9 counts,
    // their values at the previous level of that parity, the warps counted in
    // so far (running), and every rank's totals (remote stores)
    uint32_t acc[2][9], prev[2][9];
    uint32_t arrived[2];
    uint32_t slot[2][kStMaxCluster][9];
    uint32_t part[2][kStWarps][9];       // grid: each counting warp's counts of the task in buffer b;
                                         // deep levels: each warp's counts, by level parity
    StagedTask desc[2];                  // grid: the task in buffer b
    int cache_key[kStCache];             // grid: (pair, level) whose choice is known, -1 none
    int2 cache_val[kStCache];
    int task;                            // the pair a cluster draws (rank 0's word)
    int solo_base[2];                    // the base the deep levels leave for the first cluster level
    int ea[2], ne[2];                    // cluster levels: first exposure row staged in buffer b, rows
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init_n(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
// One arrival (the only one a phase expects) announcing `bytes` of copies.
__device__ __forceinline__ void mbar_arrive_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// Announces `bytes` of copies for the current phase without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// One arrival (release: the arriving thread's earlier writes are seen by the waiters).
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
// Cluster scope: the phase may be completed by other CTAs' remote stores.
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on mbarrier `mb`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mb) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mb)
                 : "memory");
}
// Address of the same shared variable in cluster rank `rank`.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
// Store of one word into another CTA's shared memory, completing 4 bytes on
// that CTA's mbarrier `rbar` (both cluster addresses).
__device__ __forceinline__ void st_remote(uint32_t raddr, uint32_t v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.u32 [%0], %1, [%2];" ::"r"(raddr), "r"(v),
                 "r"(rbar)
                 : "memory");
}
// Generic-proxy writes (the bitmap pass, seen through an acquire) before
// async-proxy reads of the same global memory.
__device__ __forceinline__ void fence_proxy_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// Generic-proxy reads of a buffer (ordered by a CTA barrier) before the bulk
// copy that overwrites it.
__device__ __forceinline__ void fence_proxy_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits (all threads) until mbarrier `k` completes the phase of parity bit k of
// `ph`, then flips that bit.  Bounded: past timeout_ns the status word is set
// to MTB_ERR_TIMEOUT and false returned.  Once the status word holds an error
// (from any wait of the search) the bound shrinks to kStQuickNs, still far
// longer than any copy takes, so a failed search ends quickly without leaving
// a copy of its own in flight.
constexpr unsigned long long kStQuickNs = 1000000ull;
__device__ __forceinline__ bool mbar_wait(StagedShared &s, int k, uint32_t &ph, int32_t *status,
                                          unsigned long long timeout_ns) {
    const uint32_t a = smem_addr(&s.mbar[k]);
    const uint32_t parity = (ph >> k) & 1u;
    bool done = mbar_test(a, parity);
    if (!done) {
        const unsigned long long start = global_timer_ns();
        for (int spin = 0; !done; ++spin) {
            done = mbar_test(a, parity);
            if (!done && (spin & 63) == 63) {
                const unsigned long long t = global_timer_ns() - start;
                if (t > timeout_ns || (t > kStQuickNs && ld_acquire(status) != 0)) {
                    atomicCAS(status, 0, MTB_ERR_TIMEOUT);
                    break;
                }
            }
        }
    }
    ph ^= 1u << k;
    return done;
}

__device__ __forceinline__ int st_exposure(const StagedPlan &P, int p) { return p < P.ref ? p : p + 1; }
__device__ __forceinline__ int st_pair_ref(const StagedPlan &P, int i) {
    return P.chain ? (i < P.ref ? i + 1 : i - 1) : P.ref;
}
__device__ __forceinline__ int st_target(const StagedPlan &P, int l) { return l >= P.ls ? 1 : P.tasks[l]; }

// Thread 0: waits until level l of exposure e is packed (only when the search
// overlaps the bitmap pass), then orders the bulk copies after those writes.
template <bool kOverlap>
__device__ __forceinline__ bool st_wait_plane(uint8_t *ws, const mtb_layout_t &L, const StagedPlan &P, int e, int l) {
    if (!kOverlap) return true;
    const bool ok = wait_at_least(Ctr::bit_done(ws, L, e, l), bitmap_target(L, l, P.bit_chunk_words),
                                  status_word(ws, L), P.timeout_ns);
    fence_proxy_global();
    return ok;
}

// The shift level l of pair exposure i chose: its base plus its argmin
// candidate.  Valid once the level's completion counter reached its target
// (acquired); the counts and base are read through L2.
__device__ __forceinline__ int2 st_choice(uint8_t *ws, const mtb_layout_t &L, int i, int l) {
    uint32_t e[9];
    const uint32_t *ep = Planes::errs(ws, L, i, l);
#pragma unroll
    for (int k = 0; k < 9; ++k) e[k] = __ldcg(ep + k);
    const int kb = first_min9(e);
    const int32_t *b = Planes::base(ws, L, i, l);
    return make_int2(__ldcg(b) + cand_dx(kb), __ldcg(b + 1) + cand_dy(kb));
}

// Thread 0: copies rows [r0, r1) of plane `src` (bp words a row) to shared
// memory at `dst`, clipped to [0, hl), on mbarrier `mb` (one arrival; zero
// bytes when nothing is left).  Returns the first row copied and sets *rows.
__device__ __forceinline__ int st_copy_rows(const uint2 *src, int bp, int hl, int r0, int r1, void *dst, uint32_t mb,
                                            int *rows) {
    if (r0 < 0) r0 = 0;
    if (r1 > hl) r1 = hl;
    const int n = r1 > r0 ? r1 - r0 : 0;
    const uint32_t bytes = (uint32_t)n * (uint32_t)bp * 8u;
    mbar_arrive_tx(mb, bytes);
    if (bytes) bulk_g2s(smem_addr(dst), src + (size_t)r0 * bp, bytes, mb);
    *rows = n;
    return r0;
}

// Moved (tb, eb) words of one staged exposure row (index rr, 0 outside the
// staged rows) for x offsets dx = 1 - j: the 32 bits starting at bit o + j of
// word q.  v0..v2: words q, q + 1, q + 2 lie inside the row.
template <bool kWide>
__device__ __forceinline__ Moved st_moved(const uint2 *sexp, int bp, int ne, int rr, int q, int o, bool v0, bool v1,
                                          bool v2) {
    uint2 a = make_uint2(0u, 0u), b = a, c = a;
    if ((unsigned)rr < (unsigned)ne) {
        const uint2 *row = sexp + rr * bp + q;
        if (v0) a = row[0];
        if (v1) b = row[1];
        if (kWide && v2) c = row[2];
    }
    Moved m;
    if (!kWide) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            m.t[j] = __funnelshift_r(a.x, b.x, o + j);
            m.e[j] = __funnelshift_r(a.y, b.y, o + j);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int off = o + j;
            const bool low = off < 32;
            m.t[j] = __funnelshift_r(low ? a.x : b.x, low ? b.x : c.x, off & 31);
            m.e[j] = __funnelshift_r(low ? a.y : b.y, low ? b.y : c.y, off & 31);
        }
    }
    return m;
}

// Adds the 9 candidate counts of a staged band: reference rows y0 .. y0+nr-1 at
// sref (bp words a row), exposure rows ea .. ea+ne-1 at sexp, base (bx, by).
// Thread u walks word column u % bp over `seg` rows of the band.
template <bool kWide>
__device__ __forceinline__ void st_count(const uint2 *sref, const uint2 *sexp, int nr, int ea, int ne, int bp, int y0,
                                         int bx, int by, int seg, int me, int threads, uint32_t (&cnt)[9]) {
    const int t = -bx - 1;
    const int qoff = t >> 5;  // arithmetic shift: floor division
    const int o = t & 31;
    const int nseg = (nr + seg - 1) / seg;
    const int items = bp * nseg;
    for (int u = me; u < items; u += threads) {
        const int sg = u / bp;
        const int w = u - sg * bp;
        const int k0 = sg * seg, k1 = min(nr, k0 + seg);
        const int q = w + qoff;
        const bool v0 = (unsigned)q < (unsigned)bp, v1 = (unsigned)(q + 1) < (unsigned)bp;
        const bool v2 = (unsigned)(q + 2) < (unsigned)bp;
        // exposure row y - by - 1 + j serves reference row y for dy = 1 - j
        const int rbase = y0 - by - ea;
        Moved m0 = st_moved<kWide>(sexp, bp, ne, rbase + k0 - 1, q, o, v0, v1, v2);
        Moved m1 = st_moved<kWide>(sexp, bp, ne, rbase + k0, q, o, v0, v1, v2);
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const uint2 r = sref[k * bp + w];
            const Moved mn = st_moved<kWide>(sexp, bp, ne, rbase + k + 1, q, o, v0, v1, v2);
            add_candidates(cnt, r, m0, m1, mn);
            m0 = m1;
            m1 = mn;
        }
    }
}

// Moved (tb, eb) words of the exposure row at p (word q of a staged row) for
// x offsets dx = 1 - j: the 32 bits starting at bit o + j of word q.  Reads
// words q, q + 1 (and q + 2 when kWide, o >= 30) without checks.
template <bool kWide>
__device__ __forceinline__ Moved st_moved_at(const uint2 *p, int o) {
    const uint2 a = p[0], b = p[1];
    Moved m;
    if (!kWide) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            m.t[j] = __funnelshift_r(a.x, b.x, o + j);
            m.e[j] = __funnelshift_r(a.y, b.y, o + j);
        }
    } else {
        const uint2 c = p[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int off = o + j;
            const bool low = off < 32;
            m.t[j] = __funnelshift_r(low ? a.x : b.x, low ? b.x : c.x, off & 31);
            m.e[j] = __funnelshift_r(low ? a.y : b.y, low ? b.y : c.y, off & 31);
        }
    }
    return m;
}

// The 9 candidate counts of a band staged in a buffer: reference rows
// y0 .. y0+nr-1 at sref, exposure rows ea .. ea+ne-1 at sexp (after the guard),
// base (bx, by), `words` data words a row.  Rows of exposure i outside the
// staged ones lie outside the image (0); only the reference rows whose moved
// rows reach past them are checked, the rest run without checks.  An item
// whose word q is outside [-2, words) reads only zeros and is skipped.
template <bool kWide>
__device__ __forceinline__ void st_count_fast(const uint2 *sref, const uint2 *sexp, int nr, int ea, int ne, int bp,
                                              int words, int y0, int bx, int by, int seg, int me, int threads,
                                              uint32_t (&cnt)[9]) {
    const int t = -bx - 1;
    const int qoff = t >> 5;  // arithmetic shift: floor division
    const int o = t & 31;
    const int nseg = (nr + seg - 1) / seg;
    const int items = bp * nseg;
    const int sb = y0 - by - ea;  // staged row of image row y0 - by (reference row 0, dy = 0)
    const Moved zero = {{0u, 0u, 0u}, {0u, 0u, 0u}};
    for (int u = me; u < items; u += threads) {
        const int sg = u / bp;
        const int w = u - sg * bp;
        const int q = w + qoff;
        if (q < -2 || q >= words) continue;
        const int k0 = sg * seg, k1 = min(nr, k0 + seg);
        // reference rows k in [kf0, kf1) have all three moved rows staged
        const int kf0 = max(k0, min(k1, 1 - sb)), kf1 = max(kf0, min(k1, ne - 1 - sb));
        const uint2 *ep = sexp + q;
        auto moved = [&](int r) { return (unsigned)r < (unsigned)ne ? st_moved_at<kWide>(ep + r * bp, o) : zero; };
        Moved m0 = moved(sb + k0 - 1), m1 = moved(sb + k0);
        int k = k0;
        for (; k < kf0; ++k) {
            const Moved mn = moved(sb + k + 1);
            add_candidates(cnt, sref[k * bp + w], m0, m1, mn);
            m0 = m1;
            m1 = mn;
        }
        const uint2 *rp = sref + k * bp + w;
        const uint2 *np = ep + (sb + k + 1) * bp;
#pragma unroll 2
        for (; k < kf1; ++k) {
            const Moved mn = st_moved_at<kWide>(np, o);
            add_candidates(cnt, *rp, m0, m1, mn);
            m0 = m1;
            m1 = mn;
            rp += bp;
            np += bp;
        }
        for (; k < k1; ++k) {
            const Moved mn = moved(sb + k + 1);
            add_candidates(cnt, sref[k * bp + w], m0, m1, mn);
            m0 = m1;
            m1 = mn;
        }
    }
}

__device__ __forceinline__ void st_count_staged(const uint2 *sref, const uint2 *sexp, int nr, int ea, int ne, int bp,
                                                int words, int y0, int bx, int by, int seg, int me, int threads,
                                                uint32_t (&cnt)[9]) {
    if (((-bx - 1) & 31) >= 30)
        st_count_fast<true>(sref, sexp, nr, ea, ne, bp, words, y0, bx, by, seg, me, threads, cnt);
    else
        st_count_fast<false>(sref, sexp, nr, ea, ne, bp, words, y0, bx, by, seg, me, threads, cnt);
}

// Thread `me` of `threads` counting threads.
__device__ __forceinline__ void st_count_any(const uint2 *sref, const uint2 *sexp, int nr, int ea, int ne, int bp,
                                             int y0, int bx, int by, int seg, int me, int threads,
                                             uint32_t (&cnt)[9]) {
    if (((-bx - 1) & 31) >= 30) st_count<true>(sref, sexp, nr, ea, ne, bp, y0, bx, by, seg, me, threads, cnt);
    else st_count<false>(sref, sexp, nr, ea, ne, bp, y0, bx, by, seg, me, threads, cnt);
}

// Shared-memory add with acquire-release semantics at CTA scope; returns the
// old value.
__device__ __forceinline__ uint32_t atom_add_acq_rel_cta(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_addr(p)), "r"(v) : "memory");
    return old;
}

// One warp's part of a cluster level's exchange (called by every warp of the
// CTA): its 9 counts into the CTA's running sums; the last warp to count
// itself in sends the CTA's totals to every rank's slot `rank` (parity q).
__device__ __forceinline__ void st_exchange(StagedShared &s, const uint32_t (&cnt)[9], int q, int rank, int C,
                                            int lane) {
    uint32_t v = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const uint32_t t = __reduce_add_sync(0xffffffffu, cnt[k]);
        if (lane == k) v = t;
    }
    if (lane < 9 && v) atomicAdd(&s.acc[q][lane], v);
    __syncwarp();
    uint32_t old = 0;
    if (lane == 0) old = atom_add_acq_rel_cta(&s.arrived[q], 1u);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old % kStWarps != kStWarps - 1) return;
    __syncwarp();  // lane 0's acquire covers the lanes that read the sums
    if (lane < 9) {
        const uint32_t tot = *reinterpret_cast<volatile uint32_t *>(&s.acc[q][lane]);
        const uint32_t x = tot - s.prev[q][lane];
        s.prev[q][lane] = tot;
        const uint32_t dst = smem_addr(&s.slot[q][rank][lane]), bar = smem_addr(&s.mbar[kMbLvl + q]);
        for (int k = 0; k < C; ++k) st_remote(cluster_addr(dst, (uint32_t)k), x, cluster_addr(bar, (uint32_t)k));
    }
}

// Writes level l's 9 counts, base and chosen shift of exposure i (warp 0 of the
// cluster's rank 0, lanes 0..8 the counts, lane 0 the rest).
__device__ __forceinline__ void st_store_level(const mtb_layout_t &L, uint8_t *ws, int i, int l, int lane,
                                               uint32_t e, int bx, int by, int sx, int sy) {
    if (lane < 9) Planes::errs(ws, L, i, l)[lane] = e;
    if (lane == 0) {
        int32_t *b = Planes::base(ws, L, i, l);
        int32_t *sh = Planes::shift(ws, L, i, l);
        b[0] = bx;
        b[1] = by;
        sh[0] = sx;
        sh[1] = sy;
    }
}

// The cluster's part of pair p: every level from the deepest down to ls.  A
// level has no CTA barrier: each warp adds its 9 counts into the CTA's running
// sums with shared atomics and counts itself in; the warp that arrives last
// sends the CTA's 9 totals (the running sums less their values at this
// parity's previous level) to every rank of the cluster by remote stores, which
// complete on each receiver's exchange barrier; every warp then waits on that
// barrier and takes the same argmin.  All CTAs of the cluster run it with the
// same p and reach the same barriers whatever their waits return.
template <bool kOverlap>
__device__ void st_pair(const mtb_layout_t &L, uint8_t *ws, const StagedPlan &P, int p, StagedShared &s,
                        uint8_t *dyn, uint32_t &ph, int &lv, cg::cluster_group &cluster) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int rank = (int)cluster.block_rank(), C = P.cluster;
    const int i = st_exposure(P, p), r = st_pair_ref(P, i);
    int32_t *status = status_word(ws, L);
    uint8_t *deep = dyn + 2 * kStBufBytes;
    // the deep levels: the whole planes of the reference and of exposure i
    if (tid == 0 && P.ld < L.levels) {
        for (int l = L.levels - 1; l >= P.ld; --l) st_wait_plane<kOverlap>(ws, L, P, r, l);
        for (int l = L.levels - 1; l >= P.ld; --l) st_wait_plane<kOverlap>(ws, L, P, i, l);
        uint32_t bytes = 0;
        for (int l = L.levels - 1; l >= P.ld; --l) bytes += 2u * (uint32_t)L.height[l] * (uint32_t)L.bits_pitch[l] * 8u;
        const uint32_t mb = smem_addr(&s.mbar[kMbDeep]);
        mbar_arrive_tx(mb, bytes);
        for (int l = L.levels - 1; l >= P.ld; --l) {
            const uint32_t pb = (uint32_t)L.height[l] * (uint32_t)L.bits_pitch[l] * 8u;
            uint8_t *dst = deep + P.deep_off[l];
            bulk_g2s(smem_addr(dst), Planes::bits(ws, L, r, l), pb, mb);
            bulk_g2s(smem_addr(dst + pb), Planes::bits(ws, L, i, l), pb, mb);
        }
    }
    bool deep_pending = P.ld < L.levels;
    const bool solo = tid < kStSoloThreads;
    int bx = 0, by = 0;
    for (int l = L.levels - 1; l >= P.ls; --l) {
        const int bp = L.bits_pitch[l], hl = L.height[l];
        const bool is_deep = l >= P.ld;
        if (is_deep && !solo) continue;  // these warps wait for the deep levels' base below
        if (l == P.ld - 1 && P.ld < L.levels) {
            __syncthreads();  // the deep levels are done: every warp takes their base
            bx = s.solo_base[0];
            by = s.solo_base[1];
        }
        const int y0 = is_deep ? 0 : min(hl, rank * P.band[l]), y1 = is_deep ? hl : min(hl, y0 + P.band[l]);
        const int b = l & 1;
        const int q = lv & 1;  // this (cluster) level's exchange barrier, sums and slots
        if (tid == 0) {
            // level l itself when no earlier level could stage it (the deepest
            // level when it is not copied whole: its base is 0), then level
            // l - 1 predicted from this level's base (base_(l-1) = 2 base_l + 2d);
            // ea/ne are written before the arrivals that publish them
            for (int n = l; n >= l - 1; --n) {
                if (n < P.ls || n >= P.ld || (n == l && l != L.levels - 1)) continue;
                const int bpn = L.bits_pitch[n], hn = L.height[n];
                const int z0 = min(hn, rank * P.band[n]), z1 = min(hn, z0 + P.band[n]);
                const int c = n == l ? 0 : 2 * by;
                const int halo = n == l ? 1 : kStHalo;
                st_wait_plane<kOverlap>(ws, L, P, r, n);
                st_wait_plane<kOverlap>(ws, L, P, i, n);
                fence_proxy_shared();
                const int bn = n & 1;
                uint8_t *buf = dyn + bn * kStBufBytes;
                const int lo = max(0, z0 - c - halo), hi = min(hn, z1 - c + halo);
                s.ea[bn] = lo;
                s.ne[bn] = hi > lo ? hi - lo : 0;
                *reinterpret_cast<uint4 *>(buf + st_exp_offset(z1 - z0, bpn) - kStGuard) = make_uint4(0, 0, 0, 0);
                int rows = 0;
                st_copy_rows(Planes::bits(ws, L, r, n), bpn, hn, z0, z1, buf, smem_addr(&s.mbar[kMbRef + bn]), &rows);
                st_copy_rows(Planes::bits(ws, L, i, n), bpn, hn, lo, hi, buf + st_exp_offset(z1 - z0, bpn),
                             smem_addr(&s.mbar[kMbExp + bn]), &rows);
            }
            // a cluster level's exchange: 9 words from every rank
            if (!is_deep) mbar_arrive_tx(smem_addr(&s.mbar[kMbLvl + q]), (uint32_t)(36 * C));
        }
        const uint2 *sref, *sexp;
        int ea, ne;
        if (is_deep) {
            if (deep_pending) {
                mbar_wait(s, kMbDeep, ph, status, P.timeout_ns);
                deep_pending = false;
            }
            sref = reinterpret_cast<const uint2 *>(deep + P.deep_off[l]);
            sexp = sref + (size_t)hl * bp;
            ea = 0;
            ne = hl;
        } else {
            mbar_wait(s, kMbRef + b, ph, status, P.timeout_ns);
            mbar_wait(s, kMbExp + b, ph, status, P.timeout_ns);
            sref = reinterpret_cast<const uint2 *>(dyn + b * kStBufBytes);
            sexp = reinterpret_cast<const uint2 *>(dyn + b * kStBufBytes + st_exp_offset(y1 - y0, bp));
            ea = s.ea[b];
            ne = s.ne[b];
        }
        uint32_t cnt[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (y1 > y0) {
            if (is_deep)
                st_count_any(sref, sexp, y1 - y0, ea, ne, bp, y0, bx, by, P.seg[l], tid, kStSoloThreads, cnt);
            else
                st_count_staged(sref, sexp, y1 - y0, ea, ne, bp, (L.width[l] + 31) >> 5, y0, bx, by, P.seg[l], tid,
                                kStThreads, cnt);
        }
        uint32_t e = 0;
        if (is_deep) {
            // the whole level in this CTA: each warp's 9 sums, one barrier, and
            // lane k of every warp adds candidate k over the warps (the buffer
            // of this level's parity is written again two levels on, after the
            // next level's barrier)
            uint32_t v = 0;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const uint32_t t = __reduce_add_sync(0xffffffffu, cnt[k]);
                if (lane == k) v = t;
            }
            if (lane < 9) s.part[b][tid >> 5][lane] = v;
            asm volatile("bar.sync 1, %0;" ::"n"(kStSoloThreads) : "memory");
            if (lane < 9)
#pragma unroll
                for (int w = 0; w < kStSoloWarps; ++w) e += s.part[b][w][lane];
        } else {
            st_exchange(s, cnt, q, rank, C, lane);
            // every warp: the level's totals and their argmin
            mbar_wait(s, kMbLvl + q, ph, status, P.timeout_ns);
            if (lane < 9)
                for (int k = 0; k < C; ++k) e += s.slot[q][k][lane];
        }
        uint32_t ev[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) ev[k] = __shfl_sync(0xffffffffu, e, k);
        const int kb = first_min9(ev);
        const int sx = bx + cand_dx(kb), sy = by + cand_dy(kb);
        if (rank == 0 && tid < 32) {
            st_store_level(L, ws, i, l, lane, e, bx, by, sx, sy);
            // the levels the grid's tasks wait for (ls) or predict from (ls + 1)
            if ((l == P.ls || l == P.ls + 1) && p != P.withhold_pair) {
                __threadfence();
                __syncwarp();
                if (lane == 0) atomicAdd(Ctr::done(ws, L, p, l), 1);
            }
        }
        bx = 2 * sx;
        by = 2 * sy;
        if (!is_deep) ++lv;
        if (is_deep && l == P.ld && tid == 0) {
            s.solo_base[0] = bx;
            s.solo_base[1] = by;
        }
    }
}

// ---------------------------------------------------------------------------
// Grid tasks.  Warp 0 of the CTA is the producer: it takes tasks from the
// queue, resolves what each depends on, issues the bulk copies and hands a
// task to the counting warps through buffer b's "full" mbarrier.  The counting
// warps report on buffer b's "counted" mbarrier; warp 1, the publisher, sums
// their counts, releases the buffer to the producer and publishes the counts
// (atomics, a fence and the completion counter).  Two buffers: while the
// counting warps work on one, the producer fills and arms the other, so the
// latency of the queue, of the dependencies and of the publication overlaps
// the counting.

__device__ __forceinline__ void st_decode(const StagedPlan &P, int t, int &g, int &p, int &band) {
    g = P.ls - 1;
    while (g > 0 && t >= P.first_task[g - 1]) --g;
    const int rel = t - P.first_task[g];
    p = rel / P.tasks[g];
    band = rel - p * P.tasks[g];
}

// Producer (lane 0): the choice of level l of pair p if the level is complete
// (cached once seen), waiting for it when `blocking`.  Returns whether it is
// known; a blocking wait that gave up returns false with the status word set.
__device__ bool st_known(const mtb_layout_t &L, uint8_t *ws, const StagedPlan &P, StagedShared &s, int p, int l,
                         bool blocking, int2 *out) {
    const int key = p * MTB_MAX_LEVELS + l;
    const int slot = key & (kStCache - 1);
    if (s.cache_key[slot] == key) {
        *out = s.cache_val[slot];
        return true;
    }
    const int32_t *ctr = Ctr::done(ws, L, p, l);
    const int target = st_target(P, l);
    if (ld_acquire(ctr) < target) {
        if (!blocking || !wait_at_least(ctr, target, status_word(ws, L), P.timeout_ns)) return false;
    }
    *out = st_choice(ws, L, st_exposure(P, p), l);
    s.cache_key[slot] = key;
    s.cache_val[slot] = *out;
    return true;
}

// Producer (lane 0): the copy of rows [r0, r1) (clipped to [0, hl)) of a plane
// into shared memory at dst, announced on mbarrier mb without arriving.
__device__ __forceinline__ int st_copy_rows_tx(const uint2 *src, int bp, int hl, int r0, int r1, void *dst,
                                               uint32_t mb, int *rows) {
    if (r0 < 0) r0 = 0;
    if (r1 > hl) r1 = hl;
    const int n = r1 > r0 ? r1 - r0 : 0;
    const uint32_t bytes = (uint32_t)n * (uint32_t)bp * 8u;
    if (bytes) {
        mbar_expect_tx(mb, bytes);
        bulk_g2s(smem_addr(dst), src + (size_t)r0 * bp, bytes, mb);
    }
    *rows = n;
    return r0;
}

// Producer (lane 0): the exposure rows of the task in buffer b -- exactly when
// level g + 1 is known, else the predicted superset when level g + 2 is (or g
// is the second deepest level); `blocking` waits for level g + 1.  Returns
// whether the copy was issued (a blocking call always issues, maybe nothing).
template <bool kOverlap>
__device__ bool st_stage_exp(const mtb_layout_t &L, uint8_t *ws, const StagedPlan &P, StagedShared &s, uint8_t *dyn,
                             int b, bool blocking) {
    StagedTask &d = s.desc[b];
    const int g = d.g, p = d.p;
    const int bp = L.bits_pitch[g], hl = L.height[g];
    const int y0 = d.band * P.band[g], y1 = min(hl, y0 + P.band[g]);
    int2 c;
    int lo = 0, hi = 0;
    if (st_known(L, ws, P, s, p, g + 1, blocking, &c)) {
        lo = y0 - 2 * c.y - 1;  // base_g = 2 s_(g+1)
        hi = y1 - 2 * c.y + 1;
    } else if (blocking) {
        d.ok = 0;  // the wait gave up: copy nothing, the task is skipped
    } else if (g + 2 >= L.levels) {
        lo = y0 - kStHalo;  // base_g = 2 s_(g+1), s_(g+1) in {-1, 0, 1}
        hi = y1 + kStHalo;
    } else if (st_known(L, ws, P, s, p, g + 2, false, &c)) {
        lo = y0 - 4 * c.y - kStHalo;  // base_g = 4 s_(g+2) + 2d
        hi = y1 - 4 * c.y + kStHalo;
    } else {
        return false;
    }
    if (!st_wait_plane<kOverlap>(ws, L, P, st_exposure(P, p), g)) d.ok = 0;
    int ne = 0;
    d.ea = st_copy_rows_tx(Planes::bits(ws, L, st_exposure(P, p), g), bp, hl, lo, hi,
                           dyn + b * kStBufBytes + st_exp_offset(y1 - y0, bp), smem_addr(&s.mbar[kMbFull + b]), &ne);
    d.ne = ne;
    return true;
}

// Producer (lane 0): task t goes into buffer b (free): its reference band, and
// its exposure rows if they are already known.
template <bool kOverlap>
__device__ bool st_stage(const mtb_layout_t &L, uint8_t *ws, const StagedPlan &P, StagedShared &s, uint8_t *dyn,
                         int b, int t) {
    StagedTask &d = s.desc[b];
    d.t = t;
    if (t >= P.total_tasks - 1) return true;  // the final task or none: nothing to copy
    st_decode(P, t, d.g, d.p, d.band);
    d.ok = 1;
    const int g = d.g;
    const int bp = L.bits_pitch[g], hl = L.height[g];
    const int y0 = d.band * P.band[g], y1 = min(hl, y0 + P.band[g]);
    if (!st_wait_plane<kOverlap>(ws, L, P, st_pair_ref(P, st_exposure(P, d.p)), g)) d.ok = 0;
    fence_proxy_shared();
    int nr = 0;
    st_copy_rows_tx(Planes::bits(ws, L, st_pair_ref(P, st_exposure(P, d.p)), g), bp, hl, y0, y1,
                    dyn + b * kStBufBytes, smem_addr(&s.mbar[kMbFull + b]), &nr);
    // the guard (ordered before the counting warps' reads by the arrival that hands the task over)
    *reinterpret_cast<uint4 *>(dyn + b * kStBufBytes + st_exp_offset(y1 - y0, bp) - kStGuard) = make_uint4(0, 0, 0, 0);
    return st_stage_exp<kOverlap>(L, ws, P, s, dyn, b, false);
}

// Producer (lane 0): hands buffer b's task to the counting warps once its base
// is known (waiting for it when `blocking`).  Returns whether it did.
template <bool kOverlap>
__device__ bool st_arm(const mtb_layout_t &L, uint8_t *ws, const StagedPlan &P, StagedShared &s, uint8_t *dyn, int b,
                       bool exp_staged, bool blocking) {
    StagedTask &d = s.desc[b];
    if (d.t < P.total_tasks - 1) {
        int2 c = make_int2(0, 0);
        if (blocking && !exp_staged && !st_known(L, ws, P, s, d.p, d.g + 1, false, &c) && d.g + 2 < L.levels) {
            // the predicted rows are copied while the level above completes
            // (level g + 2 completes first; its tasks, or the pair's cluster,
            // are held by running CTAs)
            if (st_known(L, ws, P, s, d.p, d.g + 2, true, &c)) exp_staged = st_stage_exp<kOverlap>(L, ws, P, s, dyn, b, false);
        }
        if (!st_known(L, ws, P, s, d.p, d.g + 1, blocking, &c)) {
            if (!blocking) return false;
            d.ok = 0;
        }
        if (!exp_staged) st_stage_exp<kOverlap>(L, ws, P, s, dyn, b, true);
        d.bx = 2 * c.x;
        d.by = 2 * c.y;
        if (d.ok && d.band == 0) {
            const int i = st_exposure(P, d.p);
            int32_t *s1 = Planes::shift(ws, L, i, d.g + 1);
            s1[0] = c.x;
            s1[1] = c.y;
            int32_t *b0 = Planes::base(ws, L, i, d.g);
            b0[0] = d.bx;
            b0[1] = d.by;
        }
    }
    mbar_arrive(smem_addr(&s.mbar[kMbFull + b]));
    return true;
}

// Final task (warp 0): waits for level 0 of every pair, then writes the
// outputs and the stream's last status (MTB_OK or the first error any wait
// left).
__device__ void st_final(const mtb_layout_t &L, uint8_t *ws, const StagedPlan &P) {
    const int lane = threadIdx.x & 31;
    int ok = 1;
    if (lane == 0) {
        for (int p = 0; p < P.pairs && ok; ++p)
            ok = wait_at_least(Ctr::done(ws, L, p, 0), st_target(P, 0), status_word(ws, L), P.timeout_ns);
        __threadfence();
        if (P.status_out) {
            const int st = ld_acquire(status_word(ws, L));
            *reinterpret_cast<volatile int32_t *>(P.status_out) = st != 0 ? st : (ok ? MTB_OK : MTB_ERR_TIMEOUT);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return;
    // level 0's shift of every exposure at once, one exposure a lane: the
    // choice its counts make (0 for the reference)
    for (int e = lane; e < L.n; e += 32) {
        int sx = 0, sy = 0;
        if (e != P.ref) {
            const int2 c = st_choice(ws, L, e, 0);
            sx = c.x;
            sy = c.y;
        }
        int32_t *s0 = Planes::shift(ws, L, e, 0);
        s0[0] = sx;
        s0[1] = sy;
        if (P.shifts_out && !P.chain) {
            P.shifts_out[2 * e] = sx;
            P.shifts_out[2 * e + 1] = sy;
        }
    }
    __syncwarp();  // the level-0 rows above are read back below
    // the per-level outputs, when asked for: the lanes split the (exposure,
    // level) items, so the reads of different items are in flight together
    if (P.level_shifts_out || P.level_errs_out) {
        const int items = L.n * L.levels;
        for (int it = lane; it < items; it += 32) {
            const int e = it / L.levels, l = it - e * L.levels;
            if (P.level_shifts_out) {
                const int32_t *sl = Planes::shift(ws, L, e, l);
                P.level_shifts_out[(size_t)it * 2] = __ldcg(sl);
                P.level_shifts_out[(size_t)it * 2 + 1] = __ldcg(sl + 1);
            }
            if (P.level_errs_out) {
                const uint32_t *el = Planes::errs(ws, L, e, l);
                uint32_t v[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) v[k] = __ldcg(el + k);
#pragma unroll
                for (int k = 0; k < 9; ++k) P.level_errs_out[(size_t)it * 9 + k] = v[k];
            }
        }
    }
    if (!P.chain || !P.shifts_out) return;
    // chain mode: the shift of exposure e is the sum of the pair shifts along
    // its chain to ref (the level-0 shift rows hold the pairs' own shifts)
    __syncwarp();
    for (int e = lane; e < L.n; e += 32) {
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

// Warp 0 in the grid phase.
template <bool kOverlap>
__device__ void st_producer(const mtb_layout_t &L, uint8_t *ws, const StagedPlan &P, StagedShared &s, uint8_t *dyn,
                            uint32_t &ph) {
    const int lane = threadIdx.x & 31;
    int32_t *head = Ctr::queue(ws, L);
    int32_t *status = status_word(ws, L);
    const int final_task = P.total_tasks - 1;
    for (int k = lane; k < kStCache; k += 32) s.cache_key[k] = -1;
    __syncwarp();
    // lane 0's view: whether buffer b's exposure copy is issued, whether b is
    // armed, how many times it was armed (its "full" phases), and whether any
    // task of this CTA failed (then it takes no more)
    bool exp_staged[2] = {false, false}, armed[2] = {false, false}, failed = false;
    int held[2] = {0, 0}, arms[2] = {0, 0};
    if (lane == 0) {
        for (int b = 0; b < 2; ++b) {
            held[b] = atomicAdd(head, 1);
            exp_staged[b] = st_stage<kOverlap>(L, ws, P, s, dyn, b, held[b]);
        }
        armed[0] = st_arm<kOverlap>(L, ws, P, s, dyn, 0, exp_staged[0], true);
        arms[0] = 1;
        failed = held[0] < final_task && !s.desc[0].ok;
    }
    int cur = 0;
    for (;;) {
        const int t = __shfl_sync(0xffffffffu, held[cur], 0);
        if (t >= final_task) {
            if (t == final_task) st_final(L, ws, P);
            break;  // the other buffer holds a later index: nothing is left
        }
        int next = 0;
        if (lane == 0) {
            next = atomicAdd(head, 1);  // its latency hides behind the wait below
            if (!armed[cur ^ 1]) {
                armed[cur ^ 1] = st_arm<kOverlap>(L, ws, P, s, dyn, cur ^ 1, exp_staged[cur ^ 1], false);
                arms[cur ^ 1] += armed[cur ^ 1] ? 1 : 0;
            }
            if (!armed[cur ^ 1] && !exp_staged[cur ^ 1] && held[cur ^ 1] < final_task)
                exp_staged[cur ^ 1] = st_stage_exp<kOverlap>(L, ws, P, s, dyn, cur ^ 1, false);
        }
        __syncwarp();
        // buffer cur is free once the publisher has taken its counts
        mbar_wait(s, kMbReleased + cur, ph, status, 2 * P.timeout_ns);
        if (lane == 0) {
            // the next task is handed over before this buffer is refilled: the
            // counting warps take the buffers in turn
            if (!armed[cur ^ 1]) {
                armed[cur ^ 1] = st_arm<kOverlap>(L, ws, P, s, dyn, cur ^ 1, exp_staged[cur ^ 1], true);
                arms[cur ^ 1] += 1;
            }
            failed = failed || (held[cur ^ 1] < final_task && !s.desc[cur ^ 1].ok);
            held[cur] = failed ? P.total_tasks : next;  // after a failure no new task is taken
            armed[cur] = false;
            exp_staged[cur] = st_stage<kOverlap>(L, ws, P, s, dyn, cur, held[cur]);
        }
        __syncwarp();
        cur ^= 1;
    }
    // drain: every copy this CTA issued lands before it exits (a buffer staged
    // but never handed over is handed over now; the other warps have stopped)
    if (lane == 0) {
        for (int b = 0; b < 2; ++b) {
            if (!armed[b]) {
                mbar_arrive(smem_addr(&s.mbar[kMbFull + b]));
                arms[b] += 1;
            }
            uint32_t phb = (uint32_t)((arms[b] - 1) & 1) << (kMbFull + b);
            mbar_wait(s, kMbFull + b, phb, status, P.timeout_ns);
        }
    }
}

// Warp 1 in the grid phase: publishes each task's counts.
__device__ void st_publisher(const mtb_layout_t &L, uint8_t *ws, const StagedPlan &P, StagedShared &s, uint32_t &ph) {
    const int lane = threadIdx.x & 31;
    int32_t *status = status_word(ws, L);
    for (int b = 0;; b ^= 1) {
        if (!mbar_wait(s, kMbFull + b, ph, status, 2 * P.timeout_ns)) break;
        const StagedTask d = s.desc[b];
        if (d.t >= P.total_tasks - 1) break;
        if (!mbar_wait(s, kMbCounted + b, ph, status, 2 * P.timeout_ns)) break;
        uint32_t sum = 0;
        if (lane < 9)
            for (int w = kStWarps - kStCountWarps; w < kStWarps; ++w) sum += s.part[b][w][lane];
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&s.mbar[kMbReleased + b]));
        if (d.ok) {
            if (lane < 9) {
                if (sum) atomicAdd(Planes::errs(ws, L, st_exposure(P, d.p), d.g) + lane, sum);
                __threadfence();
            }
            __syncwarp();
            if (lane == 0) atomicAdd(Ctr::done(ws, L, d.p, d.g), 1);
        }
    }
}

// Warps 2.. in the grid phase: count the task in each buffer in turn.
__device__ void st_counter(const mtb_layout_t &L, uint8_t *ws, const StagedPlan &P, StagedShared &s, uint8_t *dyn,
                           uint32_t &ph) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int me = (int)threadIdx.x - 32 * (kStWarps - kStCountWarps);
    int32_t *status = status_word(ws, L);
    for (int b = 0;; b ^= 1) {
        // the producer's blocking waits are bounded by timeout_ns; this one by twice that
        if (!mbar_wait(s, kMbFull + b, ph, status, 2 * P.timeout_ns)) break;
        const StagedTask d = s.desc[b];
        if (d.t >= P.total_tasks - 1) break;
        uint32_t cnt[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (d.ok) {
            const int bp = L.bits_pitch[d.g], hl = L.height[d.g];
            const int y0 = d.band * P.band[d.g], y1 = min(hl, y0 + P.band[d.g]);
            const uint2 *sref = reinterpret_cast<const uint2 *>(dyn + b * kStBufBytes);
            const uint2 *sexp = reinterpret_cast<const uint2 *>(dyn + b * kStBufBytes + st_exp_offset(y1 - y0, bp));
            st_count_staged(sref, sexp, y1 - y0, d.ea, d.ne, bp, (L.width[d.g] + 31) >> 5, y0, d.bx, d.by,
                            P.seg[d.g], me, kStCounters, cnt);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[k]);
            if (lane == 0) s.part[b][warp][k] = v;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&s.mbar[kMbCounted + b]));
    }
}

template <bool kOverlap>
__device__ void st_grid(const mtb_layout_t &L, uint8_t *ws, const StagedPlan &P, StagedShared &s, uint8_t *dyn,
                        uint32_t &ph) {
    if (threadIdx.x < 32) st_producer<kOverlap>(L, ws, P, s, dyn, ph);
    else if (threadIdx.x < 64) st_publisher(L, ws, P, s, ph);
    else st_counter(L, ws, P, s, dyn, ph);
}

}  // namespace
}  // namespace mtb
