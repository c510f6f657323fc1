// mtb_device.cuh -- device helpers shared by the kernels of the library.
#pragma once

#include "mtb_internal.cuh"

namespace mtb {

// Lower median (smallest v with cumulative count >= ceil(N/2)) of a 256-bin
// histogram in global memory (read through L2) or shared memory; called by all
// 32 lanes of one warp, returns the median to all of them.
template <bool kL2>
__device__ __forceinline__ int warp_median(const uint32_t *hist) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t c[8];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        c[k] = kL2 ? __ldcg(hist + lane * 8 + k) : hist[lane * 8 + k];
        s += c[k];
    }
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(full, inc, o);
        if (lane >= o) inc += t;
    }
    const uint32_t total = __shfl_sync(full, inc, 31);
    const uint32_t half = total / 2 + (total & 1u);  // ceil(total / 2)
    const uint32_t before = inc - s;
    const unsigned owner_mask = __ballot_sync(full, half > before && half <= inc);
    if (owner_mask == 0) return 0;
    const int owner = __ffs(owner_mask) - 1;
    int m = 0;
    if (lane == owner) {
        uint32_t cum = before;
        m = lane * 8 + 7;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            cum += c[k];
            if (cum >= half) {
                m = lane * 8 + k;
                break;
            }
        }
    }
    return __shfl_sync(full, m, owner);
}

// Programmatic dependent launch.  A kernel launched with
// cudaLaunchAttributeProgrammaticStreamSerialization may start while the
// previous kernel of the stream still runs; pdl_wait() blocks until that kernel
// has finished and its writes are visible (a no-op without the attribute), and
// pdl_trigger() lets the next kernel start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__host__ __device__ __forceinline__ int32_t *counters(uint8_t *ws, const mtb_layout_t &L) {
    return reinterpret_cast<int32_t *>(ws + L.counter_offset);
}

// The counter area of a stack (int32, layout counter_offset):
//   tiles[e]          pyramid tiles of exposure e finished
//   pyr_ready[e]      1 once exposure e's pyramid, histograms and medians are done
//   bit_done[e][l]    bitmap chunks of exposure e, level l finished
//   queue             work-queue head of a search or engine launch
//   done[p][l]        search chunks of pair p, level l finished
//   window[p]         window items of pair p finished
// The pyramid stage clears everything up to bit_done; the search stage the rest.
struct Ctr {
    static __device__ __forceinline__ int32_t *tiles(uint8_t *ws, const mtb_layout_t &L, int e) {
        return counters(ws, L) + e;
    }
    static __device__ __forceinline__ int32_t *pyr_ready(uint8_t *ws, const mtb_layout_t &L, int e) {
        return counters(ws, L) + L.n + e;
    }
    static __device__ __forceinline__ int32_t *bit_done(uint8_t *ws, const mtb_layout_t &L, int e, int l) {
        return counters(ws, L) + 2 * L.n + e * L.levels + l;
    }
    static __device__ __forceinline__ int32_t *queue(uint8_t *ws, const mtb_layout_t &L) {
        return counters(ws, L) + 2 * L.n + L.n * L.levels;
    }
    static __host__ __forceinline__ int32_t *queue_host(uint8_t *ws, const mtb_layout_t &L) {
        return counters(ws, L) + 2 * L.n + L.n * L.levels;
    }
    static __device__ __forceinline__ int32_t *done(uint8_t *ws, const mtb_layout_t &L, int p, int l) {
        return counters(ws, L) + 2 * L.n + L.n * L.levels + 8 + p * L.levels + l;
    }
    static __device__ __forceinline__ int32_t *window(uint8_t *ws, const mtb_layout_t &L, int p) {
        return counters(ws, L) + 2 * L.n + 2 * L.n * L.levels + 8 + p;
    }
};
// int32 words of the counter area cleared by the pyramid and by the search stage
// (together 3n + 2 n levels + 8, within the n (2 levels + 4) + 16 of the layout)
__host__ __device__ __forceinline__ int pyramid_counter_words(const mtb_layout_t &L) { return 2 * L.n + L.n * L.levels; }
__host__ __device__ __forceinline__ int search_counter_words(const mtb_layout_t &L) { return 8 + L.n * L.levels + L.n; }

// Bitmap chunks of tile level l of one exposure, and the value of bit_done[e][l]
// once level l of an exposure is complete (deep levels are built whole).
// (chunk_words: words per bitmap chunk, bit_chunk_words(L) for the stage kernel)
__host__ __device__ __forceinline__ int bitmap_chunks(const mtb_layout_t &L, int l, int chunk_words) {
    return (L.bits_pitch[l] * L.height[l] + chunk_words - 1) / chunk_words;
}
__host__ __device__ __forceinline__ int bitmap_target(const mtb_layout_t &L, int l, int chunk_words) {
    return l < L.tile_levels ? bitmap_chunks(L, l, chunk_words) : 1;
}

// Adds 1 to a completion counter after this CTA's writes: every thread fences
// its own writes, the CTA synchronises, then one thread adds.
__device__ __forceinline__ void cta_signal(int32_t *ctr, int add = 1) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(ctr, add);
}

// Weak global load that may be served from L1.  Unlike ld.global.nc it stays
// correct for data another CTA of the same launch wrote before a completion
// counter that this CTA acquired.
__device__ __forceinline__ uint2 ld_weak(const uint2 *p) {
    uint2 v;
    asm volatile("ld.global.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

__device__ __forceinline__ int32_t *status_word(uint8_t *ws, const mtb_layout_t &L) {
    return reinterpret_cast<int32_t *>(ws + L.status_offset);
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Spins (thread-level) until *ctr >= target.  Gives up when *status is already
// set by another wait, or after timeout_ns, in which case it sets *status to
// MTB_ERR_TIMEOUT.  Returns true if the target was reached.  The sleep between
// polls grows from 32 ns to kWaitMaxSleepNs: the search's level-to-level hops
// are a few microseconds, and a longer ceiling (1 us) made each waiter notice
// its dependency up to that much late (4000x3000x3 one-call step: 90.0 us with
// 1024 ns, 86.2 us with 64 ns).
constexpr unsigned kWaitMaxSleepNs = 64;
__device__ __forceinline__ bool wait_at_least(const int32_t *ctr, int target, int32_t *status,
                                              unsigned long long timeout_ns) {
    if (ld_acquire(ctr) >= target) return true;
    const unsigned long long deadline = global_timer_ns() + timeout_ns;
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < kWaitMaxSleepNs) ns <<= 1;
        if (ld_acquire(ctr) >= target) return true;
        if (ld_acquire(status) != 0) return false;
        if (global_timer_ns() > deadline) {
            atomicCAS(status, 0, MTB_ERR_TIMEOUT);
            return false;
        }
    }
}

}  // namespace mtb
