// mtb_search.cu -- coarse-to-fine shift search.
//
// Sec. III-A: starting at the deepest level with offset (0,0), the 9 candidates
// offset + (dx, dy), dx, dy in {-1, 0, +1}, are tested; the best is doubled and
// the next finer level searched around it.  Sec. III-B: the error of a
// candidate is the number of pixels set in
//     (tb_ref XOR S(tb_i)) AND eb_ref AND S(eb_i),
// S = move by the candidate with 0 outside the image.
//
// One launch per level covers every pair of the stack.  A thread owns one
// 32-pixel word column of the reference and walks down a band of rows; the
// moved words of exposure i come from funnel shifts of three neighbouring
// words, computed once per i-row for the 3 x offsets and kept for the 3 rows
// (y offsets) that use them.  Every candidate is then XOR, AND, AND, popc.
// Counts are summed per warp with __reduce_add_sync and per CTA in shared
// memory, then added to the level's 9 counters with one atomic each.
// The argmin of level l+1 is taken by every CTA of level l (9 values), so no
// host round trip or extra launch sits between levels.
#include "mtb_internal.cuh"

namespace mtb {
namespace {

// Moved (tb, eb) words of one exposure-i row for x offsets dx = +1, 0, -1
// (index j = 1 - dx).
struct Moved {
    uint32_t t[3], e[3];
};

// Words q, q+1, q+2 of row yi, 0 outside the plane; j-th result is the 32 bits
// starting at bit o + j of word q.
__device__ __forceinline__ Moved moved_row(const uint2 *__restrict__ plane, int bp, int hl, int yi, int q, int o) {
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

__global__ void __launch_bounds__(kMaxShiftThreads)
k_shift(const mtb_layout_t L, uint8_t *__restrict__ ws, int l, int ref, int rows_per_cta) {
    const int p = blockIdx.z;
    const int i = p < ref ? p : p + 1;
    const int hl = L.height[l], bp = L.bits_pitch[l];
    const bool lead = blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0;

    // Offset this level starts from: twice the best shift of level l+1.
    int bx = 0, by = 0;
    if (l + 1 < L.levels) {
        const uint32_t *e1 = Planes::errs(ws, L, i, l + 1);
        int kb = 0;
        uint32_t best = e1[0];
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            const uint32_t v = e1[k];
            if (v < best) {
                best = v;
                kb = k;
            }
        }
        const int32_t *b1 = Planes::base(ws, L, i, l + 1);
        const int sx = b1[0] + cand_dx(kb), sy = b1[1] + cand_dy(kb);
        bx = 2 * sx;
        by = 2 * sy;
        if (lead) {
            int32_t *s1 = Planes::shift(ws, L, i, l + 1);
            s1[0] = sx;
            s1[1] = sy;
        }
    }
    if (lead) {
        int32_t *b0 = Planes::base(ws, L, i, l);
        b0[0] = bx;
        b0[1] = by;
    }

    const uint2 *pr = Planes::bits(ws, L, ref, l);
    const uint2 *pi = Planes::bits(ws, L, i, l);
    const int w = blockIdx.x * blockDim.x + threadIdx.x;  // reference word column
    // Bits of exposure i that land on word w for dx = +1 start at 32w - bx - 1.
    const int t = -bx - 1;
    const int q = w + (t >> 5);
    const int o = t & 31;
    const int y0 = blockIdx.y * rows_per_cta;
    const int y1 = min(hl, y0 + rows_per_cta);

    uint32_t cnt[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) cnt[k] = 0;
    // rows of exposure i used by reference row y: y - by - dy
    Moved rm = moved_row(pi, bp, hl, y0 - by - 1, q, o);  // dy = +1
    Moved r0 = moved_row(pi, bp, hl, y0 - by, q, o);      // dy = 0
    for (int y = y0; y < y1; ++y) {
        const Moved rp = moved_row(pi, bp, hl, y - by + 1, q, o);  // dy = -1
        uint2 r = make_uint2(0u, 0u);
        if (w < bp) r = __ldg(pr + (size_t)y * bp + w);
        // candidate order: (0,0), (-1,-1), (0,-1), (1,-1), (-1,0), (1,0), (-1,1), (0,1), (1,1)
        cnt[0] += cand_err(r, r0, 1);
        cnt[1] += cand_err(r, rp, 2);
        cnt[2] += cand_err(r, rp, 1);
        cnt[3] += cand_err(r, rp, 0);
        cnt[4] += cand_err(r, r0, 2);
        cnt[5] += cand_err(r, r0, 0);
        cnt[6] += cand_err(r, rm, 2);
        cnt[7] += cand_err(r, rm, 1);
        cnt[8] += cand_err(r, rm, 0);
        rm = r0;
        r0 = rp;
    }

    __shared__ uint32_t s_red[kMaxShiftThreads / 32][9];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[k]);
        if (lane == 0) s_red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        uint32_t sum = 0;
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) sum += s_red[wi][threadIdx.x];
        if (sum) atomicAdd(Planes::errs(ws, L, i, l) + threadIdx.x, sum);
    }
}

// Level 0's argmin gives the final shift; copies the per-level outputs.
__global__ void k_finalize(const mtb_layout_t L, uint8_t *__restrict__ ws, int ref, int32_t *shifts_out,
                           uint32_t *level_errs_out, int32_t *level_shifts_out) {
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
        int sx = 0, sy = 0;
        if (i != ref) {
            const uint32_t *e0 = Planes::errs(ws, L, i, 0);
            int kb = 0;
            uint32_t best = e0[0];
            for (int k = 1; k < 9; ++k)
                if (e0[k] < best) {
                    best = e0[k];
                    kb = k;
                }
            const int32_t *b0 = Planes::base(ws, L, i, 0);
            sx = b0[0] + cand_dx(kb);
            sy = b0[1] + cand_dy(kb);
        } else {
            for (int l = 0; l < L.levels; ++l) {
                int32_t *sl = Planes::shift(ws, L, i, l);
                int32_t *bl = Planes::base(ws, L, i, l);
                sl[0] = sl[1] = bl[0] = bl[1] = 0;
            }
        }
        int32_t *s0 = Planes::shift(ws, L, i, 0);
        s0[0] = sx;
        s0[1] = sy;
        if (shifts_out) {
            shifts_out[2 * i] = sx;
            shifts_out[2 * i + 1] = sy;
        }
        for (int l = 0; l < L.levels; ++l) {
            if (level_shifts_out) {
                const int32_t *sl = Planes::shift(ws, L, i, l);
                level_shifts_out[((size_t)i * L.levels + l) * 2] = sl[0];
                level_shifts_out[((size_t)i * L.levels + l) * 2 + 1] = sl[1];
            }
            if (level_errs_out) {
                const uint32_t *el = Planes::errs(ws, L, i, l);
                for (int k = 0; k < 9; ++k) level_errs_out[((size_t)i * L.levels + l) * 9 + k] = el[k];
            }
        }
    }
}

}  // namespace

cudaError_t launch_search(const mtb_layout_t &L, int ref_idx, uint8_t *ws, int32_t *shifts_out,
                          uint32_t *level_errs_out, int32_t *level_shifts_out, cudaStream_t s) {
    const int pairs = L.n - 1;
    const int target_ctas = 4 * device_sm_count();
    for (int l = L.levels - 1; l >= 0; --l) {
        const int bp = L.bits_pitch[l], hl = L.height[l];
        const int threads = bp >= kMaxShiftThreads ? kMaxShiftThreads : ((bp + 31) / 32) * 32;
        const int col_blocks = (bp + threads - 1) / threads;
        long long rows = ((long long)hl * col_blocks * pairs + target_ctas - 1) / target_ctas;
        rows = rows < 4 ? 4 : (rows > 64 ? 64 : rows);
        const int row_blocks = (int)((hl + rows - 1) / rows);
        if (pairs > 65535) return cudaErrorInvalidValue;
        dim3 grid(col_blocks, row_blocks, pairs);
        k_shift<<<grid, threads, 0, s>>>(L, ws, l, ref_idx, (int)rows);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    const int fin_threads = L.n >= 256 ? 256 : ((L.n + 31) / 32) * 32;
    k_finalize<<<1, fin_threads, 0, s>>>(L, ws, ref_idx, shifts_out, level_errs_out, level_shifts_out);
    return cudaGetLastError();
}

}  // namespace mtb
