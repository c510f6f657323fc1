// mtb_quadrants.cu -- Ward's rotation test, which the paper's Sec. II recalls:
// each exposure is split into four quadrants, every quadrant stack is aligned
// on its own, and an exposure whose quadrants move differently is flagged.
//
// Quadrant q = 2 * qy + qx (top-left, top-right, bottom-left, bottom-right) is
// the floor(w/2) x floor(h/2) block at (qx * floor(w/2), qy * floor(h/2)).
// k_gather_quadrants copies the four quadrant stacks into contiguous buffers
// (the alignment kernels read whole rows of pitch 3 * w); each is then aligned
// by the one-call path; k_quadrant_flags writes [n][4][2] and the flags.
#include "mtb_internal.cuh"

namespace mtb {
namespace {

constexpr int kGatherThreads = 256;

// Warp v copies rows v, v + warps, ... of the 4 * n * hq quadrant rows; the
// lanes copy 4 bytes at a time (byte loads: the rows start at any byte).
__global__ void __launch_bounds__(kGatherThreads)
k_gather_quadrants(const uint8_t *__restrict__ in, int n, int w, int h, uint8_t *__restrict__ out,
                   long long quad_stride) {
    const int wq = w / 2, hq = h / 2;
    const long long rows = 4ll * n * hq;
    const long long warps = (long long)gridDim.x * (kGatherThreads / 32);
    const int row_bytes = 3 * wq;
    for (long long r = (long long)blockIdx.x * (kGatherThreads / 32) + (threadIdx.x >> 5); r < rows; r += warps) {
        const int q = (int)(r / ((long long)n * hq));
        const long long rem = r - (long long)q * n * hq;
        const int e = (int)(rem / hq), y = (int)(rem - (long long)e * hq);
        const int x0 = (q & 1) * wq, y0 = (q >> 1) * hq;
        const uint8_t *src = in + (((long long)e * h + y0 + y) * w + x0) * 3;
        uint8_t *dst = out + q * quad_stride + ((long long)e * hq + y) * row_bytes;
        for (int c = (threadIdx.x & 31) * 4; c < row_bytes; c += 128) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (c + j < row_bytes) dst[c + j] = __ldcs(src + c + j);
        }
    }
}

// quad[q][e] (the four alignments' outputs) -> out[e][q]; flag = the spread of
// the four shifts in x or in y exceeds rot_tol.
__global__ void k_quadrant_flags(const int32_t *__restrict__ quad, int n, int rot_tol, int32_t *__restrict__ out,
                                 int32_t *__restrict__ flags) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        int lo[2] = {0, 0}, hi[2] = {0, 0};
        for (int q = 0; q < 4; ++q) {
            for (int c = 0; c < 2; ++c) {
                const int v = quad[((size_t)q * n + e) * 2 + c];
                out[((size_t)e * 4 + q) * 2 + c] = v;
                lo[c] = q == 0 || v < lo[c] ? v : lo[c];
                hi[c] = q == 0 || v > hi[c] ? v : hi[c];
            }
        }
        if (flags) flags[e] = (hi[0] - lo[0] > rot_tol || hi[1] - lo[1] > rot_tol) ? 1 : 0;
    }
}

}  // namespace

cudaError_t launch_gather_quadrants(const uint8_t *images, int n, int w, int h, uint8_t *out, long long quad_stride,
                                    cudaStream_t s) {
    const long long warps = (4ll * n * (h / 2) + kGatherThreads / 32 - 1) / (kGatherThreads / 32);
    const long long cap = 8ll * device_sm_count();
    const int grid = (int)(warps < cap ? warps : cap);
    return launch_k(k_gather_quadrants, dim3(grid), dim3(kGatherThreads), s, false, images, n, w, h, out,
                    quad_stride);
}

cudaError_t launch_quadrant_flags(const int32_t *quad, int n, int rot_tol, int32_t *out, int32_t *flags,
                                  cudaStream_t s) {
    const int grid = (n + 255) / 256;
    return launch_k(k_quadrant_flags, dim3(grid), dim3(256), s, false, quad, n, rot_tol, out, flags);
}

}  // namespace mtb
