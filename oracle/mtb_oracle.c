/*
 * mtb_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, single-threaded CPU statement of Ward-style median threshold
 * bitmap (MTB) translational alignment as described in Alpay, Aydemir & Temizel,
 * "Accelerating Translational Image Registration for HDR Images on GPU"
 * (arXiv 2007.06483), Sec. III-A and Sec. III-B.  Every map is one byte per
 * pixel holding 0 or 1 (Sec. III-B keeps byte-maps instead of bit-packed
 * bitmaps; the counts are the same either way).
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * call this file.  It shares no code, header, table or helper with the CUDA
 * library, and the CUDA library never calls it.
 *
 * Points the paper leaves unstated, each fixed once here (integer arithmetic):
 *   gray      g = (4899 R + 9617 G + 1868 B + 8192) >> 14   (ITU-R BT.601 luma
 *             weights 0.299/0.587/0.114 in Q14, rounded to nearest)
 *   shrink    2x2 box mean rounded half up, (a+b+c+d+2) >> 2; an odd last row or
 *             column is dropped, so level l is floor(W/2^l) x floor(H/2^l)
 *   levels    counts every image of the pyramid, full resolution included
 *   median    lower median: the smallest v whose cumulative count reaches
 *             ceil(N/2), taken per pyramid level from that level's histogram
 *   bitmaps   tb = [g > m]; eb = [g < m - tol or g > m + tol]
 *   shift     the second image's maps are moved by (sx, sy):
 *             S(b)(x, y) = b(x - sx, y - sy), and 0 outside the image
 *   tie-break candidates in the order (0,0), then (dx,dy) row by row with dy
 *             outer and dx inner, each in -1, 0, +1; the first minimum wins
 *   pairs     every exposure i != ref is aligned directly to exposure ref
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Search candidates of one pyramid level (Sec. III-A: +-1 pixel tests in both
 * directions, 9 per level).  Index k is also the error-array index. */
static const int CAND_DX[9] = {0, -1, 0, 1, -1, 1, -1, 0, 1};
static const int CAND_DY[9] = {0, -1, -1, -1, 0, 0, 1, 1, 1};

int orc_candidate(int k, int *dx, int *dy)
{
    if (k < 0 || k > 8) return -1;
    *dx = CAND_DX[k];
    *dy = CAND_DY[k];
    return 0;
}

/* Sec. III-A: the exposures are first converted to gray-scale. */
void orc_gray(const uint8_t *rgb, long npix, uint8_t *gray)
{
    for (long p = 0; p < npix; ++p) {
        uint32_t r = rgb[3 * p + 0];
        uint32_t g = rgb[3 * p + 1];
        uint32_t b = rgb[3 * p + 2];
        gray[p] = (uint8_t)((4899u * r + 9617u * g + 1868u * b + 8192u) >> 14);
    }
}

/* Sec. III-A: the pyramid is made by halving both dimensions, level by level
 * (Sec. III-B: iterated down-sampling of the previous level). */
void orc_shrink(const uint8_t *src, int w, int h, uint8_t *dst)
{
    int w2 = w / 2, h2 = h / 2;
    for (int y = 0; y < h2; ++y) {
        for (int x = 0; x < w2; ++x) {
            uint32_t a = src[(long)(2 * y) * w + 2 * x];
            uint32_t b = src[(long)(2 * y) * w + 2 * x + 1];
            uint32_t c = src[(long)(2 * y + 1) * w + 2 * x];
            uint32_t d = src[(long)(2 * y + 1) * w + 2 * x + 1];
            dst[(long)y * w2 + x] = (uint8_t)((a + b + c + d + 2) >> 2);
        }
    }
}

/* Sec. III-B: a 256-bin histogram of every gray image in the pyramid. */
void orc_histogram(const uint8_t *g, long npix, uint32_t *hist)
{
    for (int v = 0; v < 256; ++v) hist[v] = 0;
    for (long p = 0; p < npix; ++p) hist[g[p]] += 1;
}

/* Sec. III-A: the median pixel value, found from the histogram. */
int orc_median(const uint32_t *hist)
{
    uint64_t n = 0;
    for (int v = 0; v < 256; ++v) n += hist[v];
    if (n == 0) return -1;
    uint64_t half = (n + 1) / 2; /* ceil(n / 2) */
    uint64_t cum = 0;
    for (int v = 0; v < 256; ++v) {
        cum += hist[v];
        if (cum >= half) return v;
    }
    return 255;
}

/* Sec. III-A: pixels <= median become 0 in the MTB, the others 1.
 * Sec. III-B: the exclusion bitmap drops pixels within +-tol of the median. */
void orc_bitmaps(const uint8_t *g, long npix, int median, int tol, uint8_t *tb, uint8_t *eb)
{
    for (long p = 0; p < npix; ++p) {
        int v = g[p];
        tb[p] = (uint8_t)(v > median);
        eb[p] = (uint8_t)(v < median - tol || v > median + tol);
    }
}

/* Sec. III-A / III-B: error of one shift candidate.  XOR the reference MTB with
 * the shifted MTB of the second image, AND both exclusion bitmaps onto it, and
 * count the pixels left set.  The shifted maps are 0 outside the image. */
uint32_t orc_shift_error(const uint8_t *tb_r, const uint8_t *eb_r,
                         const uint8_t *tb_i, const uint8_t *eb_i,
                         int w, int h, int sx, int sy)
{
    uint32_t count = 0;
    for (int y = 0; y < h; ++y) {
        int yi = y - sy;
        if (yi < 0 || yi >= h) continue;
        for (int x = 0; x < w; ++x) {
            int xi = x - sx;
            if (xi < 0 || xi >= w) continue;
            long pr = (long)y * w + x;
            long pi = (long)yi * w + xi;
            uint8_t err = (uint8_t)((tb_r[pr] ^ tb_i[pi]) & eb_r[pr] & eb_i[pi]);
            count += err;
        }
    }
    return count;
}

/* Size of pyramid level l: floor(W / 2^l) x floor(H / 2^l). */
static void level_dims(int w, int h, int l, int *wl, int *hl)
{
    *wl = w >> l;
    *hl = h >> l;
}

/* Offset of level l inside a concatenation of levels 0..levels-1. */
long orc_level_offset(int w, int h, int l)
{
    long off = 0;
    for (int k = 0; k < l; ++k) {
        int wk, hk;
        level_dims(w, h, k, &wk, &hk);
        off += (long)wk * hk;
    }
    return off;
}

/* Sec. III-A: coarse-to-fine search.  Start at the deepest level with offset
 * (0,0), test the 9 candidates offset + (dx,dy), keep the best, double it and
 * move one level finer.  tb/eb hold every level, concatenated (level 0 first).
 * errs[l][k] and best[l] = the chosen shift at level l. */
void orc_search_pair(const uint8_t *tb_r, const uint8_t *eb_r,
                     const uint8_t *tb_i, const uint8_t *eb_i,
                     int w, int h, int levels, uint32_t *errs, int32_t *best)
{
    int bx = 0, by = 0;
    for (int l = levels - 1; l >= 0; --l) {
        int wl, hl;
        level_dims(w, h, l, &wl, &hl);
        long off = orc_level_offset(w, h, l);
        uint32_t *e = errs + (long)l * 9;
        int kbest = 0;
        for (int k = 0; k < 9; ++k) {
            e[k] = orc_shift_error(tb_r + off, eb_r + off, tb_i + off, eb_i + off,
                                   wl, hl, bx + CAND_DX[k], by + CAND_DY[k]);
            if (e[k] < e[kbest]) kbest = k;
        }
        best[2 * l + 0] = bx + CAND_DX[kbest];
        best[2 * l + 1] = by + CAND_DY[kbest];
        bx = 2 * best[2 * l + 0];
        by = 2 * best[2 * l + 1];
    }
}

/* Gray pyramid, histograms, medians and both maps of one exposure, every level
 * concatenated (level 0 first).  gray/tb/eb: orc_level_offset(w,h,levels) bytes;
 * hist: levels*256; medians: levels. */
void orc_exposure_maps(const uint8_t *rgb, int w, int h, int levels, int tol,
                       uint8_t *gray, uint32_t *hist, int32_t *medians,
                       uint8_t *tb, uint8_t *eb)
{
    orc_gray(rgb, (long)w * h, gray);
    for (int l = 0; l < levels; ++l) {
        int wl, hl;
        level_dims(w, h, l, &wl, &hl);
        long off = orc_level_offset(w, h, l);
        if (l > 0) {
            int wp, hp;
            level_dims(w, h, l - 1, &wp, &hp);
            orc_shrink(gray + orc_level_offset(w, h, l - 1), wp, hp, gray + off);
        }
        orc_histogram(gray + off, (long)wl * hl, hist + 256L * l);
        medians[l] = orc_median(hist + 256L * l);
        orc_bitmaps(gray + off, (long)wl * hl, medians[l], tol, tb + off, eb + off);
    }
}

/* Argument rules shared by the stack entry point. */
int orc_check_args(int n, int w, int h, int levels, int tol, int ref)
{
    if (n < 2 || w < 1 || h < 1 || levels < 1 || levels > 30) return -1;
    if ((w >> (levels - 1)) < 1 || (h >> (levels - 1)) < 1) return -1;
    if (tol < 0 || tol > 255) return -1;
    if (ref < 0 || ref >= n) return -1;
    return 0;
}

/* Sec. III-B: the stack is aligned pairwise, n exposures giving n-1 pair
 * alignments, each exposure's pyramid built once.  Every exposure i != ref is
 * searched against ref.  shifts: [n][2] (sx, sy) to apply to exposure i;
 * level_errs [n][levels][9] and level_shifts [n][levels][2] may be NULL; rows of
 * ref are zero.  Returns 0, -1 for invalid arguments, -2 if memory runs out. */
int orc_align_stack(const uint8_t *images, int n, int w, int h, int levels, int tol,
                    int ref, int32_t *shifts, uint32_t *level_errs, int32_t *level_shifts)
{
    if (orc_check_args(n, w, h, levels, tol, ref) != 0) return -1;
    long total = orc_level_offset(w, h, levels);
    long npix0 = (long)w * h;
    uint8_t *gray = malloc((size_t)total);
    uint32_t *hist = malloc(sizeof(uint32_t) * 256 * (size_t)levels);
    int32_t *med = malloc(sizeof(int32_t) * (size_t)levels);
    uint8_t *tb = malloc((size_t)total * n);
    uint8_t *eb = malloc((size_t)total * n);
    uint32_t *errs = malloc(sizeof(uint32_t) * 9 * (size_t)levels);
    int32_t *best = malloc(sizeof(int32_t) * 2 * (size_t)levels);
    int rc = 0;
    if (!gray || !hist || !med || !tb || !eb || !errs || !best) {
        rc = -2;
        goto done;
    }
    for (int e = 0; e < n; ++e)
        orc_exposure_maps(images + (size_t)e * npix0 * 3, w, h, levels, tol, gray, hist, med,
                          tb + (size_t)e * total, eb + (size_t)e * total);
    for (int i = 0; i < n; ++i) {
        if (i == ref) {
            memset(errs, 0, sizeof(uint32_t) * 9 * (size_t)levels);
            memset(best, 0, sizeof(int32_t) * 2 * (size_t)levels);
        } else {
            orc_search_pair(tb + (size_t)ref * total, eb + (size_t)ref * total,
                            tb + (size_t)i * total, eb + (size_t)i * total,
                            w, h, levels, errs, best);
        }
        shifts[2 * i + 0] = best[0];
        shifts[2 * i + 1] = best[1];
        if (level_errs) memcpy(level_errs + (size_t)i * levels * 9, errs, sizeof(uint32_t) * 9 * (size_t)levels);
        if (level_shifts) memcpy(level_shifts + (size_t)i * levels * 2, best, sizeof(int32_t) * 2 * (size_t)levels);
    }
done:
    free(gray);
    free(hist);
    free(med);
    free(tb);
    free(eb);
    free(errs);
    free(best);
    return rc;
}

/* ---- After the alignment, and the paper's other readings of "pairwise" ---- */

/* Moves each exposure's RGB by the shift the search found for it: the operator
 * S of the search (Sec. III-B moves the second image's maps), applied to the
 * image itself, out(x, y) = in(x - sx, y - sy) per channel.  A pixel whose
 * source lies outside the image gets 0 (fill 0) or the nearest edge pixel
 * (fill 1).  shifts: [n][2]; out: [n][h][w][3], not overlapping images. */
void orc_apply_shifts(const uint8_t *images, int n, int w, int h, const int32_t *shifts, int fill, uint8_t *out)
{
    for (int e = 0; e < n; ++e) {
        const uint8_t *src = images + (size_t)e * w * h * 3;
        uint8_t *dst = out + (size_t)e * w * h * 3;
        for (int y = 0; y < h; ++y) {
            for (int x = 0; x < w; ++x) {
                long long xs = (long long)x - shifts[2 * e + 0];
                long long ys = (long long)y - shifts[2 * e + 1];
                int inside = xs >= 0 && xs < w && ys >= 0 && ys < h;
                uint8_t *p = dst + ((size_t)y * w + x) * 3;
                if (!inside && fill == 0) {
                    p[0] = p[1] = p[2] = 0;
                    continue;
                }
                if (xs < 0) xs = 0;
                if (xs >= w) xs = w - 1;
                if (ys < 0) ys = 0;
                if (ys >= h) ys = h - 1;
                const uint8_t *q = src + ((size_t)ys * w + xs) * 3;
                p[0] = q[0];
                p[1] = q[1];
                p[2] = q[2];
            }
        }
    }
}

/* Consecutive-chain alignment.  Sec. II notes that each exposure can be
 * compared with its neighbours; Sec. III-B still takes n - 1 pair alignments.
 * Here exposure i != ref is searched against its neighbour towards ref
 * (i + 1 below ref, i - 1 above), and the translations add up along the chain:
 * shift[i] = pair shift of (neighbour, i) + shift[neighbour], shift[ref] = 0.
 * level_errs and level_shifts rows hold the pair (neighbour, i) values.  Same
 * arguments and return codes as orc_align_stack. */
int orc_align_stack_chain(const uint8_t *images, int n, int w, int h, int levels, int tol,
                          int ref, int32_t *shifts, uint32_t *level_errs, int32_t *level_shifts)
{
    if (orc_check_args(n, w, h, levels, tol, ref) != 0) return -1;
    long total = orc_level_offset(w, h, levels);
    long npix0 = (long)w * h;
    uint8_t *gray = malloc((size_t)total);
    uint32_t *hist = malloc(sizeof(uint32_t) * 256 * (size_t)levels);
    int32_t *med = malloc(sizeof(int32_t) * (size_t)levels);
    uint8_t *tb = malloc((size_t)total * n);
    uint8_t *eb = malloc((size_t)total * n);
    uint32_t *errs = malloc(sizeof(uint32_t) * 9 * (size_t)levels);
    int32_t *best = malloc(sizeof(int32_t) * 2 * (size_t)levels);
    int32_t *pair = malloc(sizeof(int32_t) * 2 * (size_t)n);
    int rc = 0;
    if (!gray || !hist || !med || !tb || !eb || !errs || !best || !pair) {
        rc = -2;
        goto done;
    }
    for (int e = 0; e < n; ++e)
        orc_exposure_maps(images + (size_t)e * npix0 * 3, w, h, levels, tol, gray, hist, med,
                          tb + (size_t)e * total, eb + (size_t)e * total);
    for (int i = 0; i < n; ++i) {
        if (i == ref) {
            memset(errs, 0, sizeof(uint32_t) * 9 * (size_t)levels);
            memset(best, 0, sizeof(int32_t) * 2 * (size_t)levels);
        } else {
            int nb = i < ref ? i + 1 : i - 1;
            orc_search_pair(tb + (size_t)nb * total, eb + (size_t)nb * total,
                            tb + (size_t)i * total, eb + (size_t)i * total,
                            w, h, levels, errs, best);
        }
        pair[2 * i + 0] = best[0];
        pair[2 * i + 1] = best[1];
        if (level_errs) memcpy(level_errs + (size_t)i * levels * 9, errs, sizeof(uint32_t) * 9 * (size_t)levels);
        if (level_shifts) memcpy(level_shifts + (size_t)i * levels * 2, best, sizeof(int32_t) * 2 * (size_t)levels);
    }
    shifts[2 * ref + 0] = 0;
    shifts[2 * ref + 1] = 0;
    for (int i = ref - 1; i >= 0; --i) {
        shifts[2 * i + 0] = pair[2 * i + 0] + shifts[2 * (i + 1) + 0];
        shifts[2 * i + 1] = pair[2 * i + 1] + shifts[2 * (i + 1) + 1];
    }
    for (int i = ref + 1; i < n; ++i) {
        shifts[2 * i + 0] = pair[2 * i + 0] + shifts[2 * (i - 1) + 0];
        shifts[2 * i + 1] = pair[2 * i + 1] + shifts[2 * (i - 1) + 1];
    }
done:
    free(gray);
    free(hist);
    free(med);
    free(tb);
    free(eb);
    free(errs);
    free(best);
    free(pair);
    return rc;
}

/* Ward's test for a rotation between exposures, which the paper's Sec. II
 * recalls: split every exposure into four quadrants and align each quadrant
 * stack on its own.  Quadrant q = 2 * qy + qx (top-left, top-right,
 * bottom-left, bottom-right) is the floor(w/2) x floor(h/2) block at
 * (qx * floor(w/2), qy * floor(h/2)); each quadrant stack is aligned directly
 * to ref.  quad_shifts: [n][4][2].  flags[i] = 1 when the four quadrant
 * shifts of exposure i spread by more than rot_tol pixels in x or in y (a pure
 * translation moves every quadrant alike), else 0.  Returns as
 * orc_align_stack; -1 also when the quadrants are too small for `levels`. */
int orc_align_quadrants(const uint8_t *images, int n, int w, int h, int levels, int tol, int ref,
                        int rot_tol, int32_t *quad_shifts, int32_t *flags)
{
    const int wq = w / 2, hq = h / 2;
    if (orc_check_args(n, wq, hq, levels, tol, ref) != 0 || rot_tol < 0) return -1;
    uint8_t *sub = malloc((size_t)n * wq * hq * 3);
    int32_t *sh = malloc(sizeof(int32_t) * 2 * (size_t)n);
    int rc = 0;
    if (!sub || !sh) {
        rc = -2;
        goto done;
    }
    for (int q = 0; q < 4; ++q) {
        const int x0 = (q & 1) * wq, y0 = (q >> 1) * hq;
        for (int e = 0; e < n; ++e)
            for (int y = 0; y < hq; ++y)
                memcpy(sub + (((size_t)e * hq + y) * wq) * 3,
                       images + (((size_t)e * h + y0 + y) * w + x0) * 3, (size_t)wq * 3);
        rc = orc_align_stack(sub, n, wq, hq, levels, tol, ref, sh, NULL, NULL);
        if (rc != 0) goto done;
        for (int e = 0; e < n; ++e) {
            quad_shifts[(e * 4 + q) * 2 + 0] = sh[2 * e + 0];
            quad_shifts[(e * 4 + q) * 2 + 1] = sh[2 * e + 1];
        }
    }
    for (int e = 0; e < n; ++e) {
        int flag = 0;
        for (int c = 0; c < 2; ++c) {
            int lo = quad_shifts[(e * 4) * 2 + c], hi = lo;
            for (int q = 1; q < 4; ++q) {
                int v = quad_shifts[(e * 4 + q) * 2 + c];
                if (v < lo) lo = v;
                if (v > hi) hi = v;
            }
            if (hi - lo > rot_tol) flag = 1;
        }
        flags[e] = flag;
    }
done:
    free(sub);
    free(sh);
    return rc;
}
