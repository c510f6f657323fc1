"""Pins of the oracle: checks against what the paper and the mathematics fix,
never against a retyped copy of the oracle's own code.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError when the
oracle departs from the fixed fact.  ``test_oracle_pins.py`` runs them on the
real oracle and on copies with planted mistakes (each mistake must trip at
least one pin).

Independent routes used here:
  * closed forms: gray(v, v, v) = v; BT.601 luma within its Q14 rounding bound
    over all 2^24 colours; the mean of a constant block is the constant
  * library routines: numpy bincount (histogram), numpy sort (lower median),
    float64 block means (2x2 shrink)
  * the candidate error as a correlation: for bits a, b, [a != b] = a + b - 2ab,
    so E(s) = corr(eb_r tb_r, eb_i) + corr(eb_r, eb_i tb_i) - 2 corr(eb_r tb_r,
    eb_i tb_i), computed with scipy's 2-D convolution over every shift
  * brute force: the global minimum of that error surface over the whole search
    window, on small images with a planted shift
  * the paper's own numbers (tests/golden/paper_facts.json)
"""
from __future__ import annotations

import numpy as np
from scipy.signal import convolve2d

# Candidate order of one level: (0,0), then dy outer / dx inner over -1, 0, +1.
CANDIDATE_ORDER = ((0, 0), (-1, -1), (0, -1), (1, -1), (-1, 0), (1, 0), (-1, 1), (0, 1), (1, 1))


def error_surface(tb_r, eb_r, tb_i, eb_i) -> np.ndarray:
    """E[sy + h - 1, sx + w - 1] for every shift (sx, sy) with |sx| < w, |sy| < h."""
    A = (tb_r & eb_r).astype(np.int64)
    C = eb_r.astype(np.int64)
    B = eb_i.astype(np.int64)
    D = (tb_i & eb_i).astype(np.int64)

    def corr(F, G):  # sum_x F(x) G(x - s)
        return convolve2d(F, G[::-1, ::-1], mode="full")

    return corr(A, B) + corr(C, D) - 2 * corr(A, D)


def surface_at(E, h, w, sx, sy) -> int:
    if abs(sx) >= w or abs(sy) >= h:
        return 0
    return int(E[sy + h - 1, sx + w - 1])


def random_maps(rng, h, w, p=0.5):
    tb = (rng.random((h, w)) < p).astype(np.uint8)
    eb = (rng.random((h, w)) < 0.7).astype(np.uint8)
    return tb, eb


# --------------------------------------------------------------------------- gray
BT601_SPOT = ((255, 0, 0, 76), (0, 255, 0, 150), (0, 0, 255, 29), (255, 255, 255, 255), (0, 0, 0, 0),
              (128, 128, 128, 128), (255, 255, 0, 226), (0, 255, 255, 179), (255, 0, 255, 105))


def pin_gray_spot(orc, spots=BT601_SPOT):
    rgb = np.array([s[:3] for s in spots], np.uint8)
    got = orc.gray(rgb).tolist()
    assert got == [s[3] for s in spots], got
    v = np.arange(256, dtype=np.uint8)
    assert np.array_equal(orc.gray(np.stack([v, v, v], -1)), v), "gray(v,v,v) != v"


def pin_gray_bt601(orc):
    """All 2^24 colours within 0.5 + (Q14 weight error) * 255 of float BT.601."""
    c = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(c >> 16) & 255, (c >> 8) & 255, c & 255], -1).astype(np.uint8)
    g = orc.gray(rgb).astype(np.float64)
    y = 0.299 * rgb[:, 0] + 0.587 * rgb[:, 1] + 0.114 * rgb[:, 2]
    bound = 0.5 + 255 * (abs(4899 / 16384 - 0.299) + abs(9617 / 16384 - 0.587) + abs(1868 / 16384 - 0.114))
    assert np.abs(g - y).max() <= bound + 1e-9, np.abs(g - y).max()
    # away from the rounding boundary the result is the nearest integer
    far = np.abs((y - np.floor(y)) - 0.5) > 0.02
    assert np.array_equal(g[far], np.floor(y[far] + 0.5))


# --------------------------------------------------------------------------- shrink
def float_shrink(g):
    h2, w2 = g.shape[0] // 2, g.shape[1] // 2
    blocks = g[:2 * h2, :2 * w2].astype(np.float64).reshape(h2, 2, w2, 2)
    return np.floor(blocks.mean(axis=(1, 3)) + 0.5).astype(np.uint8)


def pin_shrink(orc, seed=0):
    rng = np.random.default_rng(seed)
    for h, w in ((1, 1), (2, 2), (3, 5), (17, 31), (64, 48), (101, 67)):
        g = rng.integers(0, 256, (h, w), dtype=np.uint8)
        out = orc.shrink(g)
        assert out.shape == (h // 2, w // 2)
        assert np.array_equal(out, float_shrink(g)), (h, w)
    for v in (0, 1, 77, 254, 255):
        assert (orc.shrink(np.full((9, 12), v, np.uint8)) == v).all()
    small = rng.integers(0, 256, (7, 9), dtype=np.uint8)
    assert np.array_equal(orc.shrink(np.repeat(np.repeat(small, 2, 0), 2, 1)), small)


# --------------------------------------------------------------------------- histogram / median
def pin_histogram(orc, seed=1):
    rng = np.random.default_rng(seed)
    for n in (1, 2, 255, 1000, 4097):
        g = rng.integers(0, 256, n, dtype=np.uint8)
        h = orc.histogram(g)
        assert np.array_equal(h, np.bincount(g, minlength=256))
        assert int(h.sum()) == n


def pin_median(orc, seed=2):
    rng = np.random.default_rng(seed)
    cases = [rng.integers(0, 256, n, dtype=np.uint8) for n in (1, 2, 3, 4, 10, 11, 1000, 1001)]
    cases += [np.array([0, 255], np.uint8), np.array([5, 5, 9, 9], np.uint8), np.full(6, 200, np.uint8)]
    cases += [np.minimum(rng.geometric(0.05, 999), 255).astype(np.uint8)]
    for g in cases:
        m = orc.median(np.bincount(g, minlength=256))
        n = g.size
        assert m == int(np.sort(g)[(n + 1) // 2 - 1]), (g[:8], m)
        assert (g < m).sum() < (n + 1) // 2 <= (g <= m).sum()
        if n % 2 == 1:
            assert m == int(np.median(g))


# --------------------------------------------------------------------------- bitmaps
def pin_bitmaps(orc, seed=3):
    rng = np.random.default_rng(seed)
    g = rng.integers(0, 256, (40, 33), dtype=np.uint8)
    hist = np.bincount(g.ravel(), minlength=256)
    cum = np.cumsum(hist)
    for m in (0, 37, 128, 254, 255):
        for tol in (0, 1, 4, 10, 255):
            tb, eb = orc.bitmaps(g, m, tol)
            assert set(np.unique(tb)) <= {0, 1} and set(np.unique(eb)) <= {0, 1}
            assert int(tb.sum()) == g.size - int(cum[m]), "tb must count pixels above the median"
            band = hist[max(0, m - tol):min(255, m + tol) + 1].sum()
            assert int(eb.sum()) == g.size - int(band), "eb must drop pixels within +-tol"
            if tol == 255:
                assert not eb.any()
            if tol == 0:
                assert np.array_equal(eb, (g != m).astype(np.uint8))
            assert not (tb[g <= m]).any()


# --------------------------------------------------------------------------- candidate error
def pin_shift_error(orc, seed=4):
    rng = np.random.default_rng(seed)
    for h, w in ((5, 7), (12, 9), (16, 20)):
        tb_r, eb_r = random_maps(rng, h, w)
        tb_i, eb_i = random_maps(rng, h, w)
        E = error_surface(tb_r, eb_r, tb_i, eb_i)
        for sy in range(-h - 1, h + 2):
            for sx in range(-w - 1, w + 2):
                got = orc.shift_error(tb_r, eb_r, tb_i, eb_i, sx, sy)
                assert got == surface_at(E, h, w, sx, sy), (h, w, sx, sy)


def pin_shift_symmetry(orc, seed=5):
    rng = np.random.default_rng(seed)
    tb_r, eb_r = random_maps(rng, 14, 11)
    tb_i, eb_i = random_maps(rng, 14, 11)
    for sx, sy in ((0, 0), (1, 0), (0, 2), (-3, 1), (4, -4)):
        a = orc.shift_error(tb_r, eb_r, tb_i, eb_i, sx, sy)
        b = orc.shift_error(tb_i, eb_i, tb_r, eb_r, -sx, -sy)
        assert a == b
    assert orc.shift_error(tb_r, eb_r, tb_r, eb_r, 0, 0) == 0


# --------------------------------------------------------------------------- search
def pin_candidate_order(orc):
    assert orc.candidates() == CANDIDATE_ORDER


def _random_pyramid(rng, h, w, levels):
    out = []
    for l in range(levels):
        out.append(random_maps(rng, h >> l, w >> l))
    return [m[0] for m in out], [m[1] for m in out]


def pin_search_rule(orc, seed=6):
    """Every level tests base + the 9 candidates, base = 2 * (best of the level
    below), the deepest base is (0,0), and the first minimum in candidate order
    wins -- checked with error values from the correlation surfaces."""
    rng = np.random.default_rng(seed)
    ties = 0
    for trial in range(60):
        levels = int(rng.integers(1, 5))
        h = int(rng.integers(1 << (levels - 1), 24))
        w = int(rng.integers(1 << (levels - 1), 24))
        tr, er = _random_pyramid(rng, h, w, levels)
        ti, ei = _random_pyramid(rng, h, w, levels)
        errs, best = orc.search_pair(tr, er, ti, ei)
        bx = by = 0
        for l in range(levels - 1, -1, -1):
            hl, wl = h >> l, w >> l
            E = error_surface(tr[l], er[l], ti[l], ei[l])
            want = [surface_at(E, hl, wl, bx + dx, by + dy) for dx, dy in CANDIDATE_ORDER]
            assert errs[l].tolist() == want, (trial, l)
            k = int(np.argmin(want))  # numpy's argmin returns the first minimum
            ties += want.count(want[k]) > 1
            assert tuple(best[l]) == (bx + CANDIDATE_ORDER[k][0], by + CANDIDATE_ORDER[k][1]), (trial, l)
            bx, by = 2 * int(best[l][0]), 2 * int(best[l][1])
    assert ties > 5, "the trials must exercise ties"


def pin_brute_force(orc, make_pair):
    """On small stacks with a planted shift and a clear optimum, the pyramid's
    answer equals the global minimum of the full-resolution error surface over
    the whole reachable window +-(2^L - 1)."""
    for seed, w, h, levels, tol in ((1, 96, 80, 4, 4), (2, 120, 90, 4, 4), (3, 64, 64, 3, 4), (4, 160, 100, 5, 4)):
        rgb_r, rgb_i, expect = make_pair(seed, w, h, levels)
        r = orc.pyramid_maps(rgb_r, levels, tol)
        i = orc.pyramid_maps(rgb_i, levels, tol)
        E = error_surface(r["tb"][0], r["eb"][0], i["tb"][0], i["eb"][0])
        R = (1 << levels) - 1
        win = E[h - 1 - R:h + R, w - 1 - R:w + R]
        assert (win == win.min()).sum() == 1, "brute-force optimum must be unique"
        sy, sx = np.unravel_index(int(np.argmin(win)), win.shape)
        brute = (int(sx) - R, int(sy) - R)
        assert brute == tuple(expect)
        _, best = orc.search_pair(r["tb"], r["eb"], i["tb"], i["eb"])
        assert tuple(best[0]) == brute, (seed, tuple(best[0]), brute)


def pin_constant_and_identical(orc, seed=7):
    rng = np.random.default_rng(seed)
    const = np.full((2, 40, 52, 3), 90, np.uint8)
    res = orc.align_stack(const, 4, 4, 0)
    assert not res["shifts"].any() and not res["level_errs"].any() and not res["level_shifts"].any()
    img = rng.integers(0, 256, (1, 40, 52, 3), dtype=np.uint8)
    same = np.concatenate([img, img, img])
    res = orc.align_stack(same, 4, 4, 1)
    assert not res["shifts"].any() and not res["level_shifts"].any()
    assert not res["level_errs"][:, :, 0].any()


# ---- after the alignment, and the other readings of "pairwise" --------------
def pin_apply_scipy(orc, seed=8):
    """Moving the RGB by an integer shift is a nearest-order translation:
    scipy's ndimage.shift with mode 'constant' (fill 0) / 'nearest' (edge)
    computes the same image."""
    from scipy import ndimage

    rng = np.random.default_rng(seed)
    for h, w in ((7, 9), (16, 5), (1, 1), (33, 40)):
        n = 3
        img = rng.integers(0, 256, (n, h, w, 3), dtype=np.uint8)
        xs = [0, 1, -1, w - 1, -(w - 1), w, -w, w + 3, 1000, -5]
        ys = [0, 1, -1, h, -h - 2, 3]
        for fill, mode in ((0, "constant"), (1, "nearest")):
            sh = np.array([[rng.choice(xs), rng.choice(ys)] for _ in range(n)], np.int32)
            out = orc.apply_shifts(img, sh, fill)
            for e in range(n):
                want = ndimage.shift(img[e], (int(sh[e, 1]), int(sh[e, 0]), 0), order=0, mode=mode, cval=0)
                assert np.array_equal(out[e], want), (h, w, fill, sh[e].tolist())


def _stack(seed, w, h, n, levels, ref, shift_range):
    from paper_2007_06483_gb300 import synth

    spec = synth.small_spec(seed, w, h, n=n, levels=levels, shift_range=shift_range, ref=ref)
    return synth.make_stack(spec).numpy(), synth.expected_shifts(spec)


def pin_chain(orc, seed=9):
    """Chain mode: with two exposures it is the direct pair; the composed shift
    of each exposure minus its neighbour's is that pair's own level-0 shift;
    planted shifts are recovered through the chain."""
    imgs, _ = _stack(seed, 96, 80, 2, 4, 1, 5)
    a, b = orc.align_stack(imgs, 4, 4, 1), orc.align_stack_chain(imgs, 4, 4, 1)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    imgs, want = _stack(seed + 3, 160, 120, 5, 5, 2, 6)  # every planted component is non-zero
    assert all((want[i] != 0).all() for i in (0, 1, 3, 4))
    res = orc.align_stack_chain(imgs, 5, 4, 2)
    sh, lsh = res["shifts"], res["level_shifts"]
    assert not sh[2].any() and not lsh[2].any()
    for i in range(5):
        if i != 2:
            nb = i + 1 if i < 2 else i - 1
            assert np.array_equal(sh[i] - sh[nb], lsh[i, 0]), i
    assert np.array_equal(sh, want), (sh.tolist(), want.tolist())


def _rotate_nearest(img, deg):
    """[h, w, 3] image turned by deg about its centre (nearest source pixel,
    edge replicated): test input only."""
    h, w = img.shape[:2]
    t = np.deg2rad(deg)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    xs = np.cos(t) * (xx - cx) + np.sin(t) * (yy - cy) + cx
    ys = -np.sin(t) * (xx - cx) + np.cos(t) * (yy - cy) + cy
    xi = np.clip(np.rint(xs), 0, w - 1).astype(np.int64)
    yi = np.clip(np.rint(ys), 0, h - 1).astype(np.int64)
    return img[yi, xi]


def pin_quadrants(orc, seed=10):
    """Per-quadrant alignment: quadrant q equals the whole-stack oracle on the
    numpy-cropped quadrant; a pure translation moves all four quadrants alike
    (no flag); a rotation moves opposite quadrants in opposite directions
    (flagged)."""
    imgs, want = _stack(seed, 258, 194, 3, 4, 1, 4)
    res = orc.align_quadrants(imgs, 4, 4, 1, 1)
    hq, wq = 194 // 2, 258 // 2
    for q in range(4):
        y0, x0 = (q >> 1) * hq, (q & 1) * wq
        crop = np.ascontiguousarray(imgs[:, y0:y0 + hq, x0:x0 + wq])
        assert np.array_equal(res["quad_shifts"][:, q], orc.align_stack(crop, 4, 4, 1)["shifts"]), q
    for q in range(4):
        assert np.array_equal(res["quad_shifts"][:, q], want), (q, res["quad_shifts"].tolist())
    assert not res["flags"].any()
    base, _ = _stack(seed + 1, 256, 192, 1, 4, 0, 0)
    rot = np.stack([base[0], _rotate_nearest(base[0], 3.0)])
    r = orc.align_quadrants(rot, 4, 4, 0, 1)
    tl, tr, bl, br = (r["quad_shifts"][1, q] for q in range(4))
    assert r["flags"][1] == 1 and r["flags"][0] == 0, r
    # a turn about the centre moves each quadrant along the perpendicular of its
    # offset from the centre: opposite corners move in opposite directions, the
    # top two alike in x and oppositely in y (signs only: the estimates are coarse)
    sg = [np.sign(v.astype(np.int64)) for v in (tl, tr, bl, br)]
    assert all(v.all() for v in sg), r
    assert (sg[0] == -sg[3]).all() and (sg[1] == -sg[2]).all(), r
    assert sg[0][0] == sg[1][0] and sg[0][1] == -sg[1][1], r
    # the flag is "spread > rot_tol": off at rot_tol = spread, on just below it
    q = r["quad_shifts"][1]
    spread = int((q.max(axis=0) - q.min(axis=0)).max())
    assert orc.align_quadrants(rot, 4, 4, 0, spread)["flags"][1] == 0
    assert orc.align_quadrants(rot, 4, 4, 0, spread - 1)["flags"][1] == 1
