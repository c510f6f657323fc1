"""The oracle against its pins (CPU only), and planted mistakes in copies of the
oracle that the pins must catch."""
import json
import os
import re
import shutil

import numpy as np
import pytest
import torch

import oracle
from paper_2007_06483_gb300 import synth

from . import oracle_pins as P

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def make_pair(seed, w, h, levels):
    """Reference exposure and a 2x brighter (gamma 2.2) one whose content is
    displaced by d; the shift that re-aligns it is -d."""
    rng = np.random.default_rng([seed, 99])
    R = (1 << levels) - 1
    d = rng.integers(-R + 1, R, 2)
    s = synth.scene(seed, w, h)
    ref = synth.expose(s, 1.0, 2.2)
    moved = synth.expose(synth.displace(s, int(d[0]), int(d[1])), 2.0, 2.2)
    return ref.numpy(), moved.numpy(), (-int(d[0]), -int(d[1]))


ALL_PINS = [
    P.pin_gray_spot, P.pin_gray_bt601, P.pin_shrink, P.pin_histogram, P.pin_median, P.pin_bitmaps,
    P.pin_shift_error, P.pin_shift_symmetry, P.pin_candidate_order, P.pin_search_rule,
    lambda orc: P.pin_brute_force(orc, make_pair), P.pin_constant_and_identical,
    P.pin_apply_scipy, P.pin_chain, P.pin_quadrants,
]


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: getattr(f, "__name__", "brute_force"))
def test_pin(orc, pin):
    pin(orc)


def test_bt601_golden_fixture(orc):
    spots = []
    for line in open(os.path.join(GOLDEN, "bt601_spot.txt")):
        line = line.split("#")[0].strip()
        if line:
            spots.append(tuple(int(v) for v in line.split()))
    assert len(spots) >= 5
    P.pin_gray_spot(orc, spots)


def test_paper_facts(orc):
    """Numbers the paper prints: 6 levels x 9 tests = 54 shift tests (Sec. III-A),
    +-4 exclusion band (Sec. III-B), 5 images -> 4 pairwise alignments (Sec. III-B)."""
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    f = {x["name"]: x for x in facts}
    lv = f["pyramid_levels"]["value"]
    imgs = synth.make_stack(synth.small_spec(3, 128, 96, n=f["stack_images"]["value"], levels=lv, ref=2)).numpy()
    res = orc.align_stack(imgs, lv, f["exclusion_tolerance"]["value"], 2)
    per_pair = res["level_errs"].shape[1] * res["level_errs"].shape[2]
    assert per_pair == f["shift_tests_per_pair"]["value"] == 54
    aligned = [i for i in range(imgs.shape[0]) if i != 2]
    assert len(aligned) == f["pair_alignments"]["value"] == 4
    assert not res["level_errs"][2].any() and not res["shifts"][2].any()


def test_planted_shift_640(orc):
    spec = synth.PAIR_640
    res = orc.align_stack(synth.make_stack(spec).numpy(), spec.levels, spec.noise_tol, spec.ref)
    assert res["shifts"].tolist() == synth.expected_shifts(spec).tolist() == [[0, 0], [-7, 3]]


def test_planted_shifts_12mp(orc):
    spec = synth.STACK_12MP
    res = orc.align_stack(synth.make_stack(spec).numpy(), spec.levels, spec.noise_tol, spec.ref)
    assert res["shifts"].tolist() == synth.expected_shifts(spec).tolist()


def test_oracle_golden_regression(orc):
    """Values written by tests/golden/make_golden.py from the oracle alone."""
    g = json.load(open(os.path.join(GOLDEN, "pair640x480_oracle.json")))
    spec = synth.PAIR_640
    imgs = synth.make_stack(spec).numpy()
    import hashlib

    assert hashlib.sha256(imgs.tobytes()).hexdigest() == g["input_sha256"], "input generator drifted"
    res = orc.align_stack(imgs, spec.levels, spec.noise_tol, spec.ref)
    assert res["shifts"].tolist() == g["shifts"]
    assert res["level_errs"].tolist() == g["level_errs"]
    assert res["level_shifts"].tolist() == g["level_shifts"]
    for e in range(spec.n):
        assert orc.pyramid_maps(imgs[e], spec.levels, spec.noise_tol)["median"].tolist() == g["medians"][e]


def test_argument_rules(orc):
    assert orc.check_args(2, 64, 64, 7, 4, 0)
    assert not orc.check_args(2, 64, 64, 8, 4, 0)
    assert not orc.check_args(1, 64, 64, 3, 4, 0)
    assert not orc.check_args(2, 64, 64, 3, 256, 0)
    assert not orc.check_args(2, 64, 64, 3, 4, 2)
    with pytest.raises(ValueError):
        orc.align_stack(np.zeros((2, 8, 8, 3), np.uint8), 5, 4, 0)


# ---------------------------------------------------------------------------
# Planted mistakes: each is a plausible slip in the oracle; the pins must fail.
MUTATIONS = {
    "gray_channels_swapped": ("4899u * r + 9617u * g + 1868u * b", "1868u * r + 9617u * g + 4899u * b"),
    "gray_no_rounding": ("1868u * b + 8192u) >> 14", "1868u * b) >> 14"),
    "shrink_rounds_down": ("(a + b + c + d + 2) >> 2", "(a + b + c + d + 1) >> 2"),
    "shrink_drops_pixel": ("uint32_t b = src[(long)(2 * y) * w + 2 * x + 1];", "uint32_t b = src[(long)(2 * y) * w + 2 * x];"),
    "median_upper": ("uint64_t half = (n + 1) / 2;", "uint64_t half = n / 2 + 1;"),
    "tb_ge": ("tb[p] = (uint8_t)(v > median);", "tb[p] = (uint8_t)(v >= median);"),
    "eb_inverted": ("eb[p] = (uint8_t)(v < median - tol || v > median + tol);",
                    "eb[p] = (uint8_t)(v >= median - tol && v <= median + tol);"),
    "eb_band_edge": ("eb[p] = (uint8_t)(v < median - tol || v > median + tol);",
                     "eb[p] = (uint8_t)(v <= median - tol || v >= median + tol);"),
    "error_drops_eb_i": ("& eb_r[pr] & eb_i[pi]);", "& eb_r[pr]);"),
    "error_shift_sign": ("int xi = x - sx;", "int xi = x + sx;"),
    "error_moves_ref": ("(tb_r[pr] ^ tb_i[pi]) & eb_r[pr] & eb_i[pi]", "(tb_r[pi] ^ tb_i[pr]) & eb_r[pi] & eb_i[pr]"),
    "error_xy_swapped": ("int yi = y - sy;", "int yi = y - sx;"),
    "search_no_doubling": ("bx = 2 * best[2 * l + 0];", "bx = best[2 * l + 0];"),
    "search_last_minimum": ("if (e[k] < e[kbest]) kbest = k;", "if (e[k] <= e[kbest]) kbest = k;"),
    "candidate_order": ("{0, -1, 0, 1, -1, 1, -1, 0, 1}", "{0, 1, 0, -1, -1, 1, -1, 0, 1}"),
    "apply_sign": ("long long xs = (long long)x - shifts[2 * e + 0];", "long long xs = (long long)x + shifts[2 * e + 0];"),
    "apply_no_fill": ("if (!inside && fill == 0) {", "if (!inside && fill == 2) {"),
    "chain_wrong_neighbour": ("int nb = i < ref ? i + 1 : i - 1;", "int nb = i < ref ? i - 1 : i + 1;"),
    "chain_composition_sign": ("shifts[2 * i + 0] = pair[2 * i + 0] + shifts[2 * (i + 1) + 0];",
                               "shifts[2 * i + 0] = pair[2 * i + 0] - shifts[2 * (i + 1) + 0];"),
    "quadrant_origin_swapped": ("const int x0 = (q & 1) * wq, y0 = (q >> 1) * hq;", "const int x0 = (q >> 1) * wq, y0 = (q & 1) * hq;"),
    "quadrant_flag_threshold": ("if (hi - lo > rot_tol) flag = 1;", "if (hi - lo >= rot_tol) flag = 1;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    mutated = tmp_path / "mtb_oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.build(force=True, src=str(mutated), out=str(tmp_path / "libmut.so"))
    orc = oracle.Oracle(lib)
    caught = []
    for pin in ALL_PINS:
        try:
            pin(orc)
        except AssertionError:
            caught.append(getattr(pin, "__name__", "brute_force"))
    assert caught, f"planted mistake {name} passed every pin"
