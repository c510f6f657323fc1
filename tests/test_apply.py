"""Moving the RGB exposures by their shifts (mtb_apply_shifts): the kernel must
equal the oracle byte for byte, for every shape, shift and fill mode."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2007_06483_gb300 import synth


def test_apply_rejects_invalid_arguments_on_host(mtb_lib):
    lib = mtb_lib.lib()
    a, b, s = 1 << 20, 1 << 30, 1 << 24  # never dereferenced: the checks come first
    assert lib.mtb_apply_shifts(a, 2, 8, 8, s, 2, b, None) == mtb_lib.MTB_ERR_INVALID_ARG    # fill
    assert lib.mtb_apply_shifts(a, 0, 8, 8, s, 0, b, None) == mtb_lib.MTB_ERR_INVALID_ARG    # no exposure
    assert lib.mtb_apply_shifts(a, 2, 0, 8, s, 0, b, None) == mtb_lib.MTB_ERR_INVALID_ARG    # width
    assert lib.mtb_apply_shifts(a, 2, 65536, 8, s, 0, b, None) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_apply_shifts(a + 1, 2, 8, 8, s, 0, b, None) == mtb_lib.MTB_ERR_INVALID_ARG  # alignment
    assert lib.mtb_apply_shifts(a, 2, 8, 8, s, 0, b + 8, None) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_apply_shifts(a, 2, 8, 8, s + 2, 0, b, None) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_apply_shifts(a, 2, 8, 8, s, 0, a + 256, None) == mtb_lib.MTB_ERR_INVALID_ARG  # overlap
    assert lib.mtb_apply_shifts(None, 2, 8, 8, s, 0, b, None) == mtb_lib.MTB_ERR_INVALID_ARG


SHAPES = [(1, 1, 1), (2, 5, 3), (3, 7, 9), (2, 16, 16), (3, 37, 23), (2, 257, 33), (4, 640, 480), (2, 1001, 77),
          (2, 65535, 2)]


@pytest.mark.gpu
@pytest.mark.parametrize("n,w,h", SHAPES)
@pytest.mark.parametrize("fill", [0, 1])
def test_apply_matches_oracle(mtb_lib, oracle_mod, n, w, h, fill):
    rng = np.random.default_rng(w * 7 + h + fill)
    img = rng.integers(0, 256, (n, h, w, 3), dtype=np.uint8)
    xs = [0, 1, -1, 2, -3, 5, -17, w - 1, -w, w + 2, 2**31 - 1, -2**31]
    ys = [0, 1, -1, 3, -2, h, -h - 1, 2**31 - 1]
    for trial in range(3):
        sh = np.array([[rng.choice(xs), rng.choice(ys)] for _ in range(n)], np.int32)
        d_img = torch.from_numpy(img).cuda()
        out = torch.full_like(d_img, 0xAB)
        mtb_lib.apply_shifts(d_img, torch.from_numpy(sh).cuda(), fill, out=out)
        torch.cuda.synchronize()
        want = oracle_mod.apply_shifts(img, sh, fill)
        assert np.array_equal(out.cpu().numpy(), want), (n, w, h, fill, sh.tolist())


@pytest.mark.gpu
def test_apply_after_alignment_restores_the_scene(mtb_lib, oracle_mod):
    """The alignment's own shifts, read on the device: the moved exposures equal
    the oracle's, and where a planted displacement is undone the content matches
    the reference scene displaced by nothing (interior, edge fill)."""
    spec = synth.small_spec(41, 800, 600, n=4, levels=6, shift_range=20, ref=1)
    imgs = synth.make_stack(spec, "cuda")
    shifts = mtb_lib.align_stack(imgs, spec.levels, spec.noise_tol, spec.ref)
    out = mtb_lib.apply_shifts(imgs, shifts, mtb_lib.MTB_FILL_EDGE)
    torch.cuda.synchronize()
    want = oracle_mod.apply_shifts(imgs.cpu().numpy(), shifts.cpu().numpy(), 1)
    assert np.array_equal(out.cpu().numpy(), want)
    assert np.array_equal(shifts.cpu().numpy(), synth.expected_shifts(spec))


@pytest.mark.gpu
def test_apply_full_size_stack(mtb_lib, oracle_mod):
    """The 6000x4000x7 stack moved by random shifts within its search range."""
    spec = synth.STACK_24MP
    imgs = synth.make_stack(spec, "cuda")
    rng = np.random.default_rng(5)
    sh = rng.integers(-120, 121, (spec.n, 2)).astype(np.int32)
    for fill in (0, 1):
        out = mtb_lib.apply_shifts(imgs, torch.from_numpy(sh).cuda(), fill)
        torch.cuda.synchronize()
        want = oracle_mod.apply_shifts(imgs.cpu().numpy(), sh, fill)
        assert np.array_equal(out.cpu().numpy(), want), fill


@pytest.mark.gpu
def test_apply_binding_rejects_bad_out(mtb_lib):
    d = torch.zeros((2, 8, 16, 3), dtype=torch.uint8, device="cuda")
    sh = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError, match="overlap"):
        mtb_lib.apply_shifts(d, sh, 0, out=d)
    with pytest.raises(ValueError, match="shaped like"):
        mtb_lib.apply_shifts(d, sh, 0, out=torch.zeros((2, 8, 15, 3), dtype=torch.uint8, device="cuda"))
