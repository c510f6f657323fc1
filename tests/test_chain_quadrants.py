"""Consecutive-chain alignment and the per-quadrant rotation test: the CUDA
path must equal the oracle bit for bit (shifts, per-level errors and shifts,
quadrant shifts, flags)."""
import numpy as np
import pytest
import torch

from paper_2007_06483_gb300 import synth

from .oracle_pins import _rotate_nearest


def test_quadrants_reject_invalid_arguments_on_host(mtb_lib):
    lib = mtb_lib.lib()
    a, b = 1 << 20, 1 << 24  # never dereferenced: the checks come first
    E = mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_align_quadrants(a, 2, 1, 64, 2, 4, 0, 1, b, None, None, 0, None) == E   # w < 2
    assert lib.mtb_align_quadrants(a, 2, 64, 64, 2, 4, 0, -1, b, None, None, 0, None) == E  # rot_tol
    assert lib.mtb_align_quadrants(a, 2, 64, 64, 7, 4, 0, 1, b, None, None, 0, None) == E   # 32 >> 6 == 0
    assert lib.mtb_align_quadrants(a, 2, 64, 64, 3, 4, 2, 1, b, None, None, 0, None) == E   # ref
    assert lib.mtb_quadrant_workspace_bytes(2, 64, 64, 7) == 0
    assert lib.mtb_quadrant_workspace_bytes(2, 64, 64, 3) > 0
    assert lib.mtb_align_stack_chain(a + 1, 2, 64, 64, 3, 4, 0, b, None, None, None, 0, None) == E


CHAIN = [(96, 80, 2, 4, 1), (160, 120, 5, 5, 2), (333, 222, 4, 5, 0), (640, 480, 6, 6, 5), (1001, 333, 7, 4, 3),
         (37, 23, 3, 3, 1)]


@pytest.mark.gpu
@pytest.mark.parametrize("w,h,n,levels,ref", CHAIN)
def test_chain_matches_oracle(search_kernel, mtb_lib, oracle_mod, w, h, n, levels, ref):
    spec = synth.small_spec(900 + w, w, h, n=n, levels=levels, shift_range=min(6, (1 << levels) - 1), ref=ref)
    imgs = synth.make_stack(spec, "cuda")
    shifts, errs, lsh = mtb_lib.align_stack_chain(imgs, levels, 4, ref, level_outputs=True)
    torch.cuda.synchronize()
    want = oracle_mod.align_stack_chain(imgs.cpu().numpy(), levels, 4, ref)
    assert np.array_equal(errs.cpu().numpy().view(np.uint32), want["level_errs"])
    assert np.array_equal(lsh.cpu().numpy(), want["level_shifts"])
    assert np.array_equal(shifts.cpu().numpy(), want["shifts"])
    if n == 2:  # the chain of two exposures is the direct pair
        assert torch.equal(shifts, mtb_lib.align_stack(imgs, levels, 4, ref))


@pytest.mark.gpu
def test_chain_full_size(search_kernel, mtb_lib, oracle_mod):
    spec = synth.STACK_12MP
    imgs = synth.make_stack(spec, "cuda")
    shifts = mtb_lib.align_stack_chain(imgs, spec.levels, spec.noise_tol, spec.ref)
    torch.cuda.synchronize()
    want = oracle_mod.align_stack_chain(imgs.cpu().numpy(), spec.levels, spec.noise_tol, spec.ref)
    assert np.array_equal(shifts.cpu().numpy(), want["shifts"])
    assert np.array_equal(shifts.cpu().numpy(), synth.expected_shifts(spec))


QUADS = [(258, 194, 3, 4, 1), (160, 120, 4, 4, 2), (641, 479, 2, 5, 0), (1000, 700, 3, 6, 1), (5, 7, 2, 1, 0)]


@pytest.mark.gpu
@pytest.mark.parametrize("w,h,n,levels,ref", QUADS)
def test_quadrants_match_oracle(mtb_lib, oracle_mod, w, h, n, levels, ref):
    spec = synth.small_spec(700 + w, w, h, n=n, levels=levels + 1, shift_range=min(5, (1 << levels) - 1), ref=ref)
    imgs = synth.make_stack(spec, "cuda")
    for rot_tol in (0, 1, 3):
        qs, flags = mtb_lib.align_quadrants(imgs, levels, 4, ref, rot_tol)
        torch.cuda.synchronize()
        want = oracle_mod.align_quadrants(imgs.cpu().numpy(), levels, 4, ref, rot_tol)
        assert np.array_equal(qs.cpu().numpy(), want["quad_shifts"]), rot_tol
        assert np.array_equal(flags.cpu().numpy(), want["flags"]), rot_tol


@pytest.mark.gpu
def test_quadrants_flag_a_rotation(mtb_lib, oracle_mod):
    base = synth.make_stack(synth.small_spec(11, 512, 384, n=1, levels=5, shift_range=0), "cpu").numpy()[0]
    stack = np.stack([base, _rotate_nearest(base, 2.0), _rotate_nearest(base, -4.0)])
    imgs = torch.from_numpy(stack).cuda()
    qs, flags = mtb_lib.align_quadrants(imgs, 5, 4, 0, 1)
    torch.cuda.synchronize()
    want = oracle_mod.align_quadrants(stack, 5, 4, 0, 1)
    assert np.array_equal(qs.cpu().numpy(), want["quad_shifts"])
    assert np.array_equal(flags.cpu().numpy(), want["flags"])
    assert flags.cpu().tolist() == [0, 1, 1]
