"""CUDA path vs the oracle, bit-exact, through the C ABI (GPU only)."""
import numpy as np
import pytest
import torch

from paper_2007_06483_gb300 import synth

from ._parity import check_stack

pytestmark = pytest.mark.gpu


def _natural(seed, w, h, n, levels, ref=0, shift_range=5):
    spec = synth.small_spec(seed, w, h, n=n, levels=levels, shift_range=shift_range, ref=ref)
    return synth.make_stack(spec, "cuda")


# (w, h, levels, n, ref): tails in both directions, w < 32, w % 16 != 0, several
# 256 x 32 tiles with a ragged last tile, deep levels built by the bitmap pass,
# coarsest levels of 1 pixel.
SHAPES = [
    (1, 1, 1, 2, 0),
    (2, 2, 2, 2, 1),
    (31, 5, 2, 2, 0),
    (37, 23, 3, 3, 1),
    (64, 48, 4, 2, 0),
    (100, 75, 5, 3, 2),
    (257, 33, 6, 2, 1),
    (513, 97, 7, 3, 0),
    (600, 450, 8, 4, 2),
    (1000, 3, 2, 2, 0),
    (3, 1000, 2, 2, 1),
    (777, 555, 9, 5, 3),
    (1024, 1024, 11, 2, 0),
    # grid-level search launches: 2-D blocks, several word blocks, odd widths
    (1000, 700, 5, 3, 1),
    (1001, 333, 4, 2, 1),
    (4100, 300, 3, 2, 0),
    (9000, 100, 2, 3, 2),
    # widths that are a multiple of 16 (the tensor-copy pyramid): a 16-wide image
    # narrower than one copy box, ragged 32x32 tiles in x and y, deep levels
    (16, 16, 4, 2, 0),
    (48, 37, 5, 3, 1),
    (176, 1000, 7, 2, 0),
    (2064, 999, 8, 3, 2),
    (4000, 31, 5, 2, 1),
]


@pytest.mark.parametrize("w,h,levels,n,ref", SHAPES)
def test_shapes_natural(search_kernel, mtb_lib, oracle_mod, w, h, levels, n, ref):
    imgs = _natural(100 + w + 7 * h, w, h, n, levels, ref=ref, shift_range=min(5, (1 << levels) - 1))
    check_stack(mtb_lib, oracle_mod, imgs, levels, 4, ref)


@pytest.mark.parametrize("tol", [0, 1, 4, 17, 255])
def test_noise_tolerance(search_kernel, mtb_lib, oracle_mod, tol):
    imgs = _natural(7, 301, 211, 3, 5, ref=1)
    check_stack(mtb_lib, oracle_mod, imgs, 5, tol, 1)


@pytest.mark.parametrize("kind", ["zeros", "full", "constant", "uniform", "two-level", "stripes"])
def test_degenerate_content(search_kernel, mtb_lib, oracle_mod, kind):
    n, h, w, levels = 3, 130, 290, 5
    g = torch.Generator().manual_seed(5)
    if kind == "zeros":
        imgs = torch.zeros((n, h, w, 3), dtype=torch.uint8)
    elif kind == "full":
        imgs = torch.full((n, h, w, 3), 255, dtype=torch.uint8)
    elif kind == "constant":
        imgs = torch.full((n, h, w, 3), 97, dtype=torch.uint8)
    elif kind == "uniform":
        imgs = torch.randint(0, 256, (n, h, w, 3), generator=g, dtype=torch.uint8)
    elif kind == "two-level":
        imgs = (torch.randint(0, 2, (n, h, w, 1), generator=g, dtype=torch.uint8) * 255).expand(n, h, w, 3)
    else:
        x = torch.arange(w) // 3 % 2
        imgs = (x[None, None, :, None] * 200 + 20).expand(n, h, w, 3).to(torch.uint8)
    want = check_stack(mtb_lib, oracle_mod, imgs.contiguous().cuda(), levels, 4, 0)
    if kind in ("zeros", "full", "constant"):
        assert not want["shifts"].any()


def test_many_exposures(search_kernel, mtb_lib, oracle_mod):
    imgs = _natural(11, 200, 150, 9, 4, ref=4)
    check_stack(mtb_lib, oracle_mod, imgs, 4, 4, 4)


def test_widest_row(search_kernel, mtb_lib, oracle_mod):
    w, h = 65535, 3
    g = torch.Generator().manual_seed(3)
    imgs = torch.randint(0, 256, (2, h, w, 3), generator=g, dtype=torch.uint8).cuda()
    check_stack(mtb_lib, oracle_mod, imgs, 2, 4, 1)


@pytest.mark.parametrize("spec", synth.PLAIN_CONFIGS, ids=lambda s: s.name)
def test_config_parity(search_kernel, mtb_lib, oracle_mod, spec):
    imgs = synth.make_stack(spec, "cuda")
    want = check_stack(mtb_lib, oracle_mod, imgs, spec.levels, spec.noise_tol, spec.ref,
                       maps=spec.w * spec.h <= 12_000_000)
    exp = synth.expected_shifts(spec)
    ok = [bool((want["shifts"][i] == exp[i]).all()) for i in range(spec.n)]
    if spec is not synth.STACK_24MP:
        assert all(ok), (want["shifts"].tolist(), exp.tolist())


def test_one_call_matches_stages(search_kernel, mtb_lib, oracle_mod):
    spec = synth.small_spec(21, 640, 480, n=4, levels=6, shift_range=30, ref=2)
    imgs = synth.make_stack(spec, "cuda")
    shifts, errs, lsh = mtb_lib.align_stack(imgs, spec.levels, 4, spec.ref, level_outputs=True)
    plain = mtb_lib.align_stack(imgs, spec.levels, 4, spec.ref)
    host = mtb_lib.align_stack_host(imgs.cpu().pin_memory(), spec.levels, 4, spec.ref)  # pinned
    paged = mtb_lib.align_stack_host(imgs.cpu().contiguous(), spec.levels, 4, spec.ref)  # pageable
    torch.cuda.synchronize()
    want = oracle_mod.align_stack(imgs.cpu().numpy(), spec.levels, 4, spec.ref)
    assert np.array_equal(errs.cpu().numpy().view(np.uint32), want["level_errs"])
    assert np.array_equal(lsh.cpu().numpy(), want["level_shifts"])
    assert np.array_equal(shifts.cpu().numpy(), want["shifts"])
    assert np.array_equal(plain.cpu().numpy(), want["shifts"])
    assert np.array_equal(host.numpy(), want["shifts"])
    assert np.array_equal(paged.numpy(), want["shifts"])


def test_repeatable(mtb_lib):
    imgs = _natural(5, 333, 222, 3, 5, ref=1)
    a = [mtb_lib.align_stack(imgs, 5, 4, 1, level_outputs=True) for _ in range(3)]
    torch.cuda.synchronize()
    for r in a[1:]:
        for x, y in zip(a[0], r):
            assert torch.equal(x, y)


def test_invalid_arguments_enqueue_nothing(mtb_lib):
    imgs = torch.zeros((2, 8, 8, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(mtb_lib.MtbError) as ei:
        mtb_lib.align_stack(imgs, 5, 4, 0)  # 8 >> 4 == 0: too deep
    assert ei.value.status == mtb_lib.MTB_ERR_INVALID_ARG
    with pytest.raises(mtb_lib.MtbError):
        mtb_lib.align_stack(imgs, 2, 4, 2)  # ref out of range
    with pytest.raises(mtb_lib.MtbError):
        mtb_lib.align_stack(imgs, 2, 256, 0)  # tolerance out of range
    raw = torch.zeros(2 * 8 * 8 * 3 + 1, dtype=torch.uint8, device="cuda")[1:].view(2, 8, 8, 3)
    with pytest.raises(mtb_lib.MtbError):
        mtb_lib.align_stack(raw, 2, 4, 0)  # base not 16-byte aligned


def test_bounded_wait_reports_timeout(search_kernel, mtb_lib):
    """A search whose coarse work for pair 0 never reports completion: the work
    that depends on it must give up after the timeout and leave MTB_ERR_TIMEOUT
    in the status word (no hang), and a normal search afterwards is correct."""
    spec = synth.small_spec(77, 640, 480, n=3, levels=6, shift_range=20, ref=1)
    imgs = synth.make_stack(spec, "cuda")
    n, w, h, L = spec.n, spec.w, spec.h, spec.levels
    ws = mtb_lib.new_workspace(n, w, h, L)
    mtb_lib.build_pyramids(imgs, L, ws)
    mtb_lib.build_bitmaps(n, w, h, L, spec.noise_tol, ws)
    stream = torch.cuda.current_stream().cuda_stream
    rc = mtb_lib.lib().mtb_debug_search_withheld(n, w, h, L, spec.ref, ws.data_ptr(), ws.numel(), 2_000_000, stream)
    assert rc == mtb_lib.MTB_ERR_TIMEOUT
    assert mtb_lib.workspace_status(ws, n, w, h, L) == mtb_lib.MTB_ERR_TIMEOUT
    assert mtb_lib.get_last_status() == mtb_lib.MTB_ERR_TIMEOUT  # the stream's slot: no workspace needed
    shifts = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    mtb_lib.search_shifts(n, w, h, L, spec.ref, ws, shifts)
    assert mtb_lib.workspace_status(ws, n, w, h, L) == mtb_lib.MTB_OK
    assert mtb_lib.get_last_status() == mtb_lib.MTB_OK
    assert np.array_equal(shifts.cpu().numpy(), synth.expected_shifts(spec))


@pytest.mark.gpu
def test_last_status_per_stream(mtb_lib):
    """Each stream keeps the status of its own last search; a stream that never
    ran one reports MTB_OK; a call whose workspace the library allocated and
    freed still reports through its stream."""
    spec = synth.small_spec(78, 320, 240, n=3, levels=5, shift_range=5, ref=1)
    imgs = synth.make_stack(spec, "cuda")
    torch.cuda.synchronize()  # the images come from the current stream; the test uses others
    n, w, h, L = spec.n, spec.w, spec.h, spec.levels
    s1, s2, s3 = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    assert mtb_lib.get_last_status(s3) == mtb_lib.MTB_OK
    ws = mtb_lib.new_workspace(n, w, h, L)
    mtb_lib.build_pyramids(imgs, L, ws, stream=s1)
    mtb_lib.build_bitmaps(n, w, h, L, spec.noise_tol, ws, stream=s1)
    rc = mtb_lib.lib().mtb_debug_search_withheld(n, w, h, L, spec.ref, ws.data_ptr(), ws.numel(), 2_000_000,
                                                 s1.cuda_stream)
    assert rc == mtb_lib.MTB_ERR_TIMEOUT
    out = mtb_lib.align_stack(imgs, L, spec.noise_tol, spec.ref, stream=s2)  # workspace allocated and freed
    assert mtb_lib.get_last_status(s2) == mtb_lib.MTB_OK
    assert mtb_lib.get_last_status(s1) == mtb_lib.MTB_ERR_TIMEOUT
    assert np.array_equal(out.cpu().numpy(), synth.expected_shifts(spec))


@pytest.mark.gpu
def test_binding_rejects_outputs_it_could_overrun(mtb_lib):
    imgs = torch.zeros((3, 32, 64, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError, match="out must be"):
        mtb_lib.align_stack(imgs, 3, out=torch.empty((2, 2), dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError, match="out must be"):
        mtb_lib.align_stack_chain(imgs, 3, out=torch.empty((3, 2), dtype=torch.int64, device="cuda"))
    ws = mtb_lib.new_workspace(3, 64, 32, 3)
    with pytest.raises(ValueError, match="level_errs_out must be"):
        mtb_lib.search_shifts(3, 64, 32, 3, 0, ws, level_errs_out=torch.empty((3, 2, 9), dtype=torch.int32,
                                                                               device="cuda"))
    with pytest.raises(ValueError, match="workspace must be"):
        mtb_lib.align_stack(imgs, 3, workspace=ws[::2])


@pytest.mark.parametrize("w,h,n,levels,ref", [(64, 48, 3, 4, 1), (640, 480, 4, 6, 2), (2000, 1500, 3, 7, 1)])
def test_dirty_workspace_one_call(search_kernel, mtb_lib, oracle_mod, w, h, n, levels, ref):
    """The one-call path on a workspace whose bookkeeping a previous user left
    full of large values (queue head, completion counters, status word, error
    sums): the call's own clearing must come before the search reads any of
    them, also for stacks small enough that every kernel of the call is
    resident at once.  Two different stacks run back to back on it, each
    compared with the oracle."""
    lay = mtb_lib.layout(n, w, h, levels)
    ws = mtb_lib.new_workspace(n, w, h, levels)
    stacks = [_natural(900 + k, w, h, n, levels, ref=ref, shift_range=7) for k in range(2)]
    wants = [oracle_mod.align_stack(s.cpu().numpy(), levels, 4, ref) for s in stacks]
    for rep in range(3):
        ws[lay.hist_offset:].fill_(0x7F)  # every bookkeeping word 0x7f7f7f7f
        for s, want in zip(stacks, wants):
            shifts = torch.full((n, 2), -999, dtype=torch.int32, device="cuda")
            mtb_lib.align_stack(s, levels, 4, ref, workspace=ws, out=shifts)
            torch.cuda.synchronize()
            assert mtb_lib.get_last_status() == mtb_lib.MTB_OK
            assert np.array_equal(shifts.cpu().numpy(), want["shifts"]), (rep, shifts.cpu().numpy(), want["shifts"])
