"""mtb_align_stack_noalloc, the entry point for callers that cannot allocate
device memory while they align (a per-frame loop with a deadline, a plug-in
whose host owns every allocation, a fixed memory budget).  It must give exactly
what mtb_align_stack_ex gives, call after call, although every call reuses the
same fixed scratch array.  This file sorts last so that a run stopping at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2007_06483_gb300 import synth

pytestmark = pytest.mark.gpu

NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def _c_entry(mtb):
    lib = ctypes.CDLL(mtb.library_path())
    fn = lib.mtb_align_stack_noalloc
    P, I = ctypes.c_void_p, ctypes.c_int
    fn.restype = I
    fn.argtypes = [P, I, I, I, I, I, I, P, P, P, P]
    return fn


def test_noalloc_matches_align_stack_ex_twice_in_a_row(mtb_lib):
    fn = _c_entry(mtb_lib)
    stream = torch.cuda.current_stream().cuda_stream
    # two different stacks back to back: the second must not see the first's leftovers
    specs = [synth.small_spec(41, 1280, 720, n=4, levels=6, shift_range=40, ref=1), synth.PAIR_640]
    for spec in specs:
        imgs = synth.make_stack(spec, "cuda")
        n = spec.n
        assert mtb_lib.workspace_bytes(n, spec.w, spec.h, spec.levels) <= NOALLOC_SCRATCH_BYTES
        want_s, want_e, want_l = mtb_lib.align_stack(imgs, spec.levels, spec.noise_tol, spec.ref,
                                                     level_outputs=True)
        got_s = torch.full((n, 2), -7, dtype=torch.int32, device="cuda")
        got_e = torch.full((n, spec.levels, 9), -7, dtype=torch.int32, device="cuda")
        got_l = torch.full((n, spec.levels, 2), -7, dtype=torch.int32, device="cuda")
        rc = fn(imgs.data_ptr(), n, spec.w, spec.h, spec.levels, spec.noise_tol, spec.ref, got_s.data_ptr(),
                got_e.data_ptr(), got_l.data_ptr(), stream)
        assert rc == 0, mtb_lib.status_string(rc)
        torch.cuda.synchronize()
        assert torch.equal(got_s, want_s)
        assert torch.equal(got_e, want_e)
        assert torch.equal(got_l, want_l)
        assert np.array_equal(got_s.cpu().numpy(), synth.expected_shifts(spec))


def test_noalloc_rejects_stacks_beyond_its_scratch(mtb_lib):
    fn = _c_entry(mtb_lib)
    imgs = torch.zeros((2, 16, 16, 3), dtype=torch.uint8, device="cuda")
    out = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    w, h = 6000, 4000  # 2 x 24 MP needs far more than the fixed array
    assert mtb_lib.workspace_bytes(2, w, h, 8) > NOALLOC_SCRATCH_BYTES
    rc = fn(imgs.data_ptr(), 2, w, h, 8, 4, 0, out.data_ptr(), None, None, None)
    assert rc == mtb_lib.MTB_ERR_INVALID_ARG


class _DefaultPool:
    """The device's default stream-ordered memory pool, read through the driver
    (libcuda): its used-memory high watermark shows any cudaMallocAsync made
    between two readings, also one freed again before the second."""

    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8  # CU_MEMPOOL_ATTR_*

    def __init__(self, index: int):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), index) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr: int) -> int:
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)  # the high watermark may only be set to 0, which resets it
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0


def test_noalloc_allocates_nothing(mtb_lib):
    """What the entry point is for: once set up, a call makes no device
    allocation -- none through the stream-ordered pool (whose high watermark
    would show even an allocation freed within the call) and none through
    torch's allocator."""
    fn = _c_entry(mtb_lib)
    spec = synth.small_spec(43, 960, 540, n=3, levels=5, shift_range=12, ref=1)
    imgs = synth.make_stack(spec, "cuda")
    n, L = spec.n, spec.levels
    outs = [torch.empty((n, 2), dtype=torch.int32, device="cuda"),
            torch.empty((n, L, 9), dtype=torch.int32, device="cuda"),
            torch.empty((n, L, 2), dtype=torch.int32, device="cuda")]
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        return fn(imgs.data_ptr(), n, spec.w, spec.h, L, spec.noise_tol, spec.ref, outs[0].data_ptr(),
                  outs[1].data_ptr(), outs[2].data_ptr(), stream)

    assert call() == 0  # set-up: the scratch address is looked up here
    torch.cuda.synchronize()
    want = mtb_lib.align_stack(imgs, L, spec.noise_tol, spec.ref)  # may use the pool itself
    torch.cuda.synchronize()
    pool = _DefaultPool(torch.cuda.current_device())
    used = pool.get(pool.USED_MEM_CURRENT)
    pool.reset_high()
    torch.cuda.reset_peak_memory_stats()
    torch_before = torch.cuda.memory_allocated()
    for _ in range(2):
        assert call() == 0
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) <= used, "the no-alloc call allocated from the stream-ordered pool"
    assert torch.cuda.max_memory_allocated() == torch_before, "device memory was allocated during the call"
    assert torch.equal(outs[0], want)
