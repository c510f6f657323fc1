"""The C-ABI library without a GPU: it loads, exports every function the header
declares, checks arguments before touching the device, and lays the workspace
out as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(mtb_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_core_call():
    names = declared_functions()
    assert "mtb_align_stack" in names
    assert len(names) >= 10


def test_every_declared_symbol_is_exported(mtb_lib):
    lib = ctypes.CDLL(mtb_lib.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(mtb_lib):
    for code in (0, -1, -2, -3, -4, -5):
        assert mtb_lib.status_string(code) not in ("", "unknown status")
    assert mtb_lib.status_string(12345) == "unknown status"
    assert mtb_lib.lib().mtb_abi_version() == 1


@pytest.mark.parametrize("n,w,h,levels,tol,ref", [
    (1, 64, 64, 3, 4, 0),      # one exposure: nothing to align
    (2, 0, 64, 3, 4, 0),
    (2, 64, 0, 3, 4, 0),
    (2, 65536, 4, 1, 4, 0),    # wider than MTB_MAX_DIM
    (2, 64, 64, 0, 4, 0),
    (2, 64, 64, 17, 4, 0),     # more than MTB_MAX_LEVELS
    (2, 64, 64, 8, 4, 0),      # 64 >> 7 == 0: coarsest level empty
    (2, 64, 64, 3, -1, 0),
    (2, 64, 64, 3, 256, 0),
    (2, 64, 64, 3, 4, 2),
    (2, 64, 64, 3, 4, -1),
])
def test_invalid_arguments_rejected_on_host(mtb_lib, n, w, h, levels, tol, ref):
    lib = mtb_lib.lib()
    # pointers are never dereferenced: the checks run before any CUDA call
    fake = 1 << 20
    rc = lib.mtb_align_stack(fake, n, w, h, levels, tol, ref, fake, None)
    assert rc == mtb_lib.MTB_ERR_INVALID_ARG
    rc = lib.mtb_align_stack_host(fake, n, w, h, levels, tol, ref, fake, None, 0, None)
    assert rc == mtb_lib.MTB_ERR_INVALID_ARG


def test_null_and_misaligned_pointers_rejected_on_host(mtb_lib):
    lib = mtb_lib.lib()
    assert lib.mtb_align_stack(None, 2, 64, 64, 3, 4, 0, 1 << 20, None) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_align_stack(1 << 20, 2, 64, 64, 3, 4, 0, None, None) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_align_stack((1 << 20) + 8, 2, 64, 64, 3, 4, 0, 1 << 20, None) == mtb_lib.MTB_ERR_INVALID_ARG
    nbytes = mtb_lib.workspace_bytes(2, 64, 64, 3)
    # workspace too small / misaligned
    assert lib.mtb_align_stack_ex(1 << 20, 2, 64, 64, 3, 4, 0, 1 << 20, None, None, 1 << 24, nbytes - 1,
                                  None) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_align_stack_ex(1 << 20, 2, 64, 64, 3, 4, 0, 1 << 20, None, None, (1 << 24) + 64, nbytes,
                                  None) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_build_pyramids(1 << 20, 2, 64, 64, 3, None, nbytes, None) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_build_bitmaps(2, 64, 64, 3, 300, 1 << 24, nbytes, None) == mtb_lib.MTB_ERR_INVALID_ARG
    assert lib.mtb_search_shifts(2, 64, 64, 3, 5, 1 << 24, nbytes, None, None, None,
                                 None) == mtb_lib.MTB_ERR_INVALID_ARG


@pytest.mark.parametrize("n,w,h,levels", [(2, 1, 1, 1), (3, 37, 23, 3), (7, 6000, 4000, 8), (2, 65535, 2, 2),
                                          (5, 777, 555, 9), (2, 1024, 1024, 11)])
def test_layout_invariants(mtb_lib, n, w, h, levels):
    lay = mtb_lib.layout(n, w, h, levels)
    assert mtb_lib.workspace_bytes(n, w, h, levels) == lay.total_bytes
    assert lay.tile_levels == min(levels, 6)
    regions = []
    for l in range(levels):
        assert lay.width[l] == w >> l and lay.height[l] == h >> l
        assert lay.gray_pitch[l] % 32 == 0 and lay.gray_pitch[l] >= lay.width[l]
        assert lay.bits_pitch[l] % 2 == 0 and lay.bits_pitch[l] * 32 >= lay.width[l]
        for e in range(n):
            go = lay.gray_offset[l] + e * lay.gray_exposure_stride
            bo = lay.bits_offset[l] + e * lay.bits_exposure_stride
            assert go % 256 == 0 and bo % 256 == 0
            regions.append((go, go + lay.gray_pitch[l] * lay.height[l]))
            regions.append((bo, bo + lay.bits_pitch[l] * 8 * lay.height[l]))
    regions.append((lay.hist_offset, lay.hist_offset + n * levels * 256 * 4))
    regions.append((lay.errs_offset, lay.errs_offset + n * levels * 9 * 4))
    regions.append((lay.median_offset, lay.median_offset + n * levels * 4))
    regions.append((lay.base_offset, lay.base_offset + n * levels * 8))
    regions.append((lay.shift_offset, lay.shift_offset + n * levels * 8))
    regions.append((lay.counter_offset, lay.counter_offset + (n * (2 * levels + 4) + 16) * 4))
    regions.append((lay.table_offset, lay.table_offset + n * 1280 * 4))
    regions.append((lay.status_offset, lay.status_offset + 16))
    regions.sort()
    for (a0, a1), (b0, b1) in zip(regions, regions[1:]):
        assert a1 <= b0, "workspace regions overlap"
    assert regions[-1][1] <= lay.total_bytes
    host = mtb_lib.host_workspace_bytes(n, w, h, levels)
    assert host >= lay.total_bytes + n * w * h * 3 + n * 8


def test_invalid_sizes_give_zero_workspace(mtb_lib):
    assert mtb_lib.workspace_bytes(1, 64, 64, 3) == 0
    assert mtb_lib.workspace_bytes(2, 64, 64, 8) == 0
    assert mtb_lib.host_workspace_bytes(2, 0, 64, 1) == 0


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: without the built library every call raises."""
    import paper_2007_06483_gb300 as mtb

    monkeypatch.setattr(mtb, "LIB_PATH", os.path.join(ROOT, "_no_such_dir", "libmtb_gb300.so"))
    monkeypatch.setattr(mtb, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        mtb.lib()
    with pytest.raises(RuntimeError, match="not built"):
        mtb.workspace_bytes(3, 64, 48, 3)
    with pytest.raises(RuntimeError, match="not built"):
        mtb.status_string(0)


def test_binding_rejects_misplaced_tensors_on_host():
    """The binding refuses, before any library call, tensors on the wrong side of
    the host/device boundary, and outputs the library could overrun."""
    import torch

    import paper_2007_06483_gb300 as mtb

    cpu_imgs = torch.zeros((2, 8, 16, 3), dtype=torch.uint8)
    with pytest.raises(ValueError, match="CUDA tensor"):
        mtb.align_stack(cpu_imgs, 2)
    with pytest.raises(ValueError, match="CUDA tensor"):
        mtb.align_stack_chain(cpu_imgs, 2)
    with pytest.raises(ValueError, match="CUDA tensor"):
        mtb.align_quadrants(cpu_imgs, 2)
    with pytest.raises(ValueError, match="CUDA tensor"):
        mtb.apply_shifts(cpu_imgs, torch.zeros((2, 2), dtype=torch.int32))
    with pytest.raises(ValueError, match="CUDA tensor"):
        mtb.build_bitmaps(2, 16, 8, 2, 4, torch.zeros(1024, dtype=torch.uint8))
    with pytest.raises(ValueError, match="CUDA tensor"):
        mtb.search_shifts(2, 16, 8, 2, 0, torch.zeros(1024, dtype=torch.uint8))
    meta_imgs = torch.empty((2, 8, 16, 3), dtype=torch.uint8, device="meta")
    with pytest.raises(ValueError, match="CPU tensor"):
        mtb.align_stack_host(meta_imgs, 2)
    with pytest.raises(ValueError, match="CUDA tensor"):
        mtb.align_stack_host(cpu_imgs, 2, device_workspace=torch.zeros(1024, dtype=torch.uint8))


@pytest.mark.parametrize("bad", ["shape", "dtype", "float", "strided", "device"])
def test_output_checks(bad):
    import torch

    import paper_2007_06483_gb300 as mtb

    dev = torch.device("cpu")
    good = torch.empty((3, 2), dtype=torch.int32)
    assert mtb._out(good, (3, 2), dev, "out") is good
    assert mtb._out(None, (3, 2), dev, "out") is None
    t = {"shape": torch.empty((2, 2), dtype=torch.int32),
         "dtype": torch.empty((3, 2), dtype=torch.int64),
         "float": torch.empty((3, 2), dtype=torch.float32),
         "strided": torch.empty((3, 4), dtype=torch.int32)[:, ::2],
         "device": torch.empty((3, 2), dtype=torch.int32, device="meta")}[bad]
    with pytest.raises(ValueError, match="out must be"):
        mtb._out(t, (3, 2), dev, "out")
    with pytest.raises(ValueError, match="workspace"):
        mtb._workspace(torch.empty(64, dtype=torch.uint8, device="meta"), dev)
    assert mtb._workspace(torch.empty(64, dtype=torch.int32), dev)[1] == 256


def test_aliasing_buffers_rejected_on_host(mtb_lib):
    """A workspace or an output that shares bytes with the images (or with each
    other) is refused before anything is enqueued: the kernels would write it
    while they read the images."""
    lib = mtb_lib.lib()
    n, w, h, L = 2, 64, 64, 3
    img = 1 << 30
    img_bytes = n * w * h * 3
    nbytes = mtb_lib.workspace_bytes(n, w, h, L)
    ws_far = 1 << 32
    bad = mtb_lib.MTB_ERR_INVALID_ARG
    # workspace over the images' last bytes
    assert lib.mtb_align_stack_ex(img, n, w, h, L, 4, 0, 1 << 20, None, None, img + img_bytes - 256 * 1, nbytes,
                                  None) == bad
    # shifts inside the images, inside the workspace; level outputs over the shifts
    assert lib.mtb_align_stack_ex(img, n, w, h, L, 4, 0, img + 64, None, None, ws_far, nbytes, None) == bad
    assert lib.mtb_align_stack_ex(img, n, w, h, L, 4, 0, ws_far + 4096, None, None, ws_far, nbytes, None) == bad
    assert lib.mtb_align_stack_ex(img, n, w, h, L, 4, 0, 1 << 20, (1 << 20) + 8, None, ws_far, nbytes, None) == bad
    assert lib.mtb_align_stack_chain(img, n, w, h, L, 4, 0, 1 << 20, None, None, img, nbytes, None) == bad
    assert lib.mtb_build_pyramids(img, n, w, h, L, img + 256, nbytes, None) == bad
    assert lib.mtb_search_shifts(n, w, h, L, 0, ws_far, nbytes, ws_far + 512, None, None, None) == bad
    qbytes = lib.mtb_quadrant_workspace_bytes(n, w, h, L - 1)
    assert lib.mtb_align_quadrants(img, n, w, h, L - 1, 4, 0, 1, 1 << 20, (1 << 20) + 16, ws_far, qbytes,
                                   None) == bad
