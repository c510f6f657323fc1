"""The host-buffer entry point copies stacks of 8 MB or more in row bands on the
library's copy stream and runs the pyramid pass band by band as the bands land.
Every gray plane, bit plane, histogram, median and shift must equal the device
entry point's on the same stack (whose parity with the oracle the other tests
establish), for one or several bands per exposure, a last tile row shorter than
32 rows, and a width that is not a multiple of 16."""
import threading

import numpy as np
import pytest
import torch

from paper_2007_06483_gb300 import synth

SHAPES = [
    (2000, 1501, 3, 6, 1),  # 9 MB per exposure: one band each
    (2048, 4099, 2, 7, 0),  # 25 MB: two bands; the last tile row is 3 rows high
    (1001, 2999, 5, 6, 2),  # width not a multiple of 16 (the general pyramid path)
    (4000, 3000, 3, 7, 1),  # 36 MB: two bands of 47 tile rows
]


def _align_up(v, a):
    return (v + a - 1) // a * a


def _device_result(mtb_lib, imgs, levels, ref):
    n, h, w, _ = imgs.shape
    ws = mtb_lib.new_workspace(n, w, h, levels)
    shifts = mtb_lib.align_stack(imgs, levels, 4, ref, workspace=ws)
    torch.cuda.synchronize()
    return shifts.cpu().numpy(), ws


@pytest.mark.gpu
@pytest.mark.parametrize("w,h,n,levels,ref", SHAPES)
def test_banded_host_path_equals_device_path(mtb_lib, w, h, n, levels, ref):
    spec = synth.small_spec(300 + w, w, h, n=n, levels=levels, shift_range=min(20, (1 << (levels - 1)) - 1),
                            ref=ref)
    imgs = synth.make_stack(spec, "cuda")
    dws = torch.empty(mtb_lib.host_workspace_bytes(n, w, h, levels), dtype=torch.uint8, device="cuda")
    host = mtb_lib.align_stack_host(imgs.cpu().pin_memory(), levels, 4, ref, device_workspace=dws)
    dev, ws = _device_result(mtb_lib, imgs, levels, ref)
    assert np.array_equal(host.numpy(), dev)
    a = mtb_lib.workspace_views(dws[_align_up(n * w * h * 3, 256):], n, w, h, levels)
    b = mtb_lib.workspace_views(ws, n, w, h, levels)
    lay = a["layout"]
    for e in range(n):
        for l in range(levels):
            W = lay.width[l]
            assert torch.equal(a["gray"][e][l][:, :W], b["gray"][e][l][:, :W]), (e, l)
            assert torch.equal(a["bits"][e][l], b["bits"][e][l]), (e, l)
    assert torch.equal(a["hist"], b["hist"])
    assert torch.equal(a["median"], b["median"])


@pytest.mark.gpu
def test_banded_host_path_back_to_back_and_from_two_threads(mtb_lib):
    """Calls on one workspace one after another (each call's copy waits for the
    work enqueued before it on the stream), then from two host threads at once
    with their own streams and workspaces, sharing the library's copy stream."""
    n, w, h, levels, ref = 3, 2000, 1501, 6, 1
    specs = [synth.small_spec(40 + k, w, h, n=n, levels=levels, shift_range=20, ref=ref) for k in range(3)]
    dev_imgs = [synth.make_stack(s, "cuda") for s in specs]
    hosts = [im.cpu().pin_memory() for im in dev_imgs]
    want = [_device_result(mtb_lib, im, levels, ref)[0] for im in dev_imgs]
    nbytes = mtb_lib.host_workspace_bytes(n, w, h, levels)
    dws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    out = torch.empty((n, 2), dtype=torch.int32, pin_memory=True)
    for rnd in range(2):
        for k in range(3):
            got = mtb_lib.align_stack_host(hosts[k], levels, 4, ref, device_workspace=dws, out=out if rnd else None,
                                           stream=stream)
            assert got is out or rnd == 0
            assert np.array_equal(got.numpy(), want[k]), (rnd, k)
    results, errors = {}, []

    def worker(t):
        try:
            st = torch.cuda.Stream()
            ws_t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            for rnd in range(3):
                for k in range(3):
                    results[(t, rnd, k)] = mtb_lib.align_stack_host(hosts[k], levels, 4, ref, device_workspace=ws_t,
                                                                    stream=st).numpy()
        except Exception as ex:  # reported below, on the test's thread
            errors.append(repr(ex))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    assert len(results) == 18
    for (t, rnd, k), got in results.items():
        assert np.array_equal(got, want[k]), (t, rnd, k)
