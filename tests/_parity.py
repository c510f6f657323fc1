"""Helpers shared by the GPU parity tests: run the CUDA stages through the C ABI
and compare every intermediate and output with the oracle, element by element.
The whole path is integer, so every comparison is exact (tolerance 0)."""
from __future__ import annotations

import numpy as np


def unpack_plane(words: np.ndarray, width: int):
    """int32 [H, bp, 2] (tb word, eb word) -> (tb, eb) uint8 [H, width] and the
    pad bits beyond width, bit b of word q being pixel 32q + b."""
    u = np.ascontiguousarray(words).view(np.uint32)
    H, bp, _ = u.shape
    out = []
    pads = []
    for c in range(2):
        plane = np.ascontiguousarray(u[:, :, c])
        bits = np.unpackbits(plane.view(np.uint8).reshape(H, bp * 4), axis=1, bitorder="little")
        out.append(bits[:, :width])
        pads.append(bits[:, width:])
    return out[0], out[1], pads


def run_stages(mtb, images, levels, tol, ref):
    import torch

    n, h, w, _ = images.shape
    ws = mtb.new_workspace(n, w, h, levels, device=images.device)
    ws.fill_(0xA5)  # stale bytes must not leak into any result
    mtb.build_pyramids(images, levels, ws)
    mtb.build_bitmaps(n, w, h, levels, tol, ws)
    dev = images.device
    shifts = torch.full((n, 2), -999, dtype=torch.int32, device=dev)
    errs = torch.full((n, levels, 9), -1, dtype=torch.int32, device=dev)
    lsh = torch.full((n, levels, 2), -999, dtype=torch.int32, device=dev)
    mtb.search_shifts(n, w, h, levels, ref, ws, shifts, errs, lsh)
    torch.cuda.synchronize()
    return ws, shifts, errs, lsh


def check_stack(mtb, oracle, images, levels, tol, ref, maps=True):
    """Stage-by-stage parity of one stack, then the one-call path
    (mtb_align_stack_ex, the three stages chained on one stream); returns the
    oracle's result."""
    import torch

    n, h, w, _ = images.shape
    ws, shifts, errs, lsh = run_stages(mtb, images, levels, tol, ref)
    imgs = images.cpu().numpy()
    want = oracle.align_stack(imgs, levels, tol, ref)
    if maps:
        views = mtb.workspace_views(ws, n, w, h, levels)
        hist = views["hist"].cpu().numpy().view(np.uint32)
        med = views["median"].cpu().numpy()
        for e in range(n):
            m = oracle.pyramid_maps(imgs[e], levels, tol)
            for l in range(levels):
                wl, hl = w >> l, h >> l
                g = views["gray"][e][l].cpu().numpy()[:, :wl]
                assert np.array_equal(g, m["gray"][l]), f"gray e={e} l={l}"
                assert np.array_equal(hist[e, l], m["hist"][l]), f"hist e={e} l={l}"
                assert med[e, l] == m["median"][l], f"median e={e} l={l}: {med[e, l]} vs {m['median'][l]}"
                tb, eb, pads = unpack_plane(views["bits"][e][l].cpu().numpy(), wl)
                assert np.array_equal(tb, m["tb"][l]), f"tb e={e} l={l}"
                assert np.array_equal(eb, m["eb"][l]), f"eb e={e} l={l}"
                assert not pads[0].any() and not pads[1].any(), f"pad bits e={e} l={l}"
    assert np.array_equal(errs.cpu().numpy().view(np.uint32), want["level_errs"]), "level errors"
    assert np.array_equal(lsh.cpu().numpy(), want["level_shifts"]), "level shifts"
    assert np.array_equal(shifts.cpu().numpy(), want["shifts"]), "shifts"
    # the one-call path: the same kernels, launched back to back with programmatic
    # dependent launch between the stages
    e_shifts, e_errs, e_lsh = mtb.align_stack(images, levels, tol, ref, level_outputs=True)
    torch.cuda.synchronize()
    assert np.array_equal(e_errs.cpu().numpy().view(np.uint32), want["level_errs"]), "one-call level errors"
    assert np.array_equal(e_lsh.cpu().numpy(), want["level_shifts"]), "one-call level shifts"
    assert np.array_equal(e_shifts.cpu().numpy(), want["shifts"]), "one-call shifts"
    return want
