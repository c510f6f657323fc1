"""Oracle for the MTB alignment path -- TEST INFRASTRUCTURE, not the product.

A plain single-threaded C statement (``mtb_oracle.c``) of Ward-style median
threshold bitmap alignment as Sec. III-A and Sec. III-B of arXiv 2007.06483
describe it, with numpy wrappers.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its CPU-baseline leg and ``--impl reference``) may import it.
It shares no code with ``paper_2007_06483_gb300`` and never imports it.

Parity status of each function (what pins it is listed in the tests):
  gray, shrink, histogram, median, bitmaps, shift_error   pinned
  search_pair / align_stack                               pinned on planted shifts,
      brute force on clear optima and invariants; the pyramid result on
      ambiguous content has no value printed by the paper to compare with.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mtb_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libmtb_oracle.so")
_lock = threading.Lock()
_lib = None

def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile an oracle source with gcc into a shared library (default
    oracle/_build/libmtb_oracle.so)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared", "-o", tmp, src]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def level_dims(w: int, h: int, levels: int):
    return [(w >> l, h >> l) for l in range(levels)]


class Oracle:
    """numpy front end of one compiled oracle library."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        P = ctypes.c_void_p
        I = ctypes.c_int
        L = ctypes.c_long
        lib.orc_gray.argtypes = [P, L, P]
        lib.orc_shrink.argtypes = [P, I, I, P]
        lib.orc_histogram.argtypes = [P, L, P]
        lib.orc_median.argtypes = [P]
        lib.orc_median.restype = I
        lib.orc_bitmaps.argtypes = [P, L, I, I, P, P]
        lib.orc_shift_error.argtypes = [P, P, P, P, I, I, I, I]
        lib.orc_shift_error.restype = ctypes.c_uint32
        lib.orc_level_offset.argtypes = [I, I, I]
        lib.orc_level_offset.restype = L
        lib.orc_search_pair.argtypes = [P, P, P, P, I, I, I, P, P]
        lib.orc_exposure_maps.argtypes = [P, I, I, I, I, P, P, P, P, P]
        lib.orc_check_args.argtypes = [I, I, I, I, I, I]
        lib.orc_check_args.restype = I
        lib.orc_align_stack.argtypes = [P, I, I, I, I, I, I, P, P, P]
        lib.orc_align_stack.restype = I
        lib.orc_apply_shifts.argtypes = [P, I, I, I, P, I, P]
        lib.orc_align_stack_chain.argtypes = [P, I, I, I, I, I, I, P, P, P]
        lib.orc_align_stack_chain.restype = I
        lib.orc_align_quadrants.argtypes = [P, I, I, I, I, I, I, I, P, P]
        lib.orc_align_quadrants.restype = I
        lib.orc_candidate.argtypes = [I, ctypes.POINTER(I), ctypes.POINTER(I)]
        lib.orc_candidate.restype = I
        self.lib = lib

    def candidates(self):
        out = []
        for k in range(9):
            dx, dy = ctypes.c_int(), ctypes.c_int()
            assert self.lib.orc_candidate(k, ctypes.byref(dx), ctypes.byref(dy)) == 0
            out.append((dx.value, dy.value))
        return tuple(out)

    def gray(self, rgb) -> np.ndarray:
        """[..., 3] uint8 RGB -> [...] uint8 gray (Sec. III-A)."""
        rgb = _u8(rgb)
        assert rgb.shape[-1] == 3
        out = np.empty(rgb.shape[:-1], np.uint8)
        self.lib.orc_gray(_ptr(rgb), out.size, _ptr(out))
        return out

    def shrink(self, g) -> np.ndarray:
        """[h, w] uint8 -> [h//2, w//2] uint8, 2x2 mean rounded half up (Sec. III-A)."""
        g = _u8(g)
        h, w = g.shape
        out = np.empty((h // 2, w // 2), np.uint8)
        if out.size:
            self.lib.orc_shrink(_ptr(g), w, h, _ptr(out))
        return out

    def histogram(self, g) -> np.ndarray:
        """256-bin histogram of a gray image (Sec. III-B)."""
        g = _u8(g)
        out = np.empty(256, np.uint32)
        self.lib.orc_histogram(_ptr(g), g.size, _ptr(out))
        return out

    def median(self, hist) -> int:
        """Lower median from a 256-bin histogram (Sec. III-A)."""
        h = np.ascontiguousarray(hist, dtype=np.uint32)
        assert h.shape == (256,)
        return int(self.lib.orc_median(_ptr(h)))

    def bitmaps(self, g, med: int, tol: int):
        """(tb, eb) byte-maps of 0/1 for a gray image (Sec. III-A, III-B)."""
        g = _u8(g)
        tb = np.empty_like(g)
        eb = np.empty_like(g)
        self.lib.orc_bitmaps(_ptr(g), g.size, int(med), int(tol), _ptr(tb), _ptr(eb))
        return tb, eb

    def shift_error(self, tb_r, eb_r, tb_i, eb_i, sx: int, sy: int) -> int:
        """Count of (tb_r XOR S(tb_i)) AND eb_r AND S(eb_i), S = shift by (sx, sy)."""
        arrs = [_u8(a) for a in (tb_r, eb_r, tb_i, eb_i)]
        h, w = arrs[0].shape
        for a in arrs:
            assert a.shape == (h, w)
        return int(self.lib.orc_shift_error(*[_ptr(a) for a in arrs], w, h, int(sx), int(sy)))

    def pyramid_maps(self, rgb, levels: int, tol: int) -> dict:
        """Gray pyramid, histograms, medians, tb and eb of one [h, w, 3] exposure,
        as lists indexed by level (level 0 = full resolution)."""
        rgb = _u8(rgb)
        h, w, c = rgb.shape
        assert c == 3
        lib = self.lib
        total = lib.orc_level_offset(w, h, levels)
        gray_all = np.empty(total, np.uint8)
        tb_all = np.empty(total, np.uint8)
        eb_all = np.empty(total, np.uint8)
        hist = np.empty((levels, 256), np.uint32)
        med = np.empty(levels, np.int32)
        lib.orc_exposure_maps(_ptr(rgb), w, h, levels, int(tol), _ptr(gray_all), _ptr(hist),
                              _ptr(med), _ptr(tb_all), _ptr(eb_all))
        out = {"gray": [], "tb": [], "eb": [], "hist": hist, "median": med}
        for l, (wl, hl) in enumerate(level_dims(w, h, levels)):
            off = lib.orc_level_offset(w, h, l)
            n = wl * hl
            out["gray"].append(gray_all[off:off + n].reshape(hl, wl))
            out["tb"].append(tb_all[off:off + n].reshape(hl, wl))
            out["eb"].append(eb_all[off:off + n].reshape(hl, wl))
        return out

    def search_pair(self, tb_r, eb_r, tb_i, eb_i):
        """Coarse-to-fine search over per-level maps (lists, level 0 first).
        Returns (errs [levels, 9] uint32, best [levels, 2] int32)."""
        levels = len(tb_r)
        h, w = tb_r[0].shape
        for l in range(levels):
            assert tb_r[l].shape == (h >> l, w >> l)
        cat = [np.ascontiguousarray(np.concatenate([_u8(a).ravel() for a in m])) for m in (tb_r, eb_r, tb_i, eb_i)]
        errs = np.zeros((levels, 9), np.uint32)
        best = np.zeros((levels, 2), np.int32)
        self.lib.orc_search_pair(*[_ptr(a) for a in cat], w, h, levels, _ptr(errs), _ptr(best))
        return errs, best

    def check_args(self, n: int, w: int, h: int, levels: int, tol: int, ref: int) -> bool:
        return self.lib.orc_check_args(n, w, h, levels, tol, ref) == 0

    def align_stack(self, images, levels: int, noise_tol: int, ref_idx: int) -> dict:
        """Align every exposure of [n, h, w, 3] uint8 to exposure ref_idx (Sec. III-B).
        Returns dict(shifts [n,2] int32, level_errs [n,levels,9] uint32,
        level_shifts [n,levels,2] int32); rows of ref_idx are zero."""
        images = _u8(images)
        n, h, w, c = images.shape
        assert c == 3
        shifts = np.zeros((n, 2), np.int32)
        errs = np.zeros((n, levels, 9), np.uint32)
        lsh = np.zeros((n, levels, 2), np.int32)
        rc = self.lib.orc_align_stack(_ptr(images), n, w, h, levels, int(noise_tol), int(ref_idx),
                                      _ptr(shifts), _ptr(errs), _ptr(lsh))
        if rc == -1:
            raise ValueError("invalid arguments")
        if rc != 0:
            raise MemoryError("oracle ran out of host memory")
        return {"shifts": shifts, "level_errs": errs, "level_shifts": lsh}


    def apply_shifts(self, images, shifts, fill: int = 0) -> np.ndarray:
        """Each exposure of [n, h, w, 3] moved by its (sx, sy); fill 0: zeros,
        1: nearest edge pixel, where the source lies outside."""
        images = _u8(images)
        n, h, w, c = images.shape
        assert c == 3
        shifts = np.ascontiguousarray(shifts, dtype=np.int32).reshape(n, 2)
        out = np.empty_like(images)
        self.lib.orc_apply_shifts(_ptr(images), n, w, h, _ptr(shifts), int(fill), _ptr(out))
        return out

    def align_stack_chain(self, images, levels: int, noise_tol: int, ref_idx: int) -> dict:
        """Consecutive-chain alignment: each exposure against its neighbour towards
        ref_idx, shifts composed along the chain.  Same outputs as align_stack
        (per-level rows hold the neighbour pair's values)."""
        images = _u8(images)
        n, h, w, c = images.shape
        assert c == 3
        shifts = np.zeros((n, 2), np.int32)
        errs = np.zeros((n, levels, 9), np.uint32)
        lsh = np.zeros((n, levels, 2), np.int32)
        rc = self.lib.orc_align_stack_chain(_ptr(images), n, w, h, levels, int(noise_tol), int(ref_idx),
                                            _ptr(shifts), _ptr(errs), _ptr(lsh))
        if rc == -1:
            raise ValueError("invalid arguments")
        if rc != 0:
            raise MemoryError("oracle ran out of host memory")
        return {"shifts": shifts, "level_errs": errs, "level_shifts": lsh}

    def align_quadrants(self, images, levels: int, noise_tol: int, ref_idx: int, rot_tol: int = 1) -> dict:
        """Per-quadrant alignment (quadrants TL, TR, BL, BR) and the rotation flag.
        Returns dict(quad_shifts [n,4,2] int32, flags [n] int32)."""
        images = _u8(images)
        n, h, w, c = images.shape
        assert c == 3
        qs = np.zeros((n, 4, 2), np.int32)
        flags = np.zeros(n, np.int32)
        rc = self.lib.orc_align_quadrants(_ptr(images), n, w, h, levels, int(noise_tol), int(ref_idx),
                                          int(rot_tol), _ptr(qs), _ptr(flags))
        if rc == -1:
            raise ValueError("invalid arguments")
        if rc != 0:
            raise MemoryError("oracle ran out of host memory")
        return {"quad_shifts": qs, "flags": flags}


def default() -> Oracle:
    """The oracle built from oracle/mtb_oracle.c."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
        return _lib


def gray(rgb):
    return default().gray(rgb)


def shrink(g):
    return default().shrink(g)


def histogram(g):
    return default().histogram(g)


def median(hist):
    return default().median(hist)


def bitmaps(g, med, tol):
    return default().bitmaps(g, med, tol)


def shift_error(tb_r, eb_r, tb_i, eb_i, sx, sy):
    return default().shift_error(tb_r, eb_r, tb_i, eb_i, sx, sy)


def pyramid_maps(rgb, levels, tol):
    return default().pyramid_maps(rgb, levels, tol)


def search_pair(tb_r, eb_r, tb_i, eb_i):
    return default().search_pair(tb_r, eb_r, tb_i, eb_i)


def check_args(n, w, h, levels, tol, ref):
    return default().check_args(n, w, h, levels, tol, ref)


def align_stack(images, levels, noise_tol, ref_idx):
    return default().align_stack(images, levels, noise_tol, ref_idx)


def apply_shifts(images, shifts, fill=0):
    return default().apply_shifts(images, shifts, fill)


def align_stack_chain(images, levels, noise_tol, ref_idx):
    return default().align_stack_chain(images, levels, noise_tol, ref_idx)


def align_quadrants(images, levels, noise_tol, ref_idx, rot_tol=1):
    return default().align_quadrants(images, levels, noise_tol, ref_idx, rot_tol)
