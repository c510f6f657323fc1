"""GB300 median-threshold-bitmap (MTB) exposure alignment.

Thin ctypes binding over the C ABI of ``include/mtb.h`` (library built in-tree
by ``paper_2007_06483_gb300.build``).  Every step of the alignment runs in the
CUDA kernels of that library; this module only marshals arguments.  PyTorch is
used for device memory and stream handles.  There is no CPU fallback: if the
library is missing the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

from .build import LIB_PATH

MTB_OK = 0
MTB_ERR_INVALID_ARG = -1
MTB_ERR_OOM = -2
MTB_ERR_CUDA = -3
MTB_ERR_TIMEOUT = -4
MTB_ERR_BUSY = -5
MTB_MAX_LEVELS = 16
MTB_FILL_ZERO = 0
MTB_FILL_EDGE = 1

_lock = threading.Lock()
_lib = None


class MtbError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = status_string(status) if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


class Layout(ctypes.Structure):
    """Mirror of mtb_layout_t."""

    _fields_ = [
        ("n", ctypes.c_int32), ("w", ctypes.c_int32), ("h", ctypes.c_int32), ("levels", ctypes.c_int32),
        ("tile_levels", ctypes.c_int32),
        ("width", ctypes.c_int32 * MTB_MAX_LEVELS),
        ("height", ctypes.c_int32 * MTB_MAX_LEVELS),
        ("gray_pitch", ctypes.c_int32 * MTB_MAX_LEVELS),
        ("bits_pitch", ctypes.c_int32 * MTB_MAX_LEVELS),
        ("gray_offset", ctypes.c_uint64 * MTB_MAX_LEVELS),
        ("gray_exposure_stride", ctypes.c_uint64),
        ("bits_offset", ctypes.c_uint64 * MTB_MAX_LEVELS),
        ("bits_exposure_stride", ctypes.c_uint64),
        ("hist_offset", ctypes.c_uint64),
        ("median_offset", ctypes.c_uint64),
        ("errs_offset", ctypes.c_uint64),
        ("base_offset", ctypes.c_uint64),
        ("shift_offset", ctypes.c_uint64),
        ("table_offset", ctypes.c_uint64),
        ("counter_offset", ctypes.c_uint64),
        ("status_offset", ctypes.c_uint64),
        ("total_bytes", ctypes.c_uint64),
    ]


class StackDesc(ctypes.Structure):
    """Mirror of mtb_stack_desc_t."""

    _fields_ = [
        ("images", ctypes.c_void_p),
        ("n_exposures", ctypes.c_int), ("w", ctypes.c_int), ("h", ctypes.c_int), ("levels", ctypes.c_int),
        ("noise_tol", ctypes.c_int), ("ref_idx", ctypes.c_int),
        ("shifts_out", ctypes.c_void_p), ("level_errs_out", ctypes.c_void_p), ("level_shifts_out", ctypes.c_void_p),
    ]


class ServerConfig(ctypes.Structure):
    """Mirror of mtb_server_config_t."""

    _fields_ = [("budget_bytes", ctypes.c_size_t), ("slots", ctypes.c_int), ("copy_streams", ctypes.c_int),
                ("max_pending", ctypes.c_int)]


class Job(ctypes.Structure):
    """Mirror of mtb_job_t."""

    _fields_ = [
        ("host_images", ctypes.c_void_p),
        ("n_exposures", ctypes.c_int), ("w", ctypes.c_int), ("h", ctypes.c_int), ("levels", ctypes.c_int),
        ("noise_tol", ctypes.c_int), ("ref_idx", ctypes.c_int),
        ("host_shifts_out", ctypes.c_void_p),
    ]


def library_path() -> str:
    return LIB_PATH


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run paper_2007_06483_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        sig = {
            "mtb_status_string": (ctypes.c_char_p, [I]),
            "mtb_abi_version": (I, []),
            "mtb_workspace_bytes": (S, [I, I, I, I]),
            "mtb_workspace_layout": (I, [I, I, I, I, ctypes.POINTER(Layout)]),
            "mtb_align_stack": (I, [P, I, I, I, I, I, I, P, P]),
            "mtb_align_stack_ex": (I, [P, I, I, I, I, I, I, P, P, P, P, S, P]),
            "mtb_build_pyramids": (I, [P, I, I, I, I, P, S, P]),
            "mtb_build_bitmaps": (I, [I, I, I, I, I, P, S, P]),
            "mtb_search_shifts": (I, [I, I, I, I, I, P, S, P, P, P, P]),
            "mtb_host_workspace_bytes": (S, [I, I, I, I]),
            "mtb_align_stack_host": (I, [P, I, I, I, I, I, I, P, P, S, P]),
            "mtb_workspace_status": (I, [P, S, I, I, I, I, P]),
            "mtb_debug_search_withheld": (I, [I, I, I, I, I, P, S, ctypes.c_longlong, P]),
            "mtb_search_kernel": (I, [I, I, I, I, I, I]),
            "mtb_server_wait_phases": (I, [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
            "mtb_batch_workspace_bytes": (S, [P, I]),
            "mtb_batch_create": (I, [P, I, P, S, ctypes.POINTER(ctypes.c_void_p)]),
            "mtb_batch_run": (I, [P, P]),
            "mtb_batch_tune": (I, [P, I, P]),
            "mtb_get_last_status": (I, [P]),
            "mtb_batch_config": (I, [P, ctypes.POINTER(ctypes.c_int), I]),
            "mtb_batch_set_config": (I, [P, ctypes.POINTER(ctypes.c_int), I]),
            "mtb_batch_status": (I, [P, P]),
            "mtb_batch_destroy": (None, [P]),
            "mtb_apply_shifts": (I, [P, I, I, I, P, I, P, P]),
            "mtb_align_stack_chain": (I, [P, I, I, I, I, I, I, P, P, P, P, S, P]),
            "mtb_quadrant_workspace_bytes": (S, [I, I, I, I]),
            "mtb_align_quadrants": (I, [P, I, I, I, I, I, I, I, P, P, P, S, P]),
            "mtb_job_bytes": (S, [ctypes.POINTER(Job)]),
            "mtb_server_create": (I, [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]),
            "mtb_server_submit": (I, [P, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)]),
            "mtb_server_poll": (I, [P, ctypes.c_uint64]),
            "mtb_server_wait": (I, [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
            "mtb_server_pause": (I, [P, I]),
            "mtb_server_stats": (I, [P, ctypes.POINTER(ctypes.c_uint64), I]),
            "mtb_server_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def status_string(status: int) -> str:
    return lib().mtb_status_string(int(status)).decode()


def _check(rc: int, what: str):
    if rc != MTB_OK:
        raise MtbError(rc, what)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def workspace_bytes(n: int, w: int, h: int, levels: int) -> int:
    return int(lib().mtb_workspace_bytes(n, w, h, levels))


def host_workspace_bytes(n: int, w: int, h: int, levels: int) -> int:
    return int(lib().mtb_host_workspace_bytes(n, w, h, levels))


def layout(n: int, w: int, h: int, levels: int) -> Layout:
    out = Layout()
    _check(lib().mtb_workspace_layout(n, w, h, levels, ctypes.byref(out)), "mtb_workspace_layout")
    return out


def _dims(images):
    import torch

    if not isinstance(images, torch.Tensor) or images.dtype != torch.uint8 or images.dim() != 4 or images.shape[-1] != 3:
        raise ValueError("images must be a uint8 tensor [n, h, w, 3]")
    if not images.is_contiguous():
        raise ValueError("images must be contiguous")
    n, h, w, _ = images.shape
    return int(n), int(w), int(h)


def _cuda_dims(images):
    """_dims for the entry points that read the images from device memory."""
    n, w, h = _dims(images)
    if images.device.type != "cuda":
        raise ValueError("images must be a CUDA tensor")
    return n, w, h


def _out(t, shape, dev, what):
    """t (or None) as an output the library writes: a contiguous 32-bit integer
    tensor of `shape` on device `dev`."""
    import torch

    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.device != dev or t.element_size() != 4 or t.dtype.is_floating_point or \
            tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous 32-bit integer tensor {list(shape)} on {dev}")
    return t


def _workspace(ws, dev):
    """(pointer, bytes) of a caller workspace on device `dev`, (None, 0) for none."""
    import torch

    if ws is None:
        return None, 0
    if not isinstance(ws, torch.Tensor) or ws.device != dev or not ws.is_contiguous():
        raise ValueError(f"workspace must be a contiguous tensor on {dev}")
    return ws.data_ptr(), ws.numel() * ws.element_size()


def new_workspace(n: int, w: int, h: int, levels: int, device="cuda"):
    import torch

    nbytes = workspace_bytes(n, w, h, levels)
    if nbytes == 0:
        raise MtbError(MTB_ERR_INVALID_ARG, "workspace size")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def align_stack(images, levels: int, noise_tol: int = 4, ref_idx: int = 0, *, level_outputs: bool = False,
                workspace=None, out=None, stream=None):
    """Align a [n, h, w, 3] uint8 CUDA stack; returns int32 [n, 2] shifts on the
    device (and, with level_outputs, uint32 [n, levels, 9] errors and int32
    [n, levels, 2] per-level shifts).  `out` may hold the int32 [n, 2] result."""
    import torch

    n, w, h = _cuda_dims(images)
    dev = images.device
    shifts = _out(out, (n, 2), dev, "out") if out is not None else torch.empty((n, 2), dtype=torch.int32, device=dev)
    errs = lsh = None
    if level_outputs:
        errs = torch.empty((n, levels, 9), dtype=torch.int32, device=dev)  # viewed as uint32
        lsh = torch.empty((n, levels, 2), dtype=torch.int32, device=dev)
    ws_ptr, ws_bytes = _workspace(workspace, dev)
    if errs is None and workspace is None:
        rc = lib().mtb_align_stack(images.data_ptr(), n, w, h, levels, noise_tol, ref_idx, shifts.data_ptr(),
                                   _stream(stream))
    else:
        rc = lib().mtb_align_stack_ex(images.data_ptr(), n, w, h, levels, noise_tol, ref_idx, shifts.data_ptr(),
                                      _ptr(errs), _ptr(lsh), ws_ptr, ws_bytes, _stream(stream))
    _check(rc, "mtb_align_stack")
    if level_outputs:
        return shifts, errs, lsh
    return shifts


def align_stack_chain(images, levels: int, noise_tol: int = 4, ref_idx: int = 0, *, level_outputs: bool = False,
                      workspace=None, out=None, stream=None):
    """mtb_align_stack_chain: every exposure searched against its neighbour
    towards ref_idx, shifts composed along the chain.  Returns and outputs as
    align_stack (per-level rows hold the neighbour pair's values)."""
    import torch

    n, w, h = _cuda_dims(images)
    dev = images.device
    shifts = _out(out, (n, 2), dev, "out") if out is not None else torch.empty((n, 2), dtype=torch.int32, device=dev)
    errs = lsh = None
    if level_outputs:
        errs = torch.empty((n, levels, 9), dtype=torch.int32, device=dev)  # viewed as uint32
        lsh = torch.empty((n, levels, 2), dtype=torch.int32, device=dev)
    ws_ptr, ws_bytes = _workspace(workspace, dev)
    _check(lib().mtb_align_stack_chain(images.data_ptr(), n, w, h, levels, noise_tol, ref_idx, shifts.data_ptr(),
                                       _ptr(errs), _ptr(lsh), ws_ptr, ws_bytes, _stream(stream)),
           "mtb_align_stack_chain")
    if level_outputs:
        return shifts, errs, lsh
    return shifts


def align_quadrants(images, levels: int, noise_tol: int = 4, ref_idx: int = 0, rot_tol: int = 1, *,
                    workspace=None, stream=None):
    """mtb_align_quadrants: per-quadrant alignment (TL, TR, BL, BR) and the
    rotation flag.  Returns (quad_shifts int32 [n, 4, 2], flags int32 [n]) on
    the device."""
    import torch

    n, w, h = _cuda_dims(images)
    dev = images.device
    qs = torch.empty((n, 4, 2), dtype=torch.int32, device=dev)
    flags = torch.empty((n,), dtype=torch.int32, device=dev)
    ws_ptr, ws_bytes = _workspace(workspace, dev)
    _check(lib().mtb_align_quadrants(images.data_ptr(), n, w, h, levels, noise_tol, ref_idx, rot_tol, qs.data_ptr(),
                                     flags.data_ptr(), ws_ptr, ws_bytes, _stream(stream)), "mtb_align_quadrants")
    return qs, flags


def build_pyramids(images, levels: int, workspace, stream=None):
    n, w, h = _cuda_dims(images)
    ws_ptr, ws_bytes = _workspace(workspace, images.device)
    _check(lib().mtb_build_pyramids(images.data_ptr(), n, w, h, levels, ws_ptr, ws_bytes, _stream(stream)),
           "mtb_build_pyramids")


def _stage_workspace(workspace):
    if workspace is None or workspace.device.type != "cuda":
        raise ValueError("workspace must be a CUDA tensor")
    return _workspace(workspace, workspace.device)


def build_bitmaps(n: int, w: int, h: int, levels: int, noise_tol: int, workspace, stream=None):
    ws_ptr, ws_bytes = _stage_workspace(workspace)
    _check(lib().mtb_build_bitmaps(n, w, h, levels, noise_tol, ws_ptr, ws_bytes, _stream(stream)),
           "mtb_build_bitmaps")


def search_shifts(n: int, w: int, h: int, levels: int, ref_idx: int, workspace, shifts_out=None,
                  level_errs_out=None, level_shifts_out=None, stream=None):
    ws_ptr, ws_bytes = _stage_workspace(workspace)
    dev = workspace.device
    sh = _out(shifts_out, (n, 2), dev, "shifts_out")
    er = _out(level_errs_out, (n, levels, 9), dev, "level_errs_out")
    ls = _out(level_shifts_out, (n, levels, 2), dev, "level_shifts_out")
    _check(lib().mtb_search_shifts(n, w, h, levels, ref_idx, ws_ptr, ws_bytes, _ptr(sh), _ptr(er), _ptr(ls),
                                   _stream(stream)), "mtb_search_shifts")


def workspace_status(workspace, n: int, w: int, h: int, levels: int, stream=None) -> int:
    """Status word of the last search in `workspace` (MTB_OK or MTB_ERR_TIMEOUT)."""
    ws_ptr, ws_bytes = _stage_workspace(workspace)
    return int(lib().mtb_workspace_status(ws_ptr, ws_bytes, n, w, h, levels, _stream(stream)))


def search_kernel(n: int, w: int, h: int, levels: int, ref_idx: int = 0, chained: bool = False) -> str:
    """mtb_search_kernel: "staged" or "items", the search kernel a search of this
    stack runs on the current device (chained: inside a whole-stack call)."""
    rc = int(lib().mtb_search_kernel(n, w, h, levels, ref_idx, 1 if chained else 0))
    if rc < 0:
        raise MtbError(rc, "mtb_search_kernel")
    return "staged" if rc == 1 else "items"


def get_last_status(stream=None) -> int:
    """mtb_get_last_status: MTB_OK or MTB_ERR_TIMEOUT for the last search enqueued
    on `stream` (torch stream or None for the current one); waits for it."""
    return int(lib().mtb_get_last_status(_stream(stream)))


def align_stack_host(images, levels: int, noise_tol: int = 4, ref_idx: int = 0, *, device_workspace=None,
                     out=None, stream=None):
    """Align a host [n, h, w, 3] uint8 stack (torch CPU tensor, ideally pinned);
    copies in, aligns and copies the shifts back.  Returns int32 [n, 2] (CPU):
    `out` if given (a contiguous host int32 [n, 2] tensor), else a new one, pinned
    when the images are."""
    import torch

    n, w, h = _dims(images)
    if images.device.type != "cpu":
        raise ValueError("images must be a CPU tensor (the call copies them to the device)")
    if out is None:
        out = torch.empty((n, 2), dtype=torch.int32, pin_memory=images.is_pinned())
    elif out.device.type != "cpu" or out.dtype != torch.int32 or tuple(out.shape) != (n, 2) or \
            not out.is_contiguous():
        raise ValueError("out must be a contiguous host int32 [n, 2] tensor")
    ws_ptr, ws_bytes = None, 0
    if device_workspace is not None:
        if device_workspace.device.type != "cuda":
            raise ValueError("device_workspace must be a CUDA tensor")
        ws_ptr, ws_bytes = _workspace(device_workspace, device_workspace.device)
    _check(lib().mtb_align_stack_host(images.data_ptr(), n, w, h, levels, noise_tol, ref_idx, out.data_ptr(),
                                      ws_ptr, ws_bytes, _stream(stream)), "mtb_align_stack_host")
    return out


def workspace_views(workspace, n: int, w: int, h: int, levels: int) -> dict:
    """Views of the workspace areas of a stack (torch tensors sharing memory):
    gray[e][l] uint8 [H_l, gray_pitch_l], bits[e][l] int32 [H_l, bits_pitch_l, 2],
    hist int32 [n, levels, 256], median int32 [n, levels], errs int32 [n, levels, 9],
    base / shift int32 [n, levels, 2].  uint32 areas are viewed as int32."""
    import torch

    lay = layout(n, w, h, levels)

    def area(off, count, dtype, shape):
        esz = torch.empty((), dtype=dtype).element_size()
        return workspace[off:off + count * esz].view(dtype).view(*shape)

    gray, bits = [], []
    for e in range(n):
        ge, be = [], []
        for l in range(levels):
            H, gp, bp = lay.height[l], lay.gray_pitch[l], lay.bits_pitch[l]
            go = lay.gray_offset[l] + e * lay.gray_exposure_stride
            bo = lay.bits_offset[l] + e * lay.bits_exposure_stride
            ge.append(area(go, H * gp, torch.uint8, (H, gp)))
            be.append(area(bo, H * bp * 2, torch.int32, (H, bp, 2)))
        gray.append(ge)
        bits.append(be)
    return {
        "layout": lay,
        "gray": gray,
        "bits": bits,
        "hist": area(lay.hist_offset, n * levels * 256, torch.int32, (n, levels, 256)),
        "median": area(lay.median_offset, n * levels, torch.int32, (n, levels)),
        "errs": area(lay.errs_offset, n * levels * 9, torch.int32, (n, levels, 9)),
        "base": area(lay.base_offset, n * levels * 2, torch.int32, (n, levels, 2)),
        "shift": area(lay.shift_offset, n * levels * 2, torch.int32, (n, levels, 2)),
    }


def apply_shifts(images, shifts, fill: int = MTB_FILL_ZERO, *, out=None, stream=None):
    """mtb_apply_shifts: every exposure of images (uint8 CUDA [n, h, w, 3]) moved
    by its (sx, sy) from shifts (int32 CUDA [n, 2]); fill MTB_FILL_ZERO or
    MTB_FILL_EDGE.  Returns out ([n, h, w, 3], allocated here if not given)."""
    import torch

    n, w, h = _cuda_dims(images)
    if shifts.dtype != torch.int32 or shifts.device != images.device or tuple(shifts.shape) != (n, 2):
        raise ValueError("shifts must be an int32 tensor [n, 2] on the images' device")
    if out is None:
        out = torch.empty_like(images)
    elif out.device != images.device or out.dtype != torch.uint8 or out.shape != images.shape or \
            not out.is_contiguous():
        raise ValueError("out must be a contiguous uint8 tensor shaped like images, on their device")
    nbytes = images.numel()
    if out.data_ptr() < images.data_ptr() + nbytes and images.data_ptr() < out.data_ptr() + nbytes:
        raise ValueError("out must not overlap images")
    _check(lib().mtb_apply_shifts(images.data_ptr(), n, w, h, shifts.contiguous().data_ptr(), int(fill),
                                  out.data_ptr(), _stream(stream)), "mtb_apply_shifts")
    return out


_noalloc_fn = None


def align_stack_noalloc(images, levels: int, noise_tol: int = 4, ref_idx: int = 0, *, stream=None):
    """mtb_align_stack_noalloc: the same alignment with the library's fixed device
    scratch array as workspace, for callers that cannot allocate device memory
    while aligning.  The output tensors are the caller's (allocated here by
    torch).  Returns (shifts [n,2], level errors [n,levels,9] viewed as int32,
    level shifts [n,levels,2]).  Stacks larger than MTB_NOALLOC_SCRATCH_BYTES of
    workspace are rejected; calls that overlap on the GPU race on the array."""
    global _noalloc_fn
    import torch

    if _noalloc_fn is None:
        fn = lib().mtb_align_stack_noalloc
        P, I = ctypes.c_void_p, ctypes.c_int
        fn.restype = I
        fn.argtypes = [P, I, I, I, I, I, I, P, P, P, P]
        _noalloc_fn = fn
    n, w, h = _cuda_dims(images)
    dev = images.device
    shifts = torch.empty((n, 2), dtype=torch.int32, device=dev)
    errs = torch.empty((n, levels, 9), dtype=torch.int32, device=dev)
    lsh = torch.empty((n, levels, 2), dtype=torch.int32, device=dev)
    _check(_noalloc_fn(images.data_ptr(), n, w, h, levels, noise_tol, ref_idx, shifts.data_ptr(), errs.data_ptr(),
                       lsh.data_ptr(), _stream(stream)), "mtb_align_stack_noalloc")
    return shifts, errs, lsh


class Batch:
    """Many stacks aligned in one persistent launch (mtb_batch_* of the C ABI).

    stacks: list of dicts with keys images (uint8 CUDA tensor [n, h, w, 3]),
    levels, noise_tol, ref_idx.  Output tensors are allocated here: after run(),
    shifts[i] ([n, 2] int32), level_errs[i] ([n, levels, 9], uint32 viewed as
    int32) and level_shifts[i] ([n, levels, 2]) hold stack i's results."""

    def __init__(self, stacks, level_outputs: bool = True, workspace=None):
        import torch

        self._keep = []
        descs = (StackDesc * len(stacks))()
        self.shifts, self.level_errs, self.level_shifts = [], [], []
        for k, st in enumerate(stacks):
            imgs = st["images"]
            n, w, h = _cuda_dims(imgs)
            L = int(st["levels"])
            dev = imgs.device
            sh = torch.zeros((n, 2), dtype=torch.int32, device=dev)
            er = torch.zeros((n, L, 9), dtype=torch.int32, device=dev) if level_outputs else None
            ls = torch.zeros((n, L, 2), dtype=torch.int32, device=dev) if level_outputs else None
            self.shifts.append(sh)
            self.level_errs.append(er)
            self.level_shifts.append(ls)
            self._keep.append(imgs)
            descs[k] = StackDesc(imgs.data_ptr(), n, w, h, L, int(st.get("noise_tol", 4)), int(st.get("ref_idx", 0)),
                                 sh.data_ptr(), _ptr(er), _ptr(ls))
        self._descs = descs
        handle = ctypes.c_void_p()
        ws_ptr, ws_bytes = None, 0
        if workspace is not None:
            if not stacks:
                raise ValueError("a batch needs at least one stack")
            ws_ptr, ws_bytes = _workspace(workspace, stacks[0]["images"].device)
            self._keep.append(workspace)
        _check(lib().mtb_batch_create(ctypes.cast(descs, ctypes.c_void_p), len(stacks), ws_ptr, ws_bytes,
                                      ctypes.byref(handle)), "mtb_batch_create")
        self._h = handle

    @staticmethod
    def workspace_bytes(stacks) -> int:
        descs = (StackDesc * len(stacks))()
        for k, st in enumerate(stacks):
            n, w, h = _dims(st["images"])
            descs[k] = StackDesc(st["images"].data_ptr(), n, w, h, int(st["levels"]), int(st.get("noise_tol", 4)),
                                 int(st.get("ref_idx", 0)), 1 << 20, None, None)
        return int(lib().mtb_batch_workspace_bytes(ctypes.cast(descs, ctypes.c_void_p), len(stacks)))

    def run(self, stream=None):
        _check(lib().mtb_batch_run(self._h, _stream(stream)), "mtb_batch_run")

    def tune(self, reps: int = 3, stream=None):
        _check(lib().mtb_batch_tune(self._h, reps, _stream(stream)), "mtb_batch_tune")

    def config(self) -> dict:
        v = (ctypes.c_int * 5)()
        _check(lib().mtb_batch_config(self._h, v, 5), "mtb_batch_config")
        return {"pyr_runs_per_cta": v[0], "bit_chunk_words": v[1], "search_waves": v[2], "graph": bool(v[3]),
                "window_kwords": v[4]}

    def set_config(self, pyr_runs_per_cta: int, bit_chunk_words: int, search_waves: int, window_kwords: int):
        """mtb_batch_set_config: pins the settings (each one of the autotuner's candidates)."""
        v = (ctypes.c_int * 5)(pyr_runs_per_cta, bit_chunk_words, search_waves, 0, window_kwords)
        _check(lib().mtb_batch_set_config(self._h, v, 5), "mtb_batch_set_config")

    def status(self, stream=None) -> int:
        return int(lib().mtb_batch_status(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().mtb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SERVER_STATS = ("admitted", "completed", "refused", "failed", "pending", "running", "bytes_in_use", "peak_bytes",
                "peak_running")


def job_bytes(n: int, w: int, h: int, levels: int, noise_tol: int = 4, ref_idx: int = 0) -> int:
    """Device bytes a serving job of this shape is charged (0 if invalid)."""
    j = Job(1 << 20, n, w, h, levels, noise_tol, ref_idx, 1 << 20)
    return int(lib().mtb_job_bytes(ctypes.byref(j)))


class Server:
    """Continuous serving of alignment jobs under a device-memory budget
    (mtb_server_* of the C ABI).  Jobs are stacks in host memory (uint8 CPU
    tensors [n, h, w, 3], pinned for overlapped copies); the native worker admits
    them in arrival order as slots and arena memory free up."""

    def __init__(self, budget_bytes: int, slots: int = 8, copy_streams: int = 1, max_pending: int = 0):
        cfg = ServerConfig(int(budget_bytes), int(slots), int(copy_streams), int(max_pending))
        handle = ctypes.c_void_p()
        _check(lib().mtb_server_create(ctypes.byref(cfg), ctypes.byref(handle)), "mtb_server_create")
        self._h = handle
        self._jobs = {}

    def submit(self, images, levels: int, noise_tol: int = 4, ref_idx: int = 0, out=None) -> int:
        """Queues one stack; returns the job id.  `out` (int32 CPU tensor [n, 2])
        receives the shifts when the job completes.  Raises MtbError with
        MTB_ERR_BUSY when the server refuses the job (back-pressure)."""
        import torch

        if images.device.type != "cpu" or images.dtype != torch.uint8 or not images.is_contiguous():
            raise ValueError("images must be a contiguous uint8 CPU tensor [n, h, w, 3]")
        n, w, h = _dims(images)
        if out is None:
            out = torch.empty((n, 2), dtype=torch.int32)
        elif out.device.type != "cpu" or out.dtype != torch.int32 or tuple(out.shape) != (n, 2) or \
                not out.is_contiguous():
            raise ValueError("out must be a contiguous host int32 [n, 2] tensor")
        job = Job(images.data_ptr(), n, w, h, int(levels), int(noise_tol), int(ref_idx), out.data_ptr())
        jid = ctypes.c_uint64()
        _check(lib().mtb_server_submit(self._h, ctypes.byref(job), ctypes.byref(jid)), "mtb_server_submit")
        self._jobs[jid.value] = (images, out)
        return jid.value

    def poll(self, job_id: int) -> int:
        return int(lib().mtb_server_poll(self._h, job_id))

    def wait(self, job_id: int):
        """Blocks until the job completes; returns (shifts, latency_ms, queue_ms).
        Raises MtbError if the job failed."""
        t = (ctypes.c_double * 2)()
        rc = lib().mtb_server_wait(self._h, job_id, t)
        _, out = self._jobs.pop(job_id, (None, None))
        _check(rc, "mtb_server_wait")
        return out, t[0], t[1]

    def wait_phases(self, job_id: int):
        """Blocks until the job completes; returns (shifts, phases) with phases
        the latency split of mtb_server_wait_phases, in ms: total, queue,
        enqueue, device (copy in, alignment, copy out, callback dispatch),
        callback.  Raises MtbError if the job failed."""
        t = (ctypes.c_double * 5)()
        rc = lib().mtb_server_wait_phases(self._h, job_id, t)
        _, out = self._jobs.pop(job_id, (None, None))
        _check(rc, "mtb_server_wait_phases")
        return out, dict(zip(("total", "queue", "enqueue", "device", "callback"), list(t)))

    def pause(self, paused: bool = True):
        _check(lib().mtb_server_pause(self._h, int(bool(paused))), "mtb_server_pause")

    def stats(self) -> dict:
        v = (ctypes.c_uint64 * len(SERVER_STATS))()
        _check(lib().mtb_server_stats(self._h, v, len(SERVER_STATS)), "mtb_server_stats")
        return dict(zip(SERVER_STATS, (int(x) for x in v)))

    def close(self):
        if getattr(self, "_h", None):
            lib().mtb_server_destroy(self._h)
            self._h = None
            self._jobs.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
