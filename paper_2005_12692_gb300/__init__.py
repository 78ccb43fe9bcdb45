"""GB300 persistent homology of cubical images (Kaji, Sudo, Ahara, "Cubical Ripser").

A thin ctypes binding over ``libcr.so`` (declared in ``include/cr.h``): it
marshals torch tensors (device pointers and the current CUDA stream) into the
C ABI and back.  Every step of the computation runs in the library's CUDA
kernels; there is no CPU fallback -- if the library is not built, every call
raises.

Public API (names as in the C ABI):
  cr_persistence(img, maxdim, keep_zero, topdim_only) -> Pairs
  cr_persistence_f64(img, maxdim, ...)               -> Pairs64 (float64 images)
  cr_persistence_batched(images, maxdim, ...)        -> BatchedPairs
  cr_backward(img, pairs, grad_birth, grad_death)    -> grad image
  cr_backward_batched(...)
  PersistentHomology.apply(img, maxdim)              -> autograd (birth, death)
  build()                                            -> compile libcr.so
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

from ._build import LIB as _LIB_PATH
from ._build import build as _build_lib

CR_OK = 0
CR_ERR_INVALID_ARG = -1
CR_ERR_NAN = -2
CR_ERR_TOO_LARGE = -3
CR_ERR_CAPACITY = -4
CR_ERR_WORKSPACE = -5
CR_ERR_CUDA = -6
CR_ERR_TIMEOUT = -7
CR_ERR_INTERNAL = -8

CR_KEEP_ZERO = 1
CR_TOPDIM_ONLY = 2
CR_LOC_DEATH = 4
CR_PAIR_LOC_DEATH = 2

# launch knobs (cr_tune_set)
CR_TUNE_UF_ITEMS = 0
CR_TUNE_RED_WARPS = 1
CR_TUNE_UF_COMPACT = 2
CR_TUNE_BATCH_THREADS = 3
CR_TUNE_RED_BUDGET = 4
CR_PAIR_ESSENTIAL = 1

PAIR_BYTES = 32
PAIR64_BYTES = 40


class CRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libcr error %d: %s" % (code, msg))
        self.code = code


def build(force: bool = False) -> str:
    """Compile libcr.so for sm_103a."""
    return _build_lib(force=force)


_lib_handle = None


def lib() -> ctypes.CDLL:
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libcr.so is not built (call paper_2005_12692_gb300.build()); "
                               "there is no fallback implementation")
        L = ctypes.CDLL(_LIB_PATH)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        szp = ctypes.POINTER(ctypes.c_size_t)
        vp = ctypes.c_void_p
        L.cr_workspace_size.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_uint32, szp]
        L.cr_workspace_size_typical.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_uint32, szp]
        L.cr_workspace_size_batched.argtypes = [i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, szp]
        L.cr_workspace_size_batched_typical.argtypes = [i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                        ctypes.c_uint32, szp]
        L.cr_persistence.argtypes = [vp, ctypes.c_int, i64p, ctypes.c_int, vp, ctypes.c_int64, i64p, vp,
                                     ctypes.c_size_t, vp, ctypes.c_uint32]
        L.cr_persistence_batched.argtypes = [vp, i64p, i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp,
                                             ctypes.c_int64, vp, i64p, vp, ctypes.c_size_t, vp, ctypes.c_uint32]
        L.cr_backward_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int, szp]
        L.cr_backward.argtypes = [vp, ctypes.c_int, i64p, vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.cr_backward_batched.argtypes = [vp, i64p, i32p, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int64, vp,
                                          vp, vp, vp, ctypes.c_size_t, vp]
        L.cr_pair_table.argtypes = [vp, ctypes.c_int64, ctypes.c_int, i64p, ctypes.c_int, vp, vp]
        L.cr_cell_location.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, i64p,
                                       ctypes.POINTER(ctypes.c_int), i64p, i64p, i64p]
        L.cr_lifetime_image.argtypes = [vp, ctypes.c_int64, ctypes.c_int, i64p, ctypes.c_int, vp, vp]
        L.cr_persistent_histogram_image.argtypes = [vp, ctypes.c_int64, ctypes.c_int, i64p, ctypes.c_int,
                                                    ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                    ctypes.c_double, vp, vp]
        L.cr_profile_enable.argtypes = [ctypes.c_int]
        L.cr_profile_enable.restype = ctypes.c_int
        L.cr_profile_select.argtypes = [ctypes.c_uint32]
        L.cr_profile_select.restype = ctypes.c_int
        L.cr_profile_reset.argtypes = []
        L.cr_profile_reset.restype = None
        L.cr_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                      i64p, ctypes.POINTER(ctypes.c_double)]
        L.cr_profile_read.restype = ctypes.c_int
        L.cr_launch_count.argtypes = []
        L.cr_launch_count.restype = ctypes.c_int64
        L.cr_last_error_detail.restype = ctypes.c_char_p
        L.cr_last_error_detail.argtypes = []
        L.cr_error_string.restype = ctypes.c_char_p
        L.cr_error_string.argtypes = [ctypes.c_int]
        L.cr_workspace_size_f64.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_uint32, ctypes.c_int64,
                                            ctypes.c_int, szp]
        L.cr_workspace_size_f64.restype = ctypes.c_int
        L.cr_persistence_f64.argtypes = [vp, ctypes.c_int, i64p, ctypes.c_int, vp, ctypes.c_int64, i64p, vp,
                                         ctypes.c_size_t, vp, ctypes.c_uint32]
        L.cr_persistence_f64.restype = ctypes.c_int
        L.cr_debug_limits.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        L.cr_debug_limits.restype = ctypes.c_int
        L.cr_tune_set.argtypes = [ctypes.c_int, ctypes.c_int]
        L.cr_tune_set.restype = ctypes.c_int
        L.cr_tune_get.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.cr_tune_get.restype = ctypes.c_int
        for f in ("cr_workspace_size", "cr_workspace_size_typical", "cr_workspace_size_batched",
                  "cr_workspace_size_batched_typical", "cr_persistence", "cr_persistence_batched",
                  "cr_backward_workspace_size", "cr_backward", "cr_backward_batched", "cr_cell_location",
                  "cr_lifetime_image", "cr_persistent_histogram_image", "cr_pair_table"):
            getattr(L, f).restype = ctypes.c_int
        _lib_handle = L
    return _lib_handle


def _check(rc: int):
    if rc != CR_OK:
        msg = lib().cr_error_string(rc).decode()
        if rc == CR_ERR_WORKSPACE:
            msg += " (" + lib().cr_last_error_detail().decode() + ")"
        raise CRError(rc, msg)


def error_string(code: int) -> str:
    return lib().cr_error_string(code).decode()


def cr_tune_set(knob: int, value: int) -> None:
    """Set a launch knob of the library (see include/cr.h); raises on an unknown knob or a bad value."""
    _check(lib().cr_tune_set(int(knob), int(value)))


def debug_limits(barrier_polls: int = 0, reduce_iters: int = 0, barrier_unsatisfiable: bool = False) -> None:
    """Lower the limits of the library's bounded device waits (tests of the
    error paths; include/cr.h, cr_debug_limits).  No arguments restores the
    defaults."""
    _check(lib().cr_debug_limits(int(barrier_polls), int(reduce_iters), int(bool(barrier_unsatisfiable))))


def cr_tune_get(knob: int) -> int:
    v = ctypes.c_int(0)
    _check(lib().cr_tune_get(int(knob), ctypes.byref(v)))
    return v.value


def cell_location(L: int, dim: int, shape: Sequence[int]):
    """(m, x, y, z) of the cube (dim, L) of an image of this shape."""
    sh = (ctypes.c_int64 * len(shape))(*[int(s) for s in shape])
    m = ctypes.c_int()
    x, y, z = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().cr_cell_location(int(L), int(dim), len(shape), sh, ctypes.byref(m), ctypes.byref(x),
                                  ctypes.byref(y), ctypes.byref(z)))
    return m.value, x.value, y.value, z.value


# ---------------------------------------------------------------------------
# results
# ---------------------------------------------------------------------------
@dataclass
class Pairs:
    """Persistence pairs on the device, in the library's canonical order
    (dim, birth, birth_cell).  ``raw`` is the (n, 32) byte view of cr_pair."""
    raw: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.raw.shape[0])

    def _f(self, dtype, col):
        return self.raw.view(dtype)[:, col] if self.n else torch.empty(0, dtype=dtype, device=self.raw.device)

    @property
    def dim(self):
        return self._f(torch.int32, 0)

    @property
    def birth(self):
        return self._f(torch.float32, 1)

    @property
    def death(self):
        return self._f(torch.float32, 2)

    @property
    def flags(self):
        return self._f(torch.int32, 3)

    @property
    def birth_cell(self):
        return self._f(torch.int64, 2)

    @property
    def death_cell(self):
        return self._f(torch.int64, 3)

    def numpy(self):
        import numpy as np
        dt = np.dtype([("dim", np.int32), ("birth", np.float32), ("death", np.float32), ("flags", np.uint32),
                       ("birth_cell", np.int64), ("death_cell", np.int64)])
        b = self.raw.detach().cpu().numpy().tobytes()
        return np.frombuffer(b, dtype=dt).copy()


@dataclass
class Pairs64:
    """Pairs of a float64 image (cr_pair64), in the same canonical order as
    ``Pairs``.  ``raw`` is the (n, 40) byte view."""
    raw: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.raw.shape[0])

    def _f(self, dtype, lo, hi):
        if not self.n:
            return torch.empty(0, dtype=dtype, device=self.raw.device)
        return self.raw[:, lo:hi].contiguous().view(dtype).reshape(-1)

    @property
    def dim(self):
        return self._f(torch.int32, 0, 4)

    @property
    def flags(self):
        return self._f(torch.int32, 4, 8)

    @property
    def birth(self):
        return self._f(torch.float64, 8, 16)

    @property
    def death(self):
        return self._f(torch.float64, 16, 24)

    @property
    def birth_cell(self):
        return self._f(torch.int64, 24, 32)

    @property
    def death_cell(self):
        return self._f(torch.int64, 32, 40)

    def numpy(self):
        import numpy as np
        dt = np.dtype([("dim", np.int32), ("flags", np.uint32), ("birth", np.float64), ("death", np.float64),
                       ("birth_cell", np.int64), ("death_cell", np.int64)])
        b = self.raw.detach().cpu().numpy().tobytes()
        return np.frombuffer(b, dtype=dt).copy()


@dataclass
class BatchedPairs:
    pairs: Pairs
    offsets: torch.Tensor  # int64[n_images+1] on the device

    def image(self, i: int) -> Pairs:
        o = self.offsets.cpu()
        return Pairs(self.pairs.raw[int(o[i]):int(o[i + 1])])


# ---------------------------------------------------------------------------
# workspace cache
# ---------------------------------------------------------------------------
class _Workspace:
    def __init__(self):
        self.buf: Optional[torch.Tensor] = None

    def get(self, nbytes: int, device) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != device:
            self.buf = None
            torch.cuda.empty_cache() if nbytes > (1 << 30) else None
            self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        return self.buf


_WS = _Workspace()
_BWS = _Workspace()


def _stream_ptr(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _flags(keep_zero: bool, topdim_only: bool, location: str = "birth") -> int:
    if location not in ("birth", "death"):
        raise ValueError("location must be 'birth' or 'death'")
    return ((CR_KEEP_ZERO if keep_zero else 0) | (CR_TOPDIM_ONLY if topdim_only else 0) |
            (CR_LOC_DEATH if location == "death" else 0))


def _require_cuda_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor (the library has no CPU path)" % name)
    if t.dtype != torch.float32:
        raise ValueError("%s must be float32" % name)
    return t.contiguous()


def _num_cells(shape) -> int:
    n = 1
    for s in shape:
        n *= 2 * int(s) - 1
    return n


def cr_persistence(img: torch.Tensor, maxdim: Optional[int] = None, keep_zero: bool = False,
                   topdim_only: bool = False, capacity: Optional[int] = None, location: str = "birth") -> Pairs:
    """Persistence pairs of one 1D/2D/3D float32 CUDA image (Sec. 2 of the paper).

    ``maxdim`` defaults to ndim-1 (all dimensions).  ``location="death"``
    records the death cell as each pair's location (CR_LOC_DEATH), which
    ``pair_table`` and the localised images then follow.  Returns pairs on the
    image's device."""
    img = _require_cuda_f32(img, "img")
    nd = img.dim()
    if nd < 1 or nd > 3:
        raise ValueError("img must be 1D, 2D or 3D")
    if maxdim is None:
        maxdim = nd - 1
    flags = _flags(keep_zero, topdim_only, location)
    shape = (ctypes.c_int64 * nd)(*img.shape)
    L = lib()
    sz = ctypes.c_size_t()
    _check(L.cr_workspace_size_typical(nd, shape, int(maxdim), flags, ctypes.byref(sz)))
    if capacity is None:
        capacity = _num_cells(img.shape) // 2 + 2 if keep_zero else max(4096, img.numel() // 4 + 16)
    out = torch.empty((int(capacity), PAIR_BYTES), dtype=torch.uint8, device=img.device)
    n = ctypes.c_int64(0)
    worst = False
    for _attempt in range(4):
        ws = _WS.get(sz.value, img.device)
        rc = L.cr_persistence(ctypes.c_void_p(img.data_ptr()), nd, shape, int(maxdim),
                              ctypes.c_void_p(out.data_ptr()), out.shape[0], ctypes.byref(n),
                              ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(img.device), flags)
        if rc == CR_ERR_CAPACITY:
            out = torch.empty((int(n.value) + 16, PAIR_BYTES), dtype=torch.uint8, device=img.device)
            continue
        if rc == CR_ERR_WORKSPACE and not worst:
            worst = True
            _check(L.cr_workspace_size(nd, shape, int(maxdim), flags, ctypes.byref(sz)))
            continue
        if rc == CR_ERR_WORKSPACE and worst:
            sz.value = int(sz.value * 2)
            continue
        _check(rc)
        return Pairs(out[: n.value])
    _check(rc)
    raise AssertionError("unreachable")


def cr_persistence_f64(img: torch.Tensor, maxdim: Optional[int] = None, keep_zero: bool = False,
                       topdim_only: bool = False, capacity: Optional[int] = None,
                       location: str = "birth") -> Pairs64:
    """Persistence pairs of one 1D/2D/3D float64 CUDA image, with float64
    births and deaths (the library ranks the values on the device and runs
    the float32 path on the ranks; include/cr.h, cr_persistence_f64)."""
    if not isinstance(img, torch.Tensor) or not img.is_cuda:
        raise ValueError("img must be a CUDA tensor (the library has no CPU path)")
    if img.dtype != torch.float64:
        raise ValueError("img must be float64")
    img = img.contiguous()
    nd = img.dim()
    if nd < 1 or nd > 3:
        raise ValueError("img must be 1D, 2D or 3D")
    if maxdim is None:
        maxdim = nd - 1
    flags = _flags(keep_zero, topdim_only, location)
    shape = (ctypes.c_int64 * nd)(*img.shape)
    L = lib()
    if capacity is None:
        capacity = _num_cells(img.shape) // 2 + 2 if keep_zero else max(4096, img.numel() // 4 + 16)
    n = ctypes.c_int64(0)
    worst, scale = False, 1
    for _attempt in range(6):
        sz = ctypes.c_size_t()
        _check(L.cr_workspace_size_f64(nd, shape, int(maxdim), flags, int(capacity), 0 if worst else 1,
                                       ctypes.byref(sz)))
        out = torch.empty((int(capacity), PAIR64_BYTES), dtype=torch.uint8, device=img.device)
        ws = _WS.get(sz.value * scale, img.device)
        rc = L.cr_persistence_f64(ctypes.c_void_p(img.data_ptr()), nd, shape, int(maxdim),
                                  ctypes.c_void_p(out.data_ptr()), int(capacity), ctypes.byref(n),
                                  ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(img.device), flags)
        if rc == CR_ERR_CAPACITY:
            capacity = int(n.value) + 16
            continue
        if rc == CR_ERR_WORKSPACE:
            if worst:
                scale *= 2
            worst = True
            continue
        _check(rc)
        return Pairs64(out[: n.value])
    _check(rc)
    raise AssertionError("unreachable")


def _pack(images: Sequence[torch.Tensor]):
    nd = images[0].dim()
    for t in images:
        if t.dim() != nd:
            raise ValueError("all images of a batch must have the same ndim")
    shapes = [tuple(int(s) for s in t.shape) for t in images]
    flat = torch.cat([_require_cuda_f32(t, "image").reshape(-1) for t in images])
    offs = [0]
    for s in shapes:
        n = 1
        for v in s:
            n *= v
        offs.append(offs[-1] + n)
    return flat, shapes, offs, nd


def cr_persistence_batched(images, maxdim: Optional[int] = None, keep_zero: bool = False,
                           topdim_only: bool = False, shapes=None, offsets=None,
                           capacity: Optional[int] = None, location: str = "birth") -> BatchedPairs:
    """Persistence of many images in one pass.  ``images`` is a list of CUDA
    float32 tensors (same ndim, any shapes), or a packed 1D tensor together
    with ``shapes`` (list of tuples) and ``offsets`` (list of n+1 ints)."""
    if isinstance(images, torch.Tensor) and shapes is not None:
        flat = _require_cuda_f32(images, "images")
        shapes = [tuple(int(v) for v in s) for s in shapes]
        nd = len(shapes[0])
        offs = list(offsets) if offsets is not None else None
        if offs is None:
            offs = [0]
            for s in shapes:
                n = 1
                for v in s:
                    n *= v
                offs.append(offs[-1] + n)
    else:
        flat, shapes, offs, nd = _pack(list(images))
    nimg = len(shapes)
    if maxdim is None:
        maxdim = nd - 1
    flags = _flags(keep_zero, topdim_only, location)
    sh = (ctypes.c_int32 * (nimg * nd))(*[v for s in shapes for v in s])
    of = (ctypes.c_int64 * (nimg + 1))(*offs)
    L = lib()
    sz = ctypes.c_size_t()
    _check(L.cr_workspace_size_batched_typical(sh, nimg, nd, int(maxdim), flags, ctypes.byref(sz)))
    if capacity is None:
        cells = sum(_num_cells(s) for s in shapes)
        capacity = cells // 2 + nimg + 2 if keep_zero else max(4096, offs[-1] // 4 + 16 * nimg)
    out = torch.empty((int(capacity), PAIR_BYTES), dtype=torch.uint8, device=flat.device)
    poffs = torch.empty(nimg + 1, dtype=torch.int64, device=flat.device)
    n = ctypes.c_int64(0)
    worst = False
    for _attempt in range(4):
        ws = _WS.get(sz.value, flat.device)
        rc = L.cr_persistence_batched(ctypes.c_void_p(flat.data_ptr()), of, sh, nimg, nd, int(maxdim),
                                      ctypes.c_void_p(out.data_ptr()), out.shape[0],
                                      ctypes.c_void_p(poffs.data_ptr()), ctypes.byref(n),
                                      ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(flat.device), flags)
        if rc == CR_ERR_CAPACITY:
            out = torch.empty((int(n.value) + 16, PAIR_BYTES), dtype=torch.uint8, device=flat.device)
            continue
        if rc == CR_ERR_WORKSPACE and not worst:
            worst = True
            _check(L.cr_workspace_size_batched(sh, nimg, nd, int(maxdim), flags, ctypes.byref(sz)))
            continue
        if rc == CR_ERR_WORKSPACE and worst:
            sz.value = int(sz.value * 2)
            continue
        _check(rc)
        return BatchedPairs(Pairs(out[: n.value]), poffs)
    _check(rc)
    raise AssertionError("unreachable")


def cr_backward(img: torch.Tensor, pairs: Pairs, grad_birth: torch.Tensor, grad_death: torch.Tensor) -> torch.Tensor:
    """Image gradient from per-pair dL/dbirth, dL/ddeath (routed to the vertex
    that attains each cube's value)."""
    img = _require_cuda_f32(img, "img")
    nd = img.dim()
    shape = (ctypes.c_int64 * nd)(*img.shape)
    gb = _require_cuda_f32(grad_birth.reshape(-1), "grad_birth")
    gd = _require_cuda_f32(grad_death.reshape(-1), "grad_death")
    L = lib()
    sz = ctypes.c_size_t()
    _check(L.cr_backward_workspace_size(pairs.n, 1, ctypes.byref(sz)))
    ws = _BWS.get(sz.value, img.device)
    grad = torch.empty_like(img)
    _check(L.cr_backward(ctypes.c_void_p(img.data_ptr()), nd, shape, ctypes.c_void_p(pairs.raw.data_ptr()), pairs.n,
                         ctypes.c_void_p(gb.data_ptr()), ctypes.c_void_p(gd.data_ptr()),
                         ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                         _stream_ptr(img.device)))
    return grad


def cr_backward_batched(flat: torch.Tensor, shapes, offsets, bp: BatchedPairs, grad_birth: torch.Tensor,
                        grad_death: torch.Tensor) -> torch.Tensor:
    flat = _require_cuda_f32(flat, "images")
    nimg = len(shapes)
    nd = len(shapes[0])
    sh = (ctypes.c_int32 * (nimg * nd))(*[int(v) for s in shapes for v in s])
    of = (ctypes.c_int64 * (nimg + 1))(*[int(v) for v in offsets])
    gb = _require_cuda_f32(grad_birth.reshape(-1), "grad_birth")
    gd = _require_cuda_f32(grad_death.reshape(-1), "grad_death")
    L = lib()
    sz = ctypes.c_size_t()
    _check(L.cr_backward_workspace_size(bp.pairs.n, nimg, ctypes.byref(sz)))
    ws = _BWS.get(sz.value, flat.device)
    grad = torch.empty_like(flat)
    _check(L.cr_backward_batched(ctypes.c_void_p(flat.data_ptr()), of, sh, nimg, nd,
                                 ctypes.c_void_p(bp.pairs.raw.data_ptr()), ctypes.c_void_p(bp.offsets.data_ptr()),
                                 bp.pairs.n, ctypes.c_void_p(gb.data_ptr()), ctypes.c_void_p(gd.data_ptr()),
                                 ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                 _stream_ptr(flat.device)))
    return grad


_LOCATIONS = {None: -1, "pairs": -1, "birth": 0, "death": 1}


def pair_table(shape: Sequence[int], pairs: Pairs, location: Optional[str] = None) -> torch.Tensor:
    """The pairs as the paper's (n, 6) float64 table (dim, birth, death, x, y, z)
    (Sec. 4, Ex. 4.1), located at the birth or death cell; ``None`` follows what
    each pair records (the ``location`` given to ``cr_persistence``)."""
    shape = tuple(int(v) for v in shape)
    nd = len(shape)
    out = torch.empty((pairs.n, 6), dtype=torch.float64, device=pairs.raw.device)
    sh = (ctypes.c_int64 * nd)(*shape)
    _check(lib().cr_pair_table(ctypes.c_void_p(pairs.raw.data_ptr() if pairs.n else 0), pairs.n, nd, sh,
                               _LOCATIONS[location], ctypes.c_void_p(out.data_ptr() if pairs.n else 0),
                               _stream_ptr(out.device)))
    return out


def lifetime_image(shape: Sequence[int], pairs: Pairs, location: Optional[str] = None) -> torch.Tensor:
    """Lifetime channels (ndim, *shape) of the lifetime enhanced image (Sec. 4):
    per dimension d, the largest lifetime of the finite pairs of dimension d
    located at each voxel (anchor of the birth or death cell; ``None`` follows
    what each pair records), 0 elsewhere."""
    shape = tuple(int(v) for v in shape)
    nd = len(shape)
    out = torch.empty((nd,) + shape, dtype=torch.float32, device=pairs.raw.device)
    sh = (ctypes.c_int64 * nd)(*shape)
    _check(lib().cr_lifetime_image(ctypes.c_void_p(pairs.raw.data_ptr() if pairs.n else 0), pairs.n, nd, sh,
                                   _LOCATIONS[location], ctypes.c_void_p(out.data_ptr()),
                                   _stream_ptr(out.device)))
    return out


def lifetime_enhanced_image(img: torch.Tensor, pairs: Optional[Pairs] = None, location: Optional[str] = None):
    """The image stacked with its lifetime channels: (1 + ndim, *shape)."""
    img = _require_cuda_f32(img, "img")
    if pairs is None:
        pairs = cr_persistence(img, location=location or "birth")
    return torch.cat([img.unsqueeze(0), lifetime_image(img.shape, pairs, location)], dim=0)


def persistent_histogram_image(shape: Sequence[int], pairs: Pairs, nb: int, birth_range, nl: int,
                               max_lifetime: float, location: Optional[str] = None) -> torch.Tensor:
    """Persistent histogram image (Sec. 4): channel (d * nb + i) * nl + j counts,
    per voxel, the finite pairs of dimension d located there with birth in bin i
    of ``birth_range`` and lifetime in bin j of [0, max_lifetime)."""
    shape = tuple(int(v) for v in shape)
    nd = len(shape)
    out = torch.empty((nd * nb * nl,) + shape, dtype=torch.float32, device=pairs.raw.device)
    sh = (ctypes.c_int64 * nd)(*shape)
    _check(lib().cr_persistent_histogram_image(ctypes.c_void_p(pairs.raw.data_ptr() if pairs.n else 0), pairs.n,
                                               nd, sh, _LOCATIONS[location], int(nb), float(birth_range[0]),
                                               float(birth_range[1]), int(nl), float(max_lifetime),
                                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(out.device)))
    return out


class PersistentHomology(torch.autograd.Function):
    """(birth, death) of every pair as differentiable outputs; dims and cells
    are returned as non-differentiable tensors.  Backward calls cr_backward."""

    @staticmethod
    def forward(ctx, img: torch.Tensor, maxdim: Optional[int] = None):
        pairs = cr_persistence(img.detach(), maxdim=maxdim)
        ctx.save_for_backward(img)
        ctx.pairs = pairs
        birth = pairs.birth.clone()
        death = pairs.death.clone()
        dim = pairs.dim.clone()
        ctx.mark_non_differentiable(dim)
        return birth, death, dim

    @staticmethod
    def backward(ctx, gb, gd, _gdim):
        (img,) = ctx.saved_tensors
        if gb is None:
            gb = torch.zeros(ctx.pairs.n, dtype=torch.float32, device=img.device)
        if gd is None:
            gd = torch.zeros(ctx.pairs.n, dtype=torch.float32, device=img.device)
        gd = torch.where(torch.isfinite(ctx.pairs.death), gd, torch.zeros_like(gd))
        return cr_backward(img.detach(), ctx.pairs, gb.float(), gd.float()), None


__all__ = [
    "build", "lib", "cr_persistence", "cr_persistence_batched", "cr_backward", "cr_backward_batched",
    "PersistentHomology", "Pairs", "BatchedPairs", "CRError", "cell_location", "error_string",
    "CR_KEEP_ZERO", "CR_TOPDIM_ONLY", "CR_LOC_DEATH", "pair_table", "cr_tune_set", "cr_tune_get", "cr_persistence_f64",
    "Pairs64",
    "CR_TUNE_UF_ITEMS", "CR_TUNE_RED_WARPS", "CR_TUNE_UF_COMPACT", "CR_TUNE_BATCH_THREADS", "CR_TUNE_RED_BUDGET",
    "debug_limits",
]
