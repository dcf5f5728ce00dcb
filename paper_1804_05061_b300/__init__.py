"""B300-native SRWCR (spatially region-weighted correlation ratio) registration.

Thin ctypes binding over ``libsrwcr.so`` (C ABI in ``include/srwcr.h``):
argument marshalling only.  Every step of the SRWCR value and gradient runs
in the library's CUDA kernels; PyTorch supplies device memory and streams.
There is no CPU fallback: if the library cannot be loaded, importing the
engine raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsrwcr.so")
_lib = None

STORAGE = {"f32": 0, "bf16": 1}
ROLE = {"mas_b": 0, "mas_a": 1}   # which image is binned (Sec. II-E)
SPATIAL = {"bspline": 0, "boxcar": 1}  # w(r, x): Eq. (7) or Eq. (6)
STATUS = {0: "SRWCR_OK", 1: "SRWCR_EINVAL", 2: "SRWCR_ENOMEM", 3: "SRWCR_ECUDA",
          4: "SRWCR_ENUMERIC", 5: "SRWCR_ELINESEARCH", 6: "SRWCR_ETIMEOUT",
          7: "SRWCR_ENOTCONVERGED"}

# Every symbol the header exports (checked by the CPU test suite).
EXPORTS = ("srwcr_create", "srwcr_destroy", "srwcr_last_error", "srwcr_level_info",
           "srwcr_value", "srwcr_value_and_grad", "srwcr_value_and_grad_async",
           "srwcr_value_and_grad_host", "srwcr_forward", "srwcr_backward",
           "srwcr_region_stats", "srwcr_debug_bins", "srwcr_debug_warp",
           "srwcr_lbfgs_default_opts", "srwcr_register", "srwcr_set_profiling",
           "srwcr_profile_read", "srwcr_value_noalloc", "srwcr_autotune",
           "srwcr_batch_create", "srwcr_batch_create_levels", "srwcr_batch_destroy", "srwcr_batch_info",
           "srwcr_batch_layout", "srwcr_batch_buffers", "srwcr_batch_value_and_grad",
           "srwcr_batch_sync", "srwcr_batch_register", "srwcr_bending_energy",
           "srwcr_rigid_value_and_grad", "srwcr_rigid_to_ffd", "srwcr_rigid_register",
           "srwcr_debug_warp_grad", "srwcr_level_images", "srwcr_refine",
           "srwcr_lbfgs_direction", "srwcr_debug_fixed_point", "srwcr_tile_order")


class SrwcrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("dims", ctypes.c_int * 3),
                ("ffd_spacing", ctypes.c_int * 3), ("sbin_intervals", ctypes.c_int * 3),
                ("n_intensity_bins", ctypes.c_int), ("storage", ctypes.c_int),
                ("pyramid_levels", ctypes.c_int), ("tile", ctypes.c_int * 3),
                ("bins_per_pass", ctypes.c_int), ("role", ctypes.c_int),
                ("finalize_lanes", ctypes.c_int), ("spatial", ctypes.c_int),
                ("keep_warp", ctypes.c_int)]


class LevelDesc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 3), ("ffd_nodes", ctypes.c_int * 3),
                ("sbins", ctypes.c_int * 3), ("n_voxels", ctypes.c_int64),
                ("n_params", ctypes.c_int64), ("n_regions", ctypes.c_int64),
                ("tile", ctypes.c_int * 3), ("kernel_path", ctypes.c_int),
                ("finalize_lanes", ctypes.c_int)]


class LbfgsOpts(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("max_iter", ctypes.c_int * 4),
                ("stable_window", ctypes.c_int), ("stable_rtol", ctypes.c_double),
                ("max_ls", ctypes.c_int), ("c1", ctypes.c_double), ("c2", ctypes.c_double),
                ("penalty_weight", ctypes.c_double), ("start_jitter", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class Report(ctypes.Structure):
    _fields_ = [("levels_run", ctypes.c_int), ("iterations", ctypes.c_int * 4),
                ("evaluations", ctypes.c_int * 4), ("final_value", ctypes.c_double * 4),
                ("status", ctypes.c_int * 4)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int), ("launches_per_eval", ctypes.c_int),
                ("n_params_total", ctypes.c_int64), ("n_voxels_total", ctypes.c_int64),
                ("work_items", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("finalize_lanes", ctypes.c_int)]


def library_path() -> str:
    return _LIB_PATH


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libsrwcr.so (building it with nvcc if it is absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libsrwcr.so not found at {_LIB_PATH}; run "
                          "`python -m paper_1804_05061_b300.build`")
    L = ctypes.CDLL(_LIB_PATH)
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    st = ctypes.c_int
    sigs = {
        "srwcr_create": (st, [ctypes.POINTER(Config), vp, vp, ctypes.c_int, vp,
                              ctypes.POINTER(vp)]),
        "srwcr_destroy": (None, [vp]),
        "srwcr_last_error": (ctypes.c_char_p, []),
        "srwcr_level_info": (st, [vp, ctypes.c_int, ctypes.POINTER(LevelDesc)]),
        "srwcr_value": (st, [vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double)]),
        "srwcr_value_and_grad": (st, [vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double), vp]),
        "srwcr_value_and_grad_async": (st, [vp, ctypes.c_int, vp, vp, vp]),
        "srwcr_value_and_grad_host": (st, [vp, ctypes.c_int, vp,
                                           ctypes.POINTER(ctypes.c_double), vp]),
        "srwcr_forward": (st, [vp, ctypes.c_int, vp, vp]),
        "srwcr_backward": (st, [vp, ctypes.c_int, vp, vp, vp]),
        "srwcr_region_stats": (st, [vp, ctypes.c_int, vp, i64p]),
        "srwcr_debug_bins": (st, [vp, ctypes.c_int, vp]),
        "srwcr_debug_warp": (st, [vp, ctypes.c_int, vp, vp]),
        "srwcr_debug_warp_grad": (st, [vp, ctypes.c_int, vp, vp]),
        "srwcr_level_images": (st, [vp, ctypes.c_int, vp, vp]),
        "srwcr_refine": (st, [vp, ctypes.c_int, vp, vp]),
        "srwcr_lbfgs_direction": (st, [vp, ctypes.c_int64, ctypes.c_int, vp, vp, vp, vp]),
        "srwcr_debug_fixed_point": (st, [vp, ctypes.c_int64, vp, vp, ctypes.c_int64, vp, vp,
                                         ctypes.c_int]),
        "srwcr_tile_order": (st, [vp, vp, vp, vp, vp]),
        "srwcr_lbfgs_default_opts": (None, [ctypes.POINTER(LbfgsOpts)]),
        "srwcr_set_profiling": (st, [vp, ctypes.c_int]),
        "srwcr_profile_read": (st, [vp, vp, vp, i64p, ctypes.c_int]),
        "srwcr_register": (st, [vp, vp, ctypes.c_int, ctypes.POINTER(LbfgsOpts),
                                ctypes.POINTER(Report)]),
        "srwcr_value_noalloc": (st, [ctypes.POINTER(Config), vp, vp, vp, vp, vp]),
        "srwcr_autotune": (st, [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "srwcr_batch_create": (st, [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]),
        "srwcr_batch_create_levels": (st, [vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)]),
        "srwcr_batch_destroy": (None, [vp]),
        "srwcr_batch_info": (st, [vp, ctypes.POINTER(BatchDesc)]),
        "srwcr_batch_layout": (st, [vp, vp, vp]),
        "srwcr_batch_buffers": (st, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(vp)]),
        "srwcr_batch_value_and_grad": (st, [vp, ctypes.c_int]),
        "srwcr_batch_sync": (st, [vp, vp]),
        "srwcr_batch_register": (st, [vp, ctypes.POINTER(LbfgsOpts), ctypes.c_int, vp, vp, vp,
                                      vp]),
        "srwcr_bending_energy": (st, [vp, ctypes.c_int, vp, vp, vp, ctypes.c_float]),
        "srwcr_rigid_value_and_grad": (st, [vp, ctypes.c_int, vp,
                                            ctypes.POINTER(ctypes.c_double), vp]),
        "srwcr_rigid_to_ffd": (st, [vp, ctypes.c_int, vp, vp]),
        "srwcr_rigid_register": (st, [vp, vp, ctypes.c_int, ctypes.POINTER(LbfgsOpts),
                                      ctypes.POINTER(Report)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise SrwcrError(status, load().srwcr_last_error().decode(errors="replace"))


def _ptr(t) -> int:
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class LevelInfo:
    dims: tuple
    ffd_nodes: tuple
    sbins: tuple
    n_voxels: int
    n_params: int
    n_regions: int
    tile: tuple
    kernel_path: int  # 1 = row-parallel kernels, 0 = general kernels
    finalize_lanes: int  # lanes per spatial bin in the finalisation


class SRWCR:
    """One fixed/moving pair on the current CUDA device.

    fixed, moving: float32 arrays shaped (ny, nx) or (nz, ny, nx), as NumPy
    (host) arrays or CUDA tensors.  ``sbin_intervals`` K > 0 puts K+3 cubic
    B-spline spatial bins per axis; 0 puts them on the FFD grid.
    """

    def __init__(self, fixed, moving, ffd_spacing: Sequence[int],
                 sbin_intervals: Sequence[int] = (0, 0, 0), n_bins: int = 32,
                 storage: str = "f32", pyramid_levels: int = 1,
                 tile: Optional[Sequence[int]] = None, stream=None, bins_per_pass: int = 0,
                 role: str = "mas_b", finalize_lanes: int = 0, spatial: str = "bspline",
                 keep_warp: int = 0):
        import torch
        self._torch = torch
        lib = load()
        shape = tuple(fixed.shape)
        if tuple(moving.shape) != shape or len(shape) not in (2, 3):
            raise ValueError("fixed and moving must share a 2-D or 3-D shape")
        ndim = len(shape)
        cfg = Config()
        cfg.ndim = ndim
        dims = list(reversed(shape)) + [1] * (3 - ndim)
        for d in range(3):
            cfg.dims[d] = int(dims[d])
            cfg.ffd_spacing[d] = int(ffd_spacing[d]) if d < len(ffd_spacing) else 1
            cfg.sbin_intervals[d] = int(sbin_intervals[d]) if d < len(sbin_intervals) else 0
            cfg.tile[d] = int(tile[d]) if tile is not None and d < len(tile) else 0
        cfg.n_intensity_bins = int(n_bins)
        cfg.storage = STORAGE[storage]
        cfg.pyramid_levels = int(pyramid_levels)
        cfg.bins_per_pass = int(bins_per_pass)
        cfg.role = ROLE[role]
        cfg.finalize_lanes = int(finalize_lanes)
        cfg.spatial = SPATIAL[spatial]
        cfg.keep_warp = int(keep_warp)
        self.cfg = cfg
        self.ndim = ndim
        self.storage = storage
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        on_dev = isinstance(fixed, torch.Tensor) and fixed.is_cuda
        if on_dev:
            f = fixed.detach().to(torch.float32).contiguous()
            m = moving.detach().to(torch.float32).contiguous()
            pf, pm = _ptr(f), _ptr(m)
        else:
            f = np.ascontiguousarray(fixed, dtype=np.float32)
            m = np.ascontiguousarray(moving, dtype=np.float32)
            pf, pm = f.ctypes.data_as(ctypes.c_void_p), m.ctypes.data_as(ctypes.c_void_p)
        handle = ctypes.c_void_p()
        _check(lib.srwcr_create(ctypes.byref(cfg), pf, pm, 1 if on_dev else 0,
                                ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle)))
        self._h = handle
        self._gen = [0] * cfg.pyramid_levels
        self.levels = [self.level_info(l) for l in range(cfg.pyramid_levels)]

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().srwcr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- geometry ----------------------------------------------------------
    def level_info(self, level: int = 0) -> LevelInfo:
        d = LevelDesc()
        _check(load().srwcr_level_info(self._h, level, ctypes.byref(d)))
        return LevelInfo(tuple(d.dims), tuple(d.ffd_nodes), tuple(d.sbins), d.n_voxels,
                         d.n_params, d.n_regions, tuple(d.tile), d.kernel_path,
                         d.finalize_lanes)

    def coef_shape(self, level: int = 0):
        n = self.levels[level].ffd_nodes
        return (self.ndim, n[1], n[0]) if self.ndim == 2 else (self.ndim, n[2], n[1], n[0])

    def zeros(self, level: int = 0):
        return self._torch.zeros(self.coef_shape(level), dtype=self._torch.float32,
                                 device=self.device)

    def _dev(self, t, n, dtype, name, inplace=False):
        """t checked as a CUDA tensor of this engine's device holding n values
        of dtype.  The library takes plain pointers and reads or writes
        exactly n values: a buffer it writes (inplace) must be contiguous
        itself; an input is passed as a contiguous copy if it is not."""
        torch = self._torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype):
            raise TypeError(f"{name} must be a {dtype} CUDA tensor")
        if t.device != self.device:
            raise ValueError(f"{name} is on {t.device}, the engine on {self.device}")
        if t.numel() != n:
            raise ValueError(f"{name} has {t.numel()} entries, needs {n}")
        if inplace and not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous (the library writes it in place)")
        return t if inplace else t.contiguous()

    def _c(self, c, level, inplace=False):
        return self._dev(c, self.levels[level].n_params, self._torch.float32,
                         f"c (level {level})", inplace)

    def _host(self, a, level, name, writes=False):
        """a checked as a C-contiguous float32 NumPy array of the level's
        coefficient count (the library copies exactly that many values)."""
        if not (isinstance(a, np.ndarray) and a.dtype == np.float32):
            raise TypeError(f"{name} must be a float32 NumPy array")
        n = self.levels[level].n_params
        if a.size != n:
            raise ValueError(f"{name} has {a.size} entries, level {level} needs {n}")
        if not a.flags.c_contiguous:
            raise ValueError(f"{name} must be C-contiguous")
        if writes and not a.flags.writeable:
            raise ValueError(f"{name} is read-only")
        return a

    # -- evaluation --------------------------------------------------------
    def value(self, c, level: int = 0) -> float:
        c = self._c(c, level)
        D = ctypes.c_double()
        _check(load().srwcr_value(self._h, level, _ptr(c), ctypes.byref(D)))
        self._gen[level] += 1
        return D.value

    def value_and_grad(self, c, level: int = 0, out=None):
        c = self._c(c, level)
        if out is None:
            g = self._torch.empty_like(c)
        else:
            g = self._dev(out, c.numel(), self._torch.float32, "out", inplace=True)
        D = ctypes.c_double()
        _check(load().srwcr_value_and_grad(self._h, level, _ptr(c), ctypes.byref(D), _ptr(g)))
        self._gen[level] += 1
        return D.value, g

    def value_and_grad_async(self, c, D_out, g_out, level: int = 0):
        """Queue value+gradient on the stream; D_out is a float64 CUDA scalar.
        Every buffer is used in place (the call may be captured in a graph),
        so c must be contiguous too."""
        t = self._torch
        c = self._c(c, level, inplace=True)
        D_out = self._dev(D_out, 1, t.float64, "D_out", inplace=True)
        g_out = self._dev(g_out, c.numel(), t.float32, "g_out", inplace=True)
        _check(load().srwcr_value_and_grad_async(self._h, level, _ptr(c), _ptr(D_out),
                                                 _ptr(g_out)))
        self._gen[level] += 1

    def value_and_grad_host(self, c_host: np.ndarray, g_host: np.ndarray, level: int = 0) -> float:
        """End-to-end call with host buffers (copies inside the library)."""
        c_host = self._host(c_host, level, "c_host")
        g_host = self._host(g_host, level, "g_host", writes=True)
        D = ctypes.c_double()
        _check(load().srwcr_value_and_grad_host(
            self._h, level, c_host.ctypes.data_as(ctypes.c_void_p), ctypes.byref(D),
            g_host.ctypes.data_as(ctypes.c_void_p)))
        self._gen[level] += 1
        return D.value

    def forward(self, c, D_out, level: int = 0) -> int:
        c = self._c(c, level)
        D_out = self._dev(D_out, 1, self._torch.float64, "D_out", inplace=True)
        _check(load().srwcr_forward(self._h, level, _ptr(c), _ptr(D_out)))
        self._gen[level] += 1
        return self._gen[level]

    def backward(self, c, gD, g_out, level: int = 0):
        t = self._torch
        c = self._c(c, level)
        if gD is not None:
            gD = self._dev(gD, 1, t.float32, "gD")
        g_out = self._dev(g_out, c.numel(), t.float32, "g_out", inplace=True)
        _check(load().srwcr_backward(self._h, level, _ptr(c),
                                     _ptr(gD) if gD is not None else None, _ptr(g_out)))

    def generation(self, level: int = 0) -> int:
        return self._gen[level]

    # -- inspection --------------------------------------------------------
    def region_stats(self, level: int = 0):
        R = self.levels[level].n_regions
        out = np.zeros((R, 4), np.float64)
        nd = ctypes.c_int64()
        _check(load().srwcr_region_stats(self._h, level, out.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(nd)))
        return out, int(nd.value)

    def debug_bins(self, level: int = 0):
        n = self.levels[level].n_voxels
        out = self._torch.empty((n, 4), dtype=self._torch.int32, device=self.device)
        _check(load().srwcr_debug_bins(self._h, level, _ptr(out)))
        return out

    def debug_warp(self, c, level: int = 0):
        c = self._c(c, level)
        out = self._torch.empty(self.levels[level].n_voxels, dtype=self._torch.float32,
                                device=self.device)
        _check(load().srwcr_debug_warp(self._h, level, _ptr(c), _ptr(out)))
        return out

    def debug_warp_grad(self, c, level: int = 0):
        """(n_voxels, 4) float32: B and the interpolant's gradient at T(x)."""
        c = self._c(c, level)
        out = self._torch.empty((self.levels[level].n_voxels, 4), dtype=self._torch.float32,
                                device=self.device)
        _check(load().srwcr_debug_warp_grad(self._h, level, _ptr(c), _ptr(out)))
        return out

    def level_images(self, level: int = 0):
        """The level's normalised fixed and moving images as float32 tensors
        shaped like the inputs at that level."""
        d = self.levels[level].dims
        shape = (d[1], d[0]) if self.ndim == 2 else (d[2], d[1], d[0])
        A = self._torch.empty(shape, dtype=self._torch.float32, device=self.device)
        M = self._torch.empty_like(A)
        _check(load().srwcr_level_images(self._h, level, _ptr(A), _ptr(M)))
        return A, M

    def refine(self, c_coarse, level: int):
        """Coefficients of `level` refined to level - 1 (dyadic subdivision,
        values doubled)."""
        c_coarse = self._c(c_coarse, level)
        out = self.zeros(level - 1)
        _check(load().srwcr_refine(self._h, level, _ptr(c_coarse), _ptr(out)))
        self._torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return out

    def lbfgs_direction(self, g, S=None, Y=None):
        """d = -H g from the library's two-loop recursion; S, Y: (k, n)
        float32 CUDA tensors of (s, y) pairs, oldest first."""
        t = self._torch
        if not isinstance(g, t.Tensor):
            raise TypeError("g must be a float32 CUDA tensor")
        n = g.numel()
        g = self._dev(g, n, t.float32, "g").view(-1)
        k = 0 if S is None else int(S.shape[0])
        d = t.empty_like(g)
        if k:
            if Y is None or tuple(S.shape) != (k, n) or tuple(Y.shape) != (k, n):
                raise ValueError(f"S and Y must both be ({k}, {n})")
            S = self._dev(S, k * n, t.float32, "S")
            Y = self._dev(Y, k * n, t.float32, "Y")
        t.cuda.current_stream(self.device).synchronize()
        _check(load().srwcr_lbfgs_direction(self._h, g.numel(), k, _ptr(S) if k else None,
                                            _ptr(Y) if k else None, _ptr(g), _ptr(d)))
        return d

    # -- benchmark hooks ---------------------------------------------------
    def set_profiling(self, on: bool = True):
        _check(load().srwcr_set_profiling(self._h, 1 if on else 0))

    def profile_read(self, reset: bool = True):
        """(ms[3], counts[3], launches): device ms per kernel kind
        (accumulate, finalize, adjoint), bracketed launches, kernels launched."""
        ms = np.zeros(3, np.float64)
        cnt = np.zeros(3, np.int64)
        n = ctypes.c_int64()
        _check(load().srwcr_profile_read(self._h, ms.ctypes.data_as(ctypes.c_void_p),
                                         cnt.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n),
                                         1 if reset else 0))
        return ms, cnt, int(n.value)

    def autotune(self, c=None, level: int = 0, reps: int = 3):
        """Pick the fastest voxel tile for this level (cached per problem)."""
        if c is None:
            c = self.zeros(level)
        c = self._c(c, level)
        t = (ctypes.c_int * 3)()
        _check(load().srwcr_autotune(self._h, level, _ptr(c), int(reps), t))
        self.levels[level] = self.level_info(level)
        return tuple(t)

    def bending_energy(self, c, level: int = 0, grad_into=None, weight: float = 1.0) -> float:
        """C_p of Eq. (1) at c (synchronises); if grad_into is given, adds
        weight * dC_p/dc to it."""
        c = self._c(c, level)
        if grad_into is not None:
            grad_into = self._dev(grad_into, c.numel(), self._torch.float32, "grad_into",
                                  inplace=True)
        E = self._torch.zeros((), dtype=self._torch.float64, device=self.device)
        _check(load().srwcr_bending_energy(self._h, level, _ptr(c), _ptr(E),
                                           _ptr(grad_into) if grad_into is not None else None,
                                           float(weight)))
        return float(E)

    # -- registration ------------------------------------------------------
    @staticmethod
    def default_opts() -> LbfgsOpts:
        o = LbfgsOpts()
        load().srwcr_lbfgs_default_opts(ctypes.byref(o))
        return o

    def register(self, c, n_levels: int = 1, opts: Optional[LbfgsOpts] = None,
                 check: bool = True) -> Report:
        c = self._c(c, 0, inplace=True)   # the result is written into c
        rep = Report()
        st = load().srwcr_register(self._h, _ptr(c), int(n_levels),
                                   ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(rep))
        if check and st not in (0, 7, 5):
            _check(st)
        rep.status_code = st
        return rep


# -- rigid model (pre-alignment with the same measure) -------------------------
def _rigid_methods():
    def n_rigid(self) -> int:
        """Rigid parameters: (t_x, t_y, t_z, alpha, beta, gamma) in 3-D,
        (t_x, t_y, theta) in 2-D; voxels of the level and radians."""
        return 6 if self.ndim == 3 else 3

    def _mu(self, mu):
        t = self._torch
        if not isinstance(mu, t.Tensor):
            mu = t.as_tensor(np.asarray(mu, np.float32))
        mu = mu.to(device=self.device, dtype=t.float32).contiguous()
        if mu.numel() != self.n_rigid():
            raise ValueError(f"expected {self.n_rigid()} rigid parameters, got {mu.numel()}")
        return mu

    def rigid_value_and_grad(self, mu, level: int = 0, grad: bool = True):
        """D and dD/dmu at the rigid transform mu."""
        mu = _mu(self, mu)
        g = self._torch.empty_like(mu) if grad else None
        D = ctypes.c_double()
        _check(load().srwcr_rigid_value_and_grad(self._h, level, _ptr(mu), ctypes.byref(D),
                                                 _ptr(g) if grad else None))
        return (D.value, g) if grad else D.value

    def rigid_to_ffd(self, mu, level: int = 0):
        """FFD coefficients whose warp equals the rigid transform mu."""
        mu = _mu(self, mu)
        c = self.zeros(level)
        _check(load().srwcr_rigid_to_ffd(self._h, level, _ptr(mu), _ptr(c)))
        self._torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return c

    def rigid_register(self, mu=None, n_levels: int = 1, opts: Optional[LbfgsOpts] = None,
                       check: bool = True):
        """Coarse-to-fine L-BFGS over the rigid parameters; returns (mu, report)."""
        mu = _mu(self, mu if mu is not None else np.zeros(self.n_rigid(), np.float32)).clone()
        rep = Report()
        st = load().srwcr_rigid_register(self._h, _ptr(mu), int(n_levels),
                                         ctypes.byref(opts) if opts is not None else None,
                                         ctypes.byref(rep))
        if check and st not in (0, 7, 5):
            _check(st)
        rep.status_code = st
        return mu, rep

    for f in (n_rigid, rigid_value_and_grad, rigid_to_ffd, rigid_register):
        setattr(SRWCR, f.__name__, f)


_rigid_methods()


class _DeviceArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3,
                                         "strides": None}


class Batch:
    """Many pairs (SRWCR engines) evaluated and registered together.

    Each phase of an evaluation is one launch over every (pair, tile) work
    item; ``use_graph`` replays the phases from a CUDA graph.  The batch owns
    packed coefficient and gradient buffers (``coef(i)``, ``grad(i)`` are
    views of pair i) and runs on a stream of its own that is ordered after
    the current torch stream on entry and before it on exit.
    """

    def __init__(self, engines: Sequence["SRWCR"], level=0):
        """level: one pyramid level for every pair, or one per pair."""
        import torch
        self._torch = torch
        lib = load()
        self.engines = list(engines)
        n = len(self.engines)
        self.levels = [int(level)] * n if np.isscalar(level) else [int(v) for v in level]
        if len(self.levels) != n:
            raise ValueError("one level per engine expected")
        self.stream = torch.cuda.Stream(device=self.engines[0].device)
        arr = (ctypes.c_void_p * n)(*[e._h.value for e in self.engines])
        lv = (ctypes.c_int * n)(*self.levels)
        h = ctypes.c_void_p()
        self.stream.wait_stream(torch.cuda.current_stream())
        _check(lib.srwcr_batch_create_levels(arr, lv, n, ctypes.c_void_p(self.stream.cuda_stream),
                                             ctypes.byref(h)))
        self._h = h
        n = len(self.engines)
        off = np.zeros(n + 1, np.int64)
        npar = np.zeros(n, np.int64)
        _check(lib.srwcr_batch_layout(h, off.ctypes.data_as(ctypes.c_void_p),
                                      npar.ctypes.data_as(ctypes.c_void_p)))
        self.offsets, self.n_params = off, npar
        pc, pg, pD = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib.srwcr_batch_buffers(h, ctypes.byref(pc), ctypes.byref(pg), ctypes.byref(pD)))
        dev = self.engines[0].device
        self.c = torch.as_tensor(_DeviceArray(pc.value, int(off[-1]), "<f4"), device=dev)
        self.g = torch.as_tensor(_DeviceArray(pg.value, int(off[-1]), "<f4"), device=dev)
        self.D = torch.as_tensor(_DeviceArray(pD.value, n, "<f8"), device=dev)

    def __len__(self):
        return len(self.engines)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.stream.synchronize()
            load().srwcr_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> BatchDesc:
        d = BatchDesc()
        _check(load().srwcr_batch_info(self._h, ctypes.byref(d)))
        return d

    def coef(self, i: int):
        """View of pair i's coefficients in the packed buffer."""
        o, n = int(self.offsets[i]), int(self.n_params[i])
        return self.c[o:o + n].view(self.engines[i].coef_shape(self.levels[i]))

    def grad(self, i: int):
        o, n = int(self.offsets[i]), int(self.n_params[i])
        return self.g[o:o + n].view(self.engines[i].coef_shape(self.levels[i]))

    def _enter(self):
        self.stream.wait_stream(self._torch.cuda.current_stream())

    def _leave(self):
        self._torch.cuda.current_stream().wait_stream(self.stream)
        for e, lv in zip(self.engines, self.levels):
            e._gen[lv] += 1

    def value_and_grad_async(self, use_graph: bool = True):
        """Queue D_i, dD_i/dc_i for every pair at the packed coefficients."""
        self._enter()
        _check(load().srwcr_batch_value_and_grad(self._h, 1 if use_graph else 0))
        self._leave()

    def value_and_grad(self, use_graph: bool = True) -> np.ndarray:
        self.value_and_grad_async(use_graph)
        return self.values()

    def values(self) -> np.ndarray:
        out = np.zeros(len(self), np.float64)
        _check(load().srwcr_batch_sync(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def register(self, opts: Optional[LbfgsOpts] = None, use_graph: bool = True,
                 check: bool = True) -> dict:
        """Single-level L-BFGS of every pair from the packed coefficients."""
        n = len(self)
        it = np.zeros(n, np.int32)
        ev = np.zeros(n, np.int32)
        fv = np.zeros(n, np.float64)
        stt = np.zeros(n, np.int32)
        self._enter()
        st = load().srwcr_batch_register(
            self._h, ctypes.byref(opts) if opts is not None else None, 1 if use_graph else 0,
            it.ctypes.data_as(ctypes.c_void_p), ev.ctypes.data_as(ctypes.c_void_p),
            fv.ctypes.data_as(ctypes.c_void_p), stt.ctypes.data_as(ctypes.c_void_p))
        self._leave()
        if check:
            _check(st)
        return {"iterations": it, "evaluations": ev, "final_value": fv, "status": stt}


def from_problem(prob, fixed, moving, storage: str = "f32", pyramid_levels: int = 1, **kw) -> SRWCR:
    """Build an engine from a ``synth.Problem``-like description."""
    return SRWCR(fixed, moving, prob.ffd_spacing[:prob.ndim], prob.sbin_intervals[:prob.ndim],
                 prob.n_bins, storage=storage, pyramid_levels=pyramid_levels, **kw)


def debug_fixed_point(v, hi, lo, reference: bool = False):
    """The flushes' fixed-point conversions on CUDA tensors: v (float32) ->
    nearest integer (int64 tensor holding the uint64 bits), and
    (hi, lo) (int32 tensors holding uint32 bits) -> nearest float32 to
    hi * 2^24 + lo.  reference=True takes CUDA's 64-bit conversions."""
    import torch
    v = v.contiguous(); hi = hi.contiguous(); lo = lo.contiguous()
    assert v.dtype == torch.float32 and hi.dtype == torch.int32 and lo.dtype == torch.int32
    assert hi.numel() == lo.numel()
    fixed = torch.empty(v.numel(), dtype=torch.int64, device=v.device)
    flt = torch.empty(hi.numel(), dtype=torch.float32, device=v.device)
    _check(load().srwcr_debug_fixed_point(_ptr(v), v.numel(), _ptr(hi), _ptr(lo), hi.numel(),
                                          _ptr(fixed), _ptr(flt), int(bool(reference))))
    return fixed, flt


def tile_order(rowdist, dims, tile):
    """The row kernels' tile launch order, computed on the host
    (srwcr_tile_order): rowdist holds one byte per 32-voxel x-row segment,
    [z][y][x block]; dims = (nx, ny[, nz]), tile = (32, ty[, tz]).  Returns
    (order, cost) as int32 arrays over the tiles."""
    rowdist = np.ascontiguousarray(rowdist, dtype=np.uint8)
    d = [int(v) for v in dims] + [1] * (3 - len(dims))
    t = [int(v) for v in tile] + [1] * (3 - len(tile))
    if min(d) < 1 or min(t) < 1:
        raise ValueError("dims and tile must be positive")
    nxb = (d[0] + 31) // 32
    if rowdist.size != nxb * d[1] * d[2]:
        raise ValueError(f"rowdist has {rowdist.size} entries, dims need {nxb * d[1] * d[2]}")
    nt = nxb * (-(-d[1] // t[1])) * (-(-d[2] // t[2]))
    order = np.empty(nt, np.int32)
    cost = np.empty(nt, np.int32)
    _check(load().srwcr_tile_order(rowdist.ctypes.data_as(ctypes.c_void_p), (ctypes.c_int * 3)(*d),
                                   (ctypes.c_int * 3)(*t), order.ctypes.data_as(ctypes.c_void_p),
                                   cost.ctypes.data_as(ctypes.c_void_p)))
    return order, cost
