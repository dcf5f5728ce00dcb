"""FP64 CPU oracle for SRWCR -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it,
and it shares no code with the CUDA path: the arithmetic lives in
``srwcr_oracle.c`` (plain C, double precision, single thread), written from
the paper's definitions (Eqs. 3-10, 12, 16, 17, 27; Sec. II-F for warping and
normalisation).  ``lbfgs.py`` holds the quasi-Newton loop (Sec. II-F).

Parity pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srwcr_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle_srwcr.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 3),
                ("ffd_sp", ctypes.c_int64 * 3), ("sb_num", ctypes.c_int64 * 3),
                ("sb_den", ctypes.c_int64 * 3), ("nbins", ctypes.c_int), ("sb_mode", ctypes.c_int),
                ("xform", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_PP = ctypes.POINTER(_Problem)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        sig = {
            "orc_bspline": (ctypes.c_double, [ctypes.c_int, ctypes.c_double]),
            "orc_parzen": (ctypes.c_double, [ctypes.c_double]),
            "orc_parzen_dleft": (ctypes.c_double, [ctypes.c_double]),
            "orc_parzen_dright": (ctypes.c_double, [ctypes.c_double]),
            "orc_parzen_dkappa": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_int]),
            "orc_normalise": (ctypes.c_int, [_F, ctypes.c_int64, ctypes.c_double, _D]),
            "orc_n_ffd_nodes": (ctypes.c_int64, [_PP, ctypes.c_int]),
            "orc_n_sbins": (ctypes.c_int64, [_PP, ctypes.c_int]),
            "orc_n_regions": (ctypes.c_int64, [_PP]),
            "orc_spatial_weights": (ctypes.c_int, [_PP, ctypes.c_int64, ctypes.c_int64,
                                                   ctypes.c_int64, _I64, _D]),
            "orc_displacement": (ctypes.c_int, [_PP, _D, ctypes.c_int64, ctypes.c_int64,
                                                ctypes.c_int64, _D]),
            "orc_interp": (ctypes.c_int, [_PP, _D, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _D]),
            "orc_warp": (ctypes.c_int, [_PP, _D, _D, _D, _D]),
            "orc_joint_pdf": (ctypes.c_int, [_PP, _D, _D, _D, _D, _D]),
            "orc_srwcr_from_pdf": (ctypes.c_int, [_D, ctypes.c_int64, ctypes.c_int, _D, _D, _D,
                                                  _D, _D, _D, _D, _U8, _I64]),
            "orc_dD_dB_image": (ctypes.c_int, [_PP, _D, _D, _D, _D, _D, _D, _D, _U8,
                                               ctypes.c_double, _D]),
            "orc_gradient": (ctypes.c_int, [_PP, _D, _D, _D, _D, _D, _D, _D, _U8,
                                            ctypes.c_double, _D]),
            "orc_gradient_at": (ctypes.c_int, [_PP, _D, _D, _D, _D, _D, _D, _D, _U8,
                                               ctypes.c_double, _I64, ctypes.c_int64, _D]),
            "orc_joint_pdf_mas_a": (ctypes.c_int, [_PP, _D, _D, _D, _D, _D]),
            "orc_gradient_mas_a": (ctypes.c_int, [_PP, _D, _D, _D, _D, _D, _D, _D, _U8,
                                                  ctypes.c_double, _D]),
            "orc_rigid_matrix": (ctypes.c_int, [ctypes.c_int, _D, _D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


@dataclass
class Geometry:
    """Oracle view of one problem (sizes only)."""
    ndim: int
    dims: tuple          # (nx, ny, nz)
    ffd_spacing: tuple
    sbin_num: tuple
    sbin_den: tuple
    n_bins: int
    boxcar: bool = False
    rigid: bool = False  # c holds the rigid parameters instead of FFD coefficients

    @classmethod
    def from_problem(cls, prob, boxcar_patches: Optional[tuple] = None) -> "Geometry":
        """Map a ``synth.Problem``.  Spatial-bin intervals K > 0 give spacing
        N/K; K = 0 puts the bins on the FFD grid (spacing delta).  With
        ``boxcar_patches`` the distribution is the boxcar of Eq. (6) over a
        regular partition into that many patches per axis."""
        num, den = [], []
        for d in range(3):
            n = prob.dims[d]
            if boxcar_patches is not None:
                num.append(n); den.append(int(boxcar_patches[d]) if d < prob.ndim else 1)
            elif d < prob.ndim and prob.sbin_intervals[d] > 0:
                num.append(n); den.append(int(prob.sbin_intervals[d]))
            else:
                num.append(int(prob.ffd_spacing[d])); den.append(1)
        return cls(prob.ndim, tuple(prob.dims), tuple(prob.ffd_spacing), tuple(num), tuple(den),
                   prob.n_bins, boxcar_patches is not None)

    def c_struct(self) -> _Problem:
        s = _Problem()
        s.ndim = self.ndim
        for d in range(3):
            s.n[d] = int(self.dims[d]); s.ffd_sp[d] = int(self.ffd_spacing[d])
            s.sb_num[d] = int(self.sbin_num[d]); s.sb_den[d] = int(self.sbin_den[d])
        s.nbins = int(self.n_bins)
        s.sb_mode = 1 if self.boxcar else 0
        s.xform = 1 if self.rigid else 0
        return s

    @property
    def n_voxels(self):
        return int(self.dims[0] * self.dims[1] * self.dims[2])

    def n_regions(self) -> int:
        s = self.c_struct()
        return int(lib().orc_n_regions(ctypes.byref(s)))

    def ffd_nodes(self):
        s = self.c_struct()
        return tuple(int(lib().orc_n_ffd_nodes(ctypes.byref(s), d)) for d in range(3))

    def sbins(self):
        s = self.c_struct()
        return tuple(int(lib().orc_n_sbins(ctypes.byref(s), d)) for d in range(3))

    def n_params(self):
        n = self.ffd_nodes()
        return self.ndim * n[0] * n[1] * n[2]


def bspline(l: int, t: float) -> float:
    return lib().orc_bspline(l, t)


def parzen(t: float) -> float:
    return lib().orc_parzen(t)


def parzen_dleft(t: float) -> float:
    return lib().orc_parzen_dleft(t)


def parzen_dright(t: float) -> float:
    return lib().orc_parzen_dright(t)


def parzen_dkappa(b: float, B: float, L: int) -> float:
    """dh/dkappa at kappa = b - B inside the cell of B (Eqs. 19, 27)."""
    return lib().orc_parzen_dkappa(b, B, L)


def normalise(img: np.ndarray, L: float) -> np.ndarray:
    """Min-max map to [0, L] in FP64 (Sec. II); raises on a constant image."""
    v = np.ascontiguousarray(img, dtype=np.float32)
    out = np.empty(v.shape, np.float64)
    rc = lib().orc_normalise(v.ctypes.data_as(_F), v.size, float(L), _d(out))
    if rc != 0:
        raise ValueError("constant image cannot be normalised")
    return out


def storage_round(x: np.ndarray, storage: str) -> np.ndarray:
    """Round normalised FP64 values to the storage type and promote back."""
    if storage == "f32":
        return x.astype(np.float32).astype(np.float64)
    if storage == "bf16":
        import torch
        t = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64)
        return t.numpy()
    raise ValueError(storage)


def prepare(fixed: np.ndarray, moving: np.ndarray, n_bins: int, storage: str = "f32"):
    """Normalise both images to [0, L] and round them to the storage type."""
    L = n_bins - 1
    A = storage_round(normalise(fixed, L), storage)
    M = storage_round(normalise(moving, L), storage)
    return np.ascontiguousarray(A.ravel()), np.ascontiguousarray(M.ravel())


def spatial_weights(geo: Geometry, x, y, z):
    s = geo.c_struct()
    bins = np.zeros(64, np.int64)
    w = np.zeros(64, np.float64)
    n = lib().orc_spatial_weights(ctypes.byref(s), x, y, z, bins.ctypes.data_as(_I64), _d(w))
    return bins[:n].copy(), w[:n].copy()


def displacement(geo: Geometry, c: np.ndarray, x, y, z):
    s = geo.c_struct()
    c = np.ascontiguousarray(c, np.float64)
    u = np.zeros(3)
    lib().orc_displacement(ctypes.byref(s), _d(c), x, y, z, _d(u))
    return u


def interp(geo: Geometry, M: np.ndarray, y):
    s = geo.c_struct()
    out = np.zeros(4)
    M = np.ascontiguousarray(M, np.float64)
    lib().orc_interp(ctypes.byref(s), _d(M), float(y[0]), float(y[1]), float(y[2]), _d(out))
    return out[0], out[1:].copy()


def warp(geo: Geometry, M: np.ndarray, c: np.ndarray):
    s = geo.c_struct()
    M = np.ascontiguousarray(M, np.float64).ravel()
    c = np.ascontiguousarray(c, np.float64)
    B = np.empty(geo.n_voxels)
    g = np.empty(3 * geo.n_voxels)
    lib().orc_warp(ctypes.byref(s), _d(M), _d(c), _d(B), _d(g))
    return B, g.reshape(-1, 3)


@dataclass
class Stats:
    """Regional statistics of Eqs. (4) and (10) and the value of Eq. (9)."""
    D: float            # Eq. (9)
    D12: float          # Eq. (12), same quantity in the concise form
    Z: float
    pr: np.ndarray
    mu_r: np.ndarray
    var_r: np.ndarray
    cr: np.ndarray
    mu_ra: np.ndarray
    valid: np.ndarray
    n_degenerate: int


def joint_pdf(geo: Geometry, A: np.ndarray, M: np.ndarray, c: np.ndarray):
    """Eq. (3): p(a, b, r), shape (R, L+1, L+1), and Z."""
    s = geo.c_struct()
    R, nb = geo.n_regions(), geo.n_bins
    p = np.zeros(R * nb * nb)
    Z = ctypes.c_double(0.0)
    A = np.ascontiguousarray(A, np.float64).ravel()
    M = np.ascontiguousarray(M, np.float64).ravel()
    c = np.ascontiguousarray(c, np.float64)
    rc = lib().orc_joint_pdf(ctypes.byref(s), _d(A), _d(M), _d(c), _d(p), ctypes.byref(Z))
    if rc != 0:
        raise RuntimeError(f"orc_joint_pdf failed ({rc})")
    return p.reshape(R, nb, nb), Z.value


def stats_from_pdf(p: np.ndarray, Z: float = float("nan")) -> Stats:
    R, nb, _ = p.shape
    pc = np.ascontiguousarray(p, np.float64)
    D9, D12 = ctypes.c_double(), ctypes.c_double()
    pr, mu, var, cr = (np.zeros(R) for _ in range(4))
    mu_ra = np.zeros(R * nb)
    valid = np.zeros(R, np.uint8)
    ndeg = ctypes.c_int64()
    lib().orc_srwcr_from_pdf(_d(pc), R, nb, ctypes.byref(D9), ctypes.byref(D12), _d(pr), _d(mu),
                             _d(var), _d(cr), _d(mu_ra), valid.ctypes.data_as(_U8),
                             ctypes.byref(ndeg))
    return Stats(D9.value, D12.value, Z, pr, mu, var, cr, mu_ra.reshape(R, nb), valid,
                 int(ndeg.value))


def value(geo: Geometry, A, M, c) -> Stats:
    """SRWCR (Eq. 9) with all regional statistics."""
    p, Z = joint_pdf(geo, A, M, c)
    return stats_from_pdf(p, Z)


def _tables(st: Stats):
    return (_d(st.mu_r), _d(st.var_r), _d(st.cr), _d(np.ascontiguousarray(st.mu_ra).ravel()),
            st.valid.ctypes.data_as(_U8), float(st.Z))


def gradient(geo: Geometry, A, M, c, st: Stats) -> np.ndarray:
    """Eqs. (16), (17), (27): dD/dc for every coefficient, shaped like c."""
    s = geo.c_struct()
    A = np.ascontiguousarray(A, np.float64).ravel()
    M = np.ascontiguousarray(M, np.float64).ravel()
    c = np.ascontiguousarray(c, np.float64)
    g = np.zeros(c.size)
    mu_ra = np.ascontiguousarray(st.mu_ra, np.float64).ravel()
    rc = lib().orc_gradient(ctypes.byref(s), _d(A), _d(M), _d(c), _d(st.mu_r), _d(st.var_r),
                            _d(st.cr), _d(mu_ra), st.valid.ctypes.data_as(_U8), float(st.Z), _d(g))
    if rc != 0:
        raise RuntimeError(f"orc_gradient failed ({rc})")
    return g.reshape(c.shape)


def gradient_at(geo: Geometry, A, M, c, st: Stats, which) -> np.ndarray:
    """Selected entries (flat indices into c) of the gradient."""
    s = geo.c_struct()
    A = np.ascontiguousarray(A, np.float64).ravel()
    M = np.ascontiguousarray(M, np.float64).ravel()
    c = np.ascontiguousarray(c, np.float64)
    w = np.ascontiguousarray(which, np.int64)
    out = np.zeros(w.size)
    mu_ra = np.ascontiguousarray(st.mu_ra, np.float64).ravel()
    rc = lib().orc_gradient_at(ctypes.byref(s), _d(A), _d(M), _d(c), _d(st.mu_r), _d(st.var_r),
                               _d(st.cr), _d(mu_ra), st.valid.ctypes.data_as(_U8), float(st.Z),
                               w.ctypes.data_as(_I64), w.size, _d(out))
    if rc != 0:
        raise RuntimeError(f"orc_gradient_at failed ({rc})")
    return out


def dD_dB_image(geo: Geometry, A, M, c, st: Stats) -> np.ndarray:
    """Eq. (27) at every voxel."""
    s = geo.c_struct()
    A = np.ascontiguousarray(A, np.float64).ravel()
    M = np.ascontiguousarray(M, np.float64).ravel()
    c = np.ascontiguousarray(c, np.float64)
    G = np.zeros(geo.n_voxels)
    mu_ra = np.ascontiguousarray(st.mu_ra, np.float64).ravel()
    lib().orc_dD_dB_image(ctypes.byref(s), _d(A), _d(M), _d(c), _d(st.mu_r), _d(st.var_r),
                          _d(st.cr), _d(mu_ra), st.valid.ctypes.data_as(_U8), float(st.Z), _d(G))
    return G


# ---------------------------------------------------------------------------
# Moving image as the model image A (Sec. II-E, Eqs. 20, 21)
# ---------------------------------------------------------------------------
def joint_pdf_mas_a(geo: Geometry, F: np.ndarray, M: np.ndarray, c: np.ndarray):
    """Eq. (3) with a from the warped moving image M(T(x)) and b from F."""
    s = geo.c_struct()
    R, nb = geo.n_regions(), geo.n_bins
    p = np.zeros(R * nb * nb)
    Z = ctypes.c_double(0.0)
    F = np.ascontiguousarray(F, np.float64).ravel()
    M = np.ascontiguousarray(M, np.float64).ravel()
    c = np.ascontiguousarray(c, np.float64)
    rc = lib().orc_joint_pdf_mas_a(ctypes.byref(s), _d(F), _d(M), _d(c), _d(p), ctypes.byref(Z))
    if rc != 0:
        raise RuntimeError(f"orc_joint_pdf_mas_a failed ({rc})")
    return p.reshape(R, nb, nb), Z.value


def value_mas_a(geo: Geometry, F, M, c) -> Stats:
    """SRWCR (Eq. 9) with the warped moving image as A and F as B."""
    p, Z = joint_pdf_mas_a(geo, F, M, c)
    return stats_from_pdf(p, Z)


def gradient_mas_a(geo: Geometry, F, M, c, st: Stats) -> np.ndarray:
    """Eqs. (15)-(17) with Eq. (21): dD/dc when the moving image is A."""
    s = geo.c_struct()
    F = np.ascontiguousarray(F, np.float64).ravel()
    M = np.ascontiguousarray(M, np.float64).ravel()
    c = np.ascontiguousarray(c, np.float64)
    g = np.zeros(c.size)
    mu_ra = np.ascontiguousarray(st.mu_ra, np.float64).ravel()
    rc = lib().orc_gradient_mas_a(ctypes.byref(s), _d(F), _d(M), _d(c), _d(st.mu_r),
                                  _d(st.var_r), _d(st.cr), _d(mu_ra),
                                  st.valid.ctypes.data_as(_U8), float(st.Z), _d(g))
    if rc != 0:
        raise RuntimeError(f"orc_gradient_mas_a failed ({rc})")
    return g.reshape(c.shape)


def value_and_grad(geo: Geometry, A, M, c):
    st = value(geo, A, M, c)
    return st.D, gradient(geo, A, M, c, st), st
