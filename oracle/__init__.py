"""Plain FP64 CPU oracle for the Wilson twisted-mass operator.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by the
CPU-baseline leg of ``bench.py``; never by the product path.  The C source
(``oracle.c``) writes out the operator definitions (eq. 2.1-2.4) as plain loops;
this module only builds it with gcc and marshals numpy arrays.

Array conventions (canonical, full lattice, x fastest):
  spinor  complex128 [Lt, Lz, Ly, Lx, nf, 4, 3]
  gauge   complex128 [4, Lt, Lz, Ly, Lx, 3, 3]     (mu = 0..3 <-> x, y, z, t)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fcx-limited-range", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("nf", ctypes.c_int), ("fsign", ctypes.c_int), ("tbc", ctypes.c_int),
                ("kappa", ctypes.c_double), ("mu", ctypes.c_double), ("eps", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Params)
        vp = ctypes.c_void_p
        _lib.orc_hop.argtypes = [P, vp, vp, vp, ctypes.c_int]
        _lib.orc_twist.argtypes = [P, vp, vp, ctypes.c_int]
        _lib.orc_twist_matrix.argtypes = [P, ctypes.c_int, vp]
        _lib.orc_M.argtypes = [P, vp, vp, vp, ctypes.c_int]
        _lib.orc_M_pc.argtypes = [P, vp, vp, vp, ctypes.c_int, ctypes.c_int]
        _lib.orc_prepare_rhs.argtypes = [P, vp, vp, vp, ctypes.c_int, ctypes.c_int]
        _lib.orc_reconstruct_odd.argtypes = [P, vp, vp, vp, vp, ctypes.c_int]
        _lib.orc_cg_normal.argtypes = [P, vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double)]
        _lib.orc_force.argtypes = [P, vp, vp, vp, ctypes.c_double, vp, ctypes.c_int]
        _lib.orc_parity_project.argtypes = [P, vp, ctypes.c_int]
        _lib.orc_gamma.argtypes = [ctypes.c_int, vp]
        _lib.orc_gamma.restype = None
        _lib.orc_hop.restype = None
        _lib.orc_force.restype = None
        _lib.orc_parity_project.restype = None
    return _lib


class Params:
    """Lattice and operator parameters.  flavor: +1 / -1 (one flavour with tau3 = +-1) or 2 (doublet)."""

    def __init__(self, L, kappa, mu, eps=0.0, flavor=2, t_antiperiodic=True):
        self.L = tuple(int(v) for v in L)
        self.kappa, self.mu, self.eps = float(kappa), float(mu), float(eps)
        self.flavor = int(flavor)
        self.nf = 2 if self.flavor == 2 else 1
        self.t_antiperiodic = bool(t_antiperiodic)

    def c(self):
        p = _Params()
        p.L[:] = self.L
        p.nf, p.fsign = self.nf, (1 if self.flavor == 2 else self.flavor)
        p.tbc = int(self.t_antiperiodic)
        p.kappa, p.mu, p.eps = self.kappa, self.mu, self.eps
        return p

    @property
    def spinor_shape(self):
        Lx, Ly, Lz, Lt = self.L
        return (Lt, Lz, Ly, Lx, self.nf, 4, 3)

    @property
    def gauge_shape(self):
        Lx, Ly, Lz, Lt = self.L
        return (4, Lt, Lz, Ly, Lx, 3, 3)


def _cv(a, shape):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    assert a.shape == tuple(shape), (a.shape, shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def gamma(mu: int) -> np.ndarray:
    """gamma_{mu+1} for mu = 0..3 (x, y, z, t), gamma5 for mu = 4, as the oracle defines them."""
    out = np.zeros(32)
    _load().orc_gamma(mu, _ptr(out))
    return (out[0::2] + 1j * out[1::2]).reshape(4, 4)


def hop(p: Params, U, psi, dagger=False):
    U, psi = _cv(U, p.gauge_shape), _cv(psi, p.spinor_shape)
    out = np.empty_like(psi)
    _load().orc_hop(ctypes.byref(p.c()), _ptr(U), _ptr(psi), _ptr(out), int(dagger))
    return out


def twist_matrix(p: Params, inverse=False, dagger=False) -> np.ndarray:
    D = 4 * p.nf
    out = np.zeros(2 * D * D)
    if _load().orc_twist_matrix(ctypes.byref(p.c()), int(inverse) | 2 * int(dagger), _ptr(out)):
        raise ZeroDivisionError("twist matrix is singular")
    return (out[0::2] + 1j * out[1::2]).reshape(D, D)


def twist(p: Params, psi, inverse=False, dagger=False):
    psi = _cv(psi, p.spinor_shape)
    out = np.empty_like(psi)
    if _load().orc_twist(ctypes.byref(p.c()), _ptr(psi), _ptr(out), int(inverse) | 2 * int(dagger)):
        raise ZeroDivisionError("twist matrix is singular")
    return out


def apply_M(p: Params, U, psi, dagger=False):
    U, psi = _cv(U, p.gauge_shape), _cv(psi, p.spinor_shape)
    out = np.empty_like(psi)
    if _load().orc_M(ctypes.byref(p.c()), _ptr(U), _ptr(psi), _ptr(out), int(dagger)):
        raise RuntimeError("orc_M failed")
    return out


def apply_M_pc(p: Params, U, psi, sym=False, dagger=False):
    U, psi = _cv(U, p.gauge_shape), _cv(psi, p.spinor_shape)
    out = np.empty_like(psi)
    if _load().orc_M_pc(ctypes.byref(p.c()), _ptr(U), _ptr(psi), _ptr(out), int(sym), int(dagger)):
        raise RuntimeError("orc_M_pc failed")
    return out


def prepare_rhs(p: Params, U, b, sym=False, dagger=False):
    U, b = _cv(U, p.gauge_shape), _cv(b, p.spinor_shape)
    out = np.empty_like(b)
    if _load().orc_prepare_rhs(ctypes.byref(p.c()), _ptr(U), _ptr(b), _ptr(out), int(sym), int(dagger)):
        raise RuntimeError("orc_prepare_rhs failed")
    return out


def reconstruct_odd(p: Params, U, psi_e, b, dagger=False):
    U, psi_e, b = _cv(U, p.gauge_shape), _cv(psi_e, p.spinor_shape), _cv(b, p.spinor_shape)
    out = np.empty_like(b)
    if _load().orc_reconstruct_odd(ctypes.byref(p.c()), _ptr(U), _ptr(psi_e), _ptr(b), _ptr(out), int(dagger)):
        raise RuntimeError("orc_reconstruct_odd failed")
    return out


def cg_normal(p: Params, U, y, sym=False, dagger=False, tol=1e-12, maxiter=10000, x0=None):
    """Solve A^dag A x = y, A = M_pc (or M_pc^dag).  Returns (x, iterations, true relative residual)."""
    U, y = _cv(U, p.gauge_shape), _cv(y, p.spinor_shape)
    x = np.zeros_like(y) if x0 is None else _cv(x0, p.spinor_shape).copy()
    res = ctypes.c_double(0.0)
    it = _load().orc_cg_normal(ctypes.byref(p.c()), _ptr(U), int(sym), int(dagger), _ptr(y), _ptr(x), tol,
                               int(maxiter), ctypes.byref(res))
    if it < 0:
        raise MemoryError("orc_cg_normal: allocation failed")
    return x, int(it), float(res.value)


def force(p: Params, U, psi, g, coef=1.0, project=True):
    """Gradient of Re<g, M(U) psi> with respect to every link (see orc_force)."""
    U, psi, g = _cv(U, p.gauge_shape), _cv(psi, p.spinor_shape), _cv(g, p.spinor_shape)
    out = np.empty_like(U)
    _load().orc_force(ctypes.byref(p.c()), _ptr(U), _ptr(psi), _ptr(g), float(coef), _ptr(out), int(project))
    return out


def parity_mask(p: Params, parity: int) -> np.ndarray:
    """Boolean array [Lt, Lz, Ly, Lx]: True where (x+y+z+t) % 2 == parity."""
    Lx, Ly, Lz, Lt = p.L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return ((x + y + z + t) % 2) == parity


def project_parity(p: Params, v, parity: int):
    v = _cv(v, p.spinor_shape).copy()
    _load().orc_parity_project(ctypes.byref(p.c()), _ptr(v), int(parity))
    return v
