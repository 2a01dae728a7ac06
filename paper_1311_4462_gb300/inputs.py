"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers; it holds none of the operator's arithmetic.

* Links: U = exp(i * 0.3 * H) per link, H traceless hermitian built from a 3x3 matrix
  A with iid N(0,1) real and imaginary parts, H = (A + A^dag)/2 - tr(.)/3.  The
  exponential is taken through the eigendecomposition of H written in closed form
  (the three real roots of the characteristic polynomial det(l - H) = l^3 - c1 l - c0,
  c1 = tr(H^2)/2, c0 = det H, by the trigonometric formula, and the spectral projectors
  P_k = prod_{j != k} (H - l_j)/(l_k - l_j)), vectorised over all links; rows 1-2 are
  then re-orthonormalised and row 3 is set to conj(row1 x row2), so every link is in
  SU(3) to rounding (which makes 12-real storage exact).
* Spinors: iid N(0,1) real and imaginary parts per (site, flavour, spin, colour).
* Z2 noise: (+-1 +- i)/sqrt(2) per entry.
* Generators: numpy PCG64; seed conventions gauge 1000+k, spinor 2000+k, noise 3000+n.

Canonical layouts (x fastest): spinor [Lt, Lz, Ly, Lx, nf, 4, 3],
gauge [4, Lt, Lz, Ly, Lx, 3, 3] with mu = 0..3 <-> x, y, z, t.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _expi_herm(H: np.ndarray, scale: float) -> np.ndarray:
    """exp(i * scale * H) for traceless hermitian 3x3 H (batched), via the closed-form spectrum."""
    H2 = H @ H
    c1 = 0.5 * np.trace(H2, axis1=-2, axis2=-1).real
    c0 = np.linalg.det(H).real
    r = np.sqrt(np.maximum(c1, 1e-300) / 3.0)
    arg = np.clip(c0 / (2.0 * r ** 3), -1.0, 1.0)
    th = np.arccos(arg) / 3.0
    lam = [2.0 * r * np.cos(th - 2.0 * np.pi * k / 3.0) for k in range(3)]
    eye = np.eye(3)
    U = np.zeros_like(H)
    for k in range(3):
        a, b = [lam[j] for j in range(3) if j != k]
        num = H2 - (a + b)[..., None, None] * H + (a * b)[..., None, None] * eye
        den = (lam[k] - a) * (lam[k] - b)
        U = U + (np.exp(1j * scale * lam[k]) / den)[..., None, None] * num
    return U


def reunitarize(U: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 1 and 2, row 3 = conj(row1 x row2): the nearest-by-construction SU(3) matrix."""
    r1 = U[..., 0, :]
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = U[..., 1, :]
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=-2)


def _su3_from_normals(A: np.ndarray, scale: float) -> np.ndarray:
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[:, None, None] * np.eye(3)
    return reunitarize(_expi_herm(H, scale))


def random_su3(n: int, g: np.random.Generator, scale: float = 0.3) -> np.ndarray:
    A = g.standard_normal((n, 3, 3)) + 1j * g.standard_normal((n, 3, 3))
    if n < 65536:
        return _su3_from_normals(A, scale)
    # same arithmetic per link, done in cache-sized chunks on a thread pool (numpy releases the GIL)
    chunks = np.array_split(A, (n + 131071) // 131072)
    with ThreadPoolExecutor(max(1, min(32, os.cpu_count() or 1))) as ex:
        return np.concatenate(list(ex.map(lambda a: _su3_from_normals(a, scale), chunks)), axis=0)


def gauge_field(L, seed: int, scale: float = 0.3) -> np.ndarray:
    Lx, Ly, Lz, Lt = L
    n = 4 * Lx * Ly * Lz * Lt
    return random_su3(n, rng(seed), scale).reshape(4, Lt, Lz, Ly, Lx, 3, 3)


def spinor_field(L, nf: int, seed: int) -> np.ndarray:
    Lx, Ly, Lz, Lt = L
    g = rng(seed)
    shape = (Lt, Lz, Ly, Lx, nf, 4, 3)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def z2_noise(L, nf: int, seed: int) -> np.ndarray:
    Lx, Ly, Lz, Lt = L
    g = rng(seed)
    shape = (Lt, Lz, Ly, Lx, nf, 4, 3)
    re = 2.0 * g.integers(0, 2, size=shape) - 1.0
    im = 2.0 * g.integers(0, 2, size=shape) - 1.0
    return (re + 1j * im) / np.sqrt(2.0)


# Counter-based Z2 noise: element i (flat index into the canonical array) of source `seed`
# takes its two sign bits from SplitMix64's output function (Steele, Lea & Flood, "Fast
# splittable pseudorandom number generators", OOPSLA 2014) applied to the counter
# state = (seed + 1) * G + (i + 1) * G, G = 0x9E3779B97F4A7C15 (mod 2^64): bit 0 -> sign of the
# real part, bit 1 -> sign of the imaginary part.  The library implements the same definition
# on the device (tm_noise_z2), so large batches of sources need not cross the host link.
_SM_G = np.uint64(0x9E3779B97F4A7C15)
_SM_M1 = np.uint64(0xBF58476D1CE4E5B9)
_SM_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state: np.ndarray) -> np.ndarray:
    z = state.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _SM_M1
        z = (z ^ (z >> np.uint64(27))) * _SM_M2
    return z ^ (z >> np.uint64(31))


def z2_noise_counter(L, nf: int, seed: int) -> np.ndarray:
    Lx, Ly, Lz, Lt = L
    shape = (Lt, Lz, Ly, Lx, nf, 4, 3)
    n = int(np.prod(shape))
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        state = np.uint64(seed + 1) * _SM_G + i * _SM_G
    z = splitmix64(state)
    re = 1.0 - 2.0 * (z & np.uint64(1)).astype(np.float64)
    im = 1.0 - 2.0 * ((z >> np.uint64(1)) & np.uint64(1)).astype(np.float64)
    h = 0.70710678118654752440  # 1/sqrt(2), the double nearest the exact value (same literal on the device)
    return ((re + 1j * im) * h).reshape(shape)


def gauge_transform(L, seed: int) -> np.ndarray:
    """Random SU(3) matrix per site, [Lt, Lz, Ly, Lx, 3, 3] (for gauge-covariance checks)."""
    Lx, Ly, Lz, Lt = L
    return random_su3(Lx * Ly * Lz * Lt, rng(seed), scale=1.5).reshape(Lt, Lz, Ly, Lx, 3, 3)


def su3_algebra_direction(shape, seed: int) -> np.ndarray:
    """Random traceless hermitian 3x3 matrices of the given leading shape (tangent directions)."""
    g = rng(seed)
    A = g.standard_normal(tuple(shape) + (3, 3)) + 1j * g.standard_normal(tuple(shape) + (3, 3))
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    return H - tr[..., None, None] * np.eye(3)
