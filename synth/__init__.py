"""Seeded synthetic inputs: SU(3) gauge fields, Gaussian right-hand sides, shift sets.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's
tests.  It holds none of the solver's arithmetic (no operator, no Krylov step,
no interpolation): it only draws random numbers and shapes them into the
canonical host layouts that the C-ABI accepts.

Canonical layouts (all complex128, C order):
  links  : [4][T][X][Y][Z][3][3]   mu = 0 is the time direction (x0 of Sec. 2)
  spinor : [nrhs][V/2][2 flavor][4 spin][3 color] on ODD sites, where the odd
           half-index of site (t,x,y,z) is lex >> 1 with
           lex = ((t*X + x)*Y + y)*Z + z, parity = (t+x+y+z) & 1.

Random numbers come from numpy's Philox4x32-10 counter-based generator
(Salmon et al., SC'11), seeded per field/vector, so the same seed gives the
same field on every machine.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann", "random_su3_field", "unit_gauge_field", "gaussian_rhs",
    "shift_set", "odd_sites", "random_gauge_transform",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_a, shape [8,3,3]."""
    l = np.zeros((8, 3, 3), np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j; l[1][1, 0] = 1j
    l[2][0, 0] = 1; l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j; l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j; l[6][2, 1] = 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3); l[7][2, 2] = -2 / np.sqrt(3)
    return l


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Project [...,3,3] matrices onto SU(3): normalise row 0, Gram-Schmidt
    row 1, row 2 = conj(row0 x row1) so that det = +1 up to rounding."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def random_su3_field(dims, roughness: float, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    """U = exp(i r H) per link, H = sum_a eta_a lambda_a / 2 with eta_a ~ N(0,1)
    (a seeded Gaussian traceless Hermitian matrix), then reunitarised.

    dims = (T, X, Y, Z), all even.  Returns complex128 [4,T,X,Y,Z,3,3]."""
    T, X, Y, Z = (int(d) for d in dims)
    n = 4 * T * X * Y * Z
    lam = gell_mann() / 2.0
    rng = _rng(seed)
    out = np.empty((n, 3, 3), np.complex128)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        eta = rng.standard_normal((m, 8))
        h = np.einsum("na,aij->nij", eta, lam)
        w, v = np.linalg.eigh(h)
        u = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * roughness * w), np.conj(v))
        out[s:s + m] = _reunitarise(u)
    return out.reshape(4, T, X, Y, Z, 3, 3)


def unit_gauge_field(dims) -> np.ndarray:
    """Free field U_mu(x) = 1."""
    T, X, Y, Z = (int(d) for d in dims)
    u = np.zeros((4, T, X, Y, Z, 3, 3), np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """A random SU(3) matrix per site, complex128 [T,X,Y,Z,3,3]."""
    T, X, Y, Z = (int(d) for d in dims)
    return random_su3_field((1, T * X * Y, Z, 1), 1.0, seed)[0].reshape(T, X, Y, Z, 3, 3)


def gaussian_rhs(dims, seed: int, nrhs: int = 1) -> np.ndarray:
    """Complex Gaussian right-hand side(s) on odd sites: Re, Im ~ N(0,1) iid.
    Returns complex128 [nrhs, V/2, 2, 4, 3]."""
    T, X, Y, Z = (int(d) for d in dims)
    vh = T * X * Y * Z // 2
    out = np.empty((nrhs, vh, 2, 4, 3), np.complex128)
    for k in range(nrhs):
        rng = _rng(seed + k)
        z = rng.standard_normal((vh, 2, 4, 3, 2))
        out[k] = z[..., 0] + 1j * z[..., 1]
    return out


def shift_set(n: int, lo: float, hi: float) -> np.ndarray:
    """n log-spaced shifts sigma_i in [lo, hi], inclusive, strictly descending."""
    return np.geomspace(hi, lo, n)


def odd_sites(dims) -> np.ndarray:
    """Full-lattice lexicographic indices of the odd sites, in half-index order."""
    T, X, Y, Z = (int(d) for d in dims)
    t, x, y, z = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
    lex = (((t * X + x) * Y + y) * Z + z).ravel()
    par = ((t + x + y + z) & 1).ravel()
    return lex[par == 1]
