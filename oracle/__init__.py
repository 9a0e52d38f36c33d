"""FP64 CPU oracle for arXiv:1805.09584 (non-degenerate twisted-mass shifted systems).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package.  It shares no code with
the GPU library (`paper_1805_09584_gb300`): the stencil, the even-odd Schur
complement and the multi-shift CG live in plain C (`tmnd_oracle.c`, written
from the paper's equations with no spin projection, compression or fusion);
the Lagrange interpolation and the dense-matrix helpers are plain numpy below.

Every function names the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tmnd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over sites, IEEE FP64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Action(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("kappa", ctypes.c_double),
                ("mu_bar", ctypes.c_double), ("eps_bar", ctypes.c_double),
                ("apbc", ctypes.c_int), ("paper_norm", ctypes.c_int)]


def action(dims, kappa, mu_bar, eps_bar, apbc=True, paper_norm=False) -> Action:
    a = Action()
    for i in range(4):
        a.dims[i] = int(dims[i])
    a.kappa, a.mu_bar, a.eps_bar = float(kappa), float(mu_bar), float(eps_bar)
    a.apbc, a.paper_norm = int(bool(apbc)), int(bool(paper_norm))
    return a


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        d = ctypes.c_void_p
        A = P(Action)
        L.or_gamma.argtypes = [ctypes.c_int, d]
        L.or_dnd.argtypes = [A, d, d, d, ctypes.c_int]
        L.or_schur.argtypes = [A, d, d, d, ctypes.c_int]
        L.or_qhat.argtypes = [A, d, d, d]
        L.or_qhat2.argtypes = [A, d, d, d, ctypes.c_double]
        L.or_cg.argtypes = [A, d, d, ctypes.c_double, ctypes.c_double, ctypes.c_int, d]
        L.or_cg.restype = ctypes.c_int
        L.or_mms_cg.argtypes = [A, d, d, ctypes.c_int, ctypes.c_int, d, ctypes.c_double,
                                ctypes.c_int, d, d, d]
        L.or_mms_cg.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def nthreads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


# --------------------------------------------------------------- operators
def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu = 0..3) or gamma_5 (mu = 5) of the chiral basis, Sec. 2."""
    out = np.zeros((4, 4), np.complex128)
    lib().or_gamma(mu, _p(out))
    return out


def dnd(act: Action, links, psi_full, dagger=False) -> np.ndarray:
    """Full-lattice D_ND (Sec. 2, Eqs. "non-degenerate" and "Wilson", c_sw = 0),
    or its adjoint.  psi_full: complex [V,2,4,3]."""
    links = _c128(links); psi = _c128(psi_full)
    out = np.empty_like(psi)
    lib().or_dnd(ctypes.byref(act), _p(links), _p(psi), _p(out), int(dagger))
    return out


def schur(act: Action, links, psi_odd, dagger=False) -> np.ndarray:
    """Mhat = D_oo - D_oe D_ee^-1 D_eo on odd sites (Sec. 2, even-odd
    reduction), or Mhat^+.  psi_odd: complex [V/2,2,4,3]."""
    links = _c128(links); psi = _c128(psi_odd)
    out = np.empty_like(psi)
    lib().or_schur(ctypes.byref(act), _p(links), _p(psi), _p(out), int(dagger))
    return out


def qhat(act: Action, links, psi_odd) -> np.ndarray:
    """Qhat = (gamma_5 (x) tau_1) Mhat (Sec. 2, Eq. "g5tau1-hermiticity")."""
    links = _c128(links); psi = _c128(psi_odd)
    out = np.empty_like(psi)
    lib().or_qhat(ctypes.byref(act), _p(links), _p(psi), _p(out))
    return out


def qhat2(act: Action, links, psi_odd, sigma=0.0) -> np.ndarray:
    """(Qhat^2 + sigma) psi = Mhat^+ Mhat psi + sigma psi (Sec. 1, Eq. "shifted_linear")."""
    links = _c128(links); psi = _c128(psi_odd)
    out = np.empty_like(psi)
    lib().or_qhat2(ctypes.byref(act), _p(links), _p(psi), _p(out), float(sigma))
    return out


def true_residual(act: Action, links, b, x, sigma) -> float:
    """|b - (Qhat^2 + sigma) x| / |b|, the stopping quantity of the paper's
    relative-residual criterion (Sec. 3.1)."""
    r = _c128(b) - qhat2(act, links, x, sigma)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


# ----------------------------------------------------------------- solvers
def cg(act: Action, links, b, sigma, rho=1e-10, maxiter=100000):
    """Plain CG on (Qhat^2 + sigma) x = b (case A of Sec. 3.1). Returns (x, iters)."""
    links = _c128(links); b = _c128(b)
    x = np.empty_like(b)
    it = lib().or_cg(ctypes.byref(act), _p(links), _p(b), float(sigma), float(rho), int(maxiter), _p(x))
    return x, it


def mms_cg(act: Action, links, b, sigmas, rho=1e-10, maxiter=100000, nsolve=None):
    """Multi-mass-shift CG (Sec. 1 "standard" solver; Sec. 4.2.2).  Shifts
    strictly descending; the first `nsolve` (default all) must converge and
    the last of them is the base system; later ones are guess shifts.
    Returns dict(x [nshift,...], iters, conv_iter, zeta)."""
    links = _c128(links); b = _c128(b)
    sig = np.ascontiguousarray(sigmas, np.float64)
    ns = len(sig)
    nsolve = ns if nsolve is None else int(nsolve)
    x = np.empty((ns,) + b.shape, np.complex128)
    conv = np.empty(ns, np.int32)
    zeta = np.empty(ns, np.float64)
    it = lib().or_mms_cg(ctypes.byref(act), _p(links), _p(b), ns, nsolve, _p(sig), float(rho),
                         int(maxiter), _p(x), _p(conv), _p(zeta))
    return {"x": x, "iters": it, "conv_iter": conv, "zeta": zeta}


# ------------------------------------------------------------ dense helpers
def dense(apply, n_complex: int) -> np.ndarray:
    """Column-probe a linear map on C^n into a dense matrix (slow; small lattices)."""
    M = np.empty((n_complex, n_complex), np.complex128)
    e = np.zeros(n_complex, np.complex128)
    for j in range(n_complex):
        e[j] = 1.0
        M[:, j] = np.asarray(apply(e)).ravel()
        e[j] = 0.0
    return M


# ------------------------------------------------------------------ Lagrange
def lagrange_weights(nodes, target) -> np.ndarray:
    """l_{i,k}(m) = prod_{j != i} (m - m_j)/(m_i - m_j)  (Sec. 4.2.1; App. B),
    evaluated at m = target, in the shift variable sigma."""
    nodes = [float(v) for v in nodes]
    k = len(nodes)
    w = np.ones(k)
    for i in range(k):
        for j in range(k):
            if j != i:
                w[i] *= (target - nodes[j]) / (nodes[i] - nodes[j])
    return w


def lebesgue(nodes, target) -> float:
    """gamma_k(m) = sum_i |l_{i,k}(m)|, the Lebesgue function (App. B)."""
    return float(np.sum(np.abs(lagrange_weights(nodes, target))))


def lagrange_guess(nodes, xs, target) -> np.ndarray:
    """x~(m) = sum_i l_{i,k}(m) x_i (Sec. 4.2.1, Eq. for p(m))."""
    w = lagrange_weights(nodes, target)
    out = np.zeros_like(np.asarray(xs[0], np.complex128))
    for wi, xi in zip(w, xs):
        out = out + wi * np.asarray(xi, np.complex128)
    return out
