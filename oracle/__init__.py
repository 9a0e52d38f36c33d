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


def lagrange_degree(nodes_nearest_first, target, gamma_max) -> tuple:
    """Degree truncation of App. B ("in case of diverging growths one can truncate the
    degree of the interpolation"): the largest k' such that the first k' nodes of the
    nearest-first list give gamma_k'(target) <= gamma_max, with gamma_1 = 1.  Returns
    (k', gamma_k'(target))."""
    nodes = [float(v) for v in nodes_nearest_first]
    best, gbest = 1, 1.0
    for k in range(2, len(nodes) + 1):
        g = lebesgue(nodes[:k], target)
        if g <= gamma_max:
            best, gbest = k, g
    return best, gbest


def lagrange_guess(nodes, xs, target) -> np.ndarray:
    """x~(m) = sum_i l_{i,k}(m) x_i (Sec. 4.2.1, Eq. for p(m))."""
    w = lagrange_weights(nodes, target)
    out = np.zeros_like(np.asarray(xs[0], np.complex128))
    for wi, xi in zip(w, xs):
        out = out + wi * np.asarray(xi, np.complex128)
    return out


# ---------------------------------------------------------------- multigrid
# Aggregation-based two-level construction of Sec. 3 (DD-alphaAMG): blocks of
# the fine lattice, a prolongator P built from test vectors that is
# Gamma_5-compatible (each block's vectors split by chirality, Sec. 3:
# Gamma_5 P = P Gamma_5,c) and orthonormal (P^+ P = 1), the coarse operator
# D_c = P^+ D P (Sec. 3), its doublet form (Sec. 3.2, Eq. "non-degenerate_coarse")
# and the error propagation of the two-level method (Eq. "error_propagation").
#
# Layouts (single flavour, full lattice): fine vectors complex [V][4 spin][3 colour]
# in lexicographic site order; coarse vectors complex [nblock][2 chirality][Nv],
# blocks in lexicographic order of their block coordinates (t slowest).
# Chirality 0 = spins 0, 1 (gamma_5 = +1), chirality 1 = spins 2, 3.

def mg_block_of_site(dims, bdims) -> np.ndarray:
    """Block index of every lexicographic site (blocks of size bdims)."""
    T, X, Y, Z = dims
    bt, bx, by, bz = bdims
    nb = (T // bt, X // bx, Y // by, Z // bz)
    t, x, y, z = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
    b = (((t // bt) * nb[1] + x // bx) * nb[2] + y // by) * nb[3] + z // bz
    return b.ravel()


def mg_prolongator(dims, bdims, vecs) -> np.ndarray:
    """Dense P [V*12, nblock*2*Nv]: for each block and chirality, the test
    vectors restricted there and orthonormalised by modified Gram-Schmidt in
    the order given (Sec. 3: aggregation over O(20) test vectors, Gamma_5
    compatible).  vecs: complex [Nv][V][4][3]."""
    vecs = np.asarray(vecs, np.complex128)
    nv = vecs.shape[0]
    V = int(np.prod(dims))
    blk = mg_block_of_site(dims, bdims)
    nblock = int(blk.max()) + 1
    P = np.zeros((V * 12, nblock * 2 * nv), np.complex128)
    for b in range(nblock):
        sites = np.nonzero(blk == b)[0]
        for chi in range(2):
            rows = (sites[:, None] * 12 + (chi * 6 + np.arange(6))[None, :]).ravel()
            cols = []
            for k in range(nv):
                v = vecs[k].reshape(V * 12)[rows].copy()
                for u in cols:
                    v = v - np.vdot(u, v) * u
                v = v / np.linalg.norm(v)
                cols.append(v)
            for k, v in enumerate(cols):
                P[rows, b * 2 * nv + chi * nv + k] = v
    return P


def wilson_apply(act: Action, links, psi_single) -> np.ndarray:
    """Single-flavour D_W (hopping form, Eq. "Wilson" with c_sw = 0) through
    the doublet oracle with mu_bar = eps_bar = 0 and the second flavour zero."""
    a0 = action(act.dims, act.kappa, 0.0, 0.0, apbc=act.apbc, paper_norm=act.paper_norm)
    V = int(np.prod(act.dims))
    psi = np.zeros((V, 2, 4, 3), np.complex128)
    psi[:, 0] = np.asarray(psi_single).reshape(V, 4, 3)
    return dnd(a0, links, psi)[:, 0]


def mg_coarse_wilson(act: Action, links, P) -> np.ndarray:
    """D_W,c = P^+ D_W P (Sec. 3), column by column."""
    V = int(np.prod(act.dims))
    DP = np.empty_like(P)
    for j in range(P.shape[1]):
        DP[:, j] = wilson_apply(act, links, P[:, j].reshape(V, 4, 3)).ravel()
    return P.conj().T @ DP


def mg_coarse_nd(Dcw, nblock, nv, mu_c, eps_c) -> np.ndarray:
    """Doublet coarse operator (Sec. 3.2, Eq. "non-degenerate_coarse"):
    D_ND,c = D_W,c (x) 1_2 + i mu_c (Gamma_5,c (x) tau_3) - eps_c (1 (x) tau_1),
    in the coarse layout [block][flavour][chirality][Nv].  In the hopping
    normalisation mu_c = 2 kappa mu_bar, eps_c = 2 kappa eps_bar."""
    n = nblock * 2 * nv
    out = np.zeros((2 * n, 2 * n), np.complex128)
    g5c = np.tile(np.repeat([1.0, -1.0], nv), nblock)

    def idx(f):  # coarse ND index of (block, flavour f, chirality, k)
        b = np.repeat(np.arange(nblock), 2 * nv)
        r = np.tile(np.arange(2 * nv), nblock)
        return b * 4 * nv + f * 2 * nv + r
    i0, i1 = idx(0), idx(1)
    out[np.ix_(i0, i0)] = Dcw + np.diag(1j * mu_c * g5c)
    out[np.ix_(i1, i1)] = Dcw - np.diag(1j * mu_c * g5c)
    out[i0, i1] = -eps_c
    out[i1, i0] = -eps_c
    return out


def dnd_odd_shift(act: Action, links, psi_full, s) -> np.ndarray:
    """D' psi = D_ND psi + i s (gamma_5 (x) tau_1) psi on odd sites: the
    full-lattice operator whose odd Schur complement is Mhat + i s gamma_5 tau_1,
    the case-C system (Qhat + i s) y = b written as (Mhat + i s g5 t1) y = g5 t1 b
    (Sec. 3.1, Eq. "lindif")."""
    psi = _c128(psi_full)
    out = dnd(act, links, psi)
    T, X, Y, Z = act.dims
    t, x, y, z = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
    odd = (((t + x + y + z) & 1) == 1).ravel()
    g5 = np.array([1.0, 1.0, -1.0, -1.0])
    term = 1j * s * g5[None, None, :, None] * psi[:, ::-1]   # tau_1 swaps the flavours
    out[odd] += term[odd]
    return out


def mg_coarse_nd_odd_shift(act: Action, links, P, nv: int, s, chunk: int = 256) -> np.ndarray:
    """Coarse operator of the case-C systems (Sec. 3.1 Eq. "lindif", Sec. 3.2):
    P_ND^+ D' P_ND with D' = D_ND + i s (gamma_5 (x) tau_1) Pi_odd (dnd_odd_shift)
    and P_ND = P (x) 1_2, formed by applying D' to every column of P_ND and
    projecting with P^+ (no block-structure shortcut).  Coarse ND layout as in
    mg_coarse_nd: index (block, flavour, chirality, k) -> b 4 Nv + f 2 Nv + chi Nv + k."""
    P = np.asarray(P, np.complex128)
    V = int(np.prod(act.dims))
    ncol = P.shape[1]
    nblock = ncol // (2 * nv)
    Ph = P.conj().T
    out = np.zeros((2 * ncol, 2 * ncol), np.complex128)

    def rows(f):
        b = np.repeat(np.arange(nblock), 2 * nv)
        r = np.tile(np.arange(2 * nv), nblock)
        return b * 4 * nv + f * 2 * nv + r
    for j0 in range(0, 2 * ncol, chunk):
        js = range(j0, min(j0 + chunk, 2 * ncol))
        Y = np.empty((2, V * 12, len(js)), np.complex128)
        for q, j in enumerate(js):
            b, rem = divmod(j, 4 * nv)
            f, r = divmod(rem, 2 * nv)
            fine = np.zeros((V, 2, 4, 3), np.complex128)
            fine[:, f] = P[:, b * 2 * nv + r].reshape(V, 4, 3)
            y = dnd_odd_shift(act, links, fine, s)
            Y[0, :, q] = y[:, 0].ravel()
            Y[1, :, q] = y[:, 1].ravel()
        for f in range(2):
            out[rows(f), j0:j0 + len(js)] = Ph @ Y[f]
    return out


# ------------------------------------------------------------ learned guess
# Not in the paper: a small network proposes interpolation weights over the
# solutions x_j of 8 already-solved shifts for a smaller target shift sigma_t,
# extending the Lagrange weights of Sec. 4.2.1.  With sum_j w_j = 1 (partition
# of unity, App. B) and exact x_j, the residual of the guess is
#   b - (Qhat^2 + sigma_t) sum_j w_j x_j = - sum_j w_j (sigma_t - sigma_j) x_j      (App. B)
# so |residual|^2 = w^T H w with H = Re(D G D), G_jk = <x_j, x_k> / |b|^2,
# D = diag(sigma_t - sigma_j): a loss that needs no operator application.
#
# Head: the network (F -> 64 -> 64 -> 2, tanh) outputs two log-poles o_k,
# p_k = exp(o_k), and the weights are those of Lagrange interpolation (Sec.
# 4.2.1) applied to prod_k (p_k + sigma) x(sigma) and divided back:
#   w_j = l_j(sigma_t) prod_k (p_k + sigma_j) / (p_k + sigma_t).
# They reproduce every x(sigma) = P_7(sigma) / prod_k (p_k + sigma) exactly, sum
# to 1 for any poles (Lagrange reproduces the degree-2 numerator), and tend to
# the Lagrange weights as p_k -> infinity.  The guess residual is tiny (down to
# ~1e-9 |b|), which raw FP32 weights could not resolve; poles can be predicted
# in FP32 and the weights are then formed in FP64.
# Per-sample loss log(w^T H w) (scale free across shifts); batch loss = mean.
MLP_H = 64
MLP_K = 8      # solved shifts the guess combines
MLP_P = 2      # network outputs: log-poles


def mlp_sizes(F):
    """Parameter blocks: input mean mu and inverse std isd (x -> (x - mu) isd, not
    trained), then W1 b1 W2 b2 W3 b3."""
    return [(F,), (F,), (MLP_H, F), (MLP_H,), (MLP_H, MLP_H), (MLP_H,), (MLP_P, MLP_H), (MLP_P,)]


def mlp_unflatten(theta, F):
    out, o = [], 0
    for shp in mlp_sizes(F):
        n = int(np.prod(shp))
        out.append(np.asarray(theta[o:o + n], np.float64).reshape(shp))
        o += n
    return out


def pole_weights(S, poles):
    """w [N, 8] from S [N, 9] = (sigma_t, sigma_1..sigma_8) and poles [N, P]:
    w_j = l_j(sigma_t) prod_k (p_k + sigma_j) / (p_k + sigma_t)."""
    S = np.asarray(S, np.float64)
    poles = np.asarray(poles, np.float64)
    t, nodes = S[:, 0], S[:, 1:]
    w = np.stack([lagrange_weights(nodes[n], t[n]) for n in range(len(S))])
    for k in range(poles.shape[1]):
        p = poles[:, k:k + 1]
        w = w * (p + nodes) / (p + t[:, None])
    return w


def mlp_forward(theta, X, S):
    """Weights w [N, 8] (each row sums to 1) for features X [N, F] and shifts S [N, 9]."""
    mu, isd, W1, b1, W2, b2, W3, b3 = mlp_unflatten(theta, np.shape(X)[1])
    X = (np.asarray(X, np.float64) - mu) * isd
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    o = h2 @ W3.T + b3
    return pole_weights(S, np.exp(o))


def mlp_loss_grad(theta, X, S, H, floor=0.0):
    """Mean over samples of log(w^T H w + floor) and its gradient in theta (plain
    backpropagation, written out layer by layer).  floor ~ rho^2 stands for the
    residuals rho |b| that the solved x_j still carry (the guess residual is not
    known below that)."""
    S = np.asarray(S, np.float64)
    H = np.asarray(H, np.float64)
    N, F = np.shape(X)
    mu, isd, W1, b1, W2, b2, W3, b3 = mlp_unflatten(theta, F)
    X = (np.asarray(X, np.float64) - mu) * isd
    a1 = X @ W1.T + b1
    h1 = np.tanh(a1)
    a2 = h1 @ W2.T + b2
    h2 = np.tanh(a2)
    o = h2 @ W3.T + b3
    p = np.exp(o)
    w = pole_weights(S, p)
    q = np.einsum("ni,nij,nj->n", w, H, w) + floor
    loss = float(np.mean(np.log(q)))
    dw = (2.0 * np.einsum("nij,nj->ni", H, w)) / q[:, None] / N
    # d w_j / d o_k = w_j p_k (1/(p_k + sigma_j) - 1/(p_k + sigma_t))
    t, nodes = S[:, :1], S[:, 1:]
    do = np.stack([np.sum(dw * w * p[:, k:k + 1] * (1.0 / (p[:, k:k + 1] + nodes) - 1.0 / (p[:, k:k + 1] + t)),
                          axis=1) for k in range(MLP_P)], axis=1)
    gW3 = do.T @ h2
    gb3 = do.sum(axis=0)
    dh2 = do @ W3
    da2 = dh2 * (1 - h2 ** 2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * (1 - h1 ** 2)
    gW1 = da1.T @ X
    gb1 = da1.sum(axis=0)
    grad = np.concatenate([np.zeros(2 * F), gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, grad


def span_optimal_weights(H):
    """argmin_w w^T H w subject to sum_j w_j = 1:  w = H^-1 1 / (1^T H^-1 1)."""
    H = np.asarray(H, np.float64)
    one = np.ones(H.shape[-1])
    v = np.linalg.solve(H, one)
    return v / v.sum()


def guess_quadratic_form(sig_nodes, sig_t, xs, bnorm2):
    """H = Re(D G D) with G_jk = <x_j, x_k> / |b|^2 and D = diag(sigma_t - sigma_j)."""
    X = np.stack([np.asarray(x, np.complex128).ravel() for x in xs])
    G = (X.conj() @ X.T) / bnorm2
    d = float(sig_t) - np.asarray(sig_nodes, np.float64)
    return np.real(d[:, None] * G * d[None, :])


# ------------------------------------------------------------ rational approximation
# Zolotarev's optimal rational approximation of 1/sqrt(y) on eps < y < 1 (Sec. 4.1,
# Eqs. "rational", "deviation", "zolotarev_shifts"), written from the paper's closed forms
# with scipy's Jacobi elliptic functions as the library primitive (parameter m = k^2,
# modulus k = sqrt(1 - eps)):
#   v = K(k) / (2n + 1),  c_k = cs^2(k v, k),  s_k = sn^2(k v, k),
#   d = (1 - eps)^((2n+1)/2) prod_j s_(2j-1)^2,  a = 2/(1 + sqrt(1 - d^2)) prod_j s_(2j-1)/s_(2j),
#   delta = d^2 / (1 + sqrt(1 - d^2))^2
# (the paper's closed form for delta prints the denominator unsquared, which is twice the
# maximum of |1 - sqrt(y) R(y)| that defines delta in Eq. "deviation"; the definition decides),
#   R(y) = a prod_j (y + c_(2j-1)) / (y + c_(2j)) = a (1 + sum_i q_i / (y + c_(2i))),
#   q_i = (c_(2i-1) - c_(2i)) prod_{j != i} (c_(2j-1) - c_(2i)) / (c_(2j) - c_(2i))   (Eq. "ratapp").
def zolotarev(n, eps):
    """(a, c[0..2n-1] = c_1..c_2n, q[0..n-1], delta) for R_{n,eps}."""
    from scipy.special import ellipj, ellipk
    m = 1.0 - float(eps)
    v = ellipk(m) / (2 * n + 1)
    k = np.arange(1, 2 * n + 1)
    sn, cn, _, _ = ellipj(k * v, m)
    c = (cn / sn) ** 2
    s = sn ** 2
    d = (1.0 - eps) ** ((2 * n + 1) / 2.0) * np.prod(s[0::2] ** 2)
    a = 2.0 / (1.0 + np.sqrt(1.0 - d * d)) * np.prod(s[0::2] / s[1::2])
    delta = d * d / (1.0 + np.sqrt(1.0 - d * d)) ** 2
    q = np.empty(n)
    for i in range(n):
        num, den = c[2 * i], c[2 * i + 1]
        p = num - den
        for j in range(n):
            if j != i:
                p *= (c[2 * j] - den) / (c[2 * j + 1] - den)
        q[i] = p
    return a, c, q, delta


def zolotarev_eval(a, c, y):
    """R(y) in the product form."""
    y = np.asarray(y, np.float64)
    r = np.full(y.shape, a)
    for j in range(len(c) // 2):
        r = r * (y + c[2 * j]) / (y + c[2 * j + 1])
    return r


def rational_apply(act: Action, links, b, n, lam_min, lam_max, rho=1e-12):
    """x = R(Qhat^2/lam_max) b / sqrt(lam_max) ~ (Qhat^2)^(-1/2) b via the oracle's multi-shift CG on
    the shifts lam_max c_(2i) and the partial-fraction form (Eq. "ratapp")."""
    a, c, q, delta = zolotarev(n, lam_min / lam_max)
    sig = lam_max * c[1::2]
    xs = mms_cg(act, links, b, sig, rho=rho)["x"]
    x = np.asarray(b, np.complex128).copy()
    for i in range(n):
        x = x + lam_max * q[i] * xs[i]
    return a / np.sqrt(lam_max) * x, delta


# ------------------------------------------------------------ hybrid cost model
# Sec. 4.3: time-to-solution fits of CG (Eq. "CGtime2") and MG (Eq. "MGtime2") per shift
# m^2 = sigma, and the hybrid's cost with the n largest shifts by MMS-CG (Eq. "costwo"):
#   t_CG(s) = a + b / ln(1 - 2 / (sqrt(kappa(s)) + 1)),  kappa(s) = (lmax + s) / (lmin + s)
#   t_MG(s) = A + B / ln(1 - (C + s) / (L + s))        (L = the spectrum's upper end, 4.7 in the paper)
#   c_HY(n) = t_CG(s_n) + sum_{i > n} t_MG(s_i),  shifts descending, n = 1..N
def t_cg(s, a, b, lmin, lmax):
    s = np.asarray(s, np.float64)
    kappa = (lmax + s) / (lmin + s)
    return a + b / np.log(1.0 - 2.0 / (np.sqrt(kappa) + 1.0))


def t_mg(s, A, B, C, L):
    s = np.asarray(s, np.float64)
    return A + B / np.log(1.0 - (C + s) / (L + s))


def hybrid_cost(sig, cg, mg):
    """c_HY(n) for n = 1..N (list) and the n that minimises it; cg = (a, b, lmin, lmax), mg = (A, B, C, L)."""
    sig = np.asarray(sig, np.float64)
    N = len(sig)
    tm = t_mg(sig, *mg)
    cost = [float(t_cg(sig[n - 1], *cg) + tm[n:].sum()) for n in range(1, N + 1)]
    return cost, int(np.argmin(cost)) + 1


def fit_cg_time(sig, t, lmin, lmax):
    """Least-squares (a, b) of Eq. "CGtime2" (linear in a, b)."""
    x = 1.0 / np.log(1.0 - 2.0 / (np.sqrt((lmax + np.asarray(sig)) / (lmin + np.asarray(sig))) + 1.0))
    M = np.stack([np.ones_like(x), x], 1)
    (a, b), *_ = np.linalg.lstsq(M, np.asarray(t, np.float64), rcond=None)
    return float(a), float(b)


def fit_mg_time(sig, t, L, grid=2001):
    """(A, B, C) of Eq. "MGtime2": least squares in (A, B) for each C on a log grid in (0, L), best C."""
    sig = np.asarray(sig, np.float64)
    t = np.asarray(t, np.float64)
    best = None
    for C in np.geomspace(1e-8 * L, 0.999 * L, grid):
        x = 1.0 / np.log(1.0 - (C + sig) / (L + sig))
        M = np.stack([np.ones_like(x), x], 1)
        sol, *_ = np.linalg.lstsq(M, t, rcond=None)
        r = float(np.sum((M @ sol - t) ** 2))
        if best is None or r < best[0]:
            best = (r, float(sol[0]), float(sol[1]), float(C))
    return best[1], best[2], best[3]


# ------------------------------------------- equivalent solutions (App. A, squared operator)
def single_system_solves(act: Action, links, b, mu, rho=1e-10):
    """Solutions of the single systems (Qhat +- i mu) x_pm = b (App. A, methods E, F and D).
    Qhat is hermitian, so (Qhat +- i mu)^-1 = (Qhat -+ i mu) (Qhat^2 + mu^2)^-1.
      E (normal equation, transformed right-hand side): x = CG[(Qhat -+ i mu) b], stopped
        at rho |(Qhat -+ i mu) b|;
      F (normal equation, transformed solution): y = CG[b], x = (Qhat -+ i mu) y;
      D (a solve of the single system to |b - (Qhat +- i mu) x| <= rho |b|): E followed by one
        F step on its residual, x += (Qhat -+ i mu) CG[r], stopped at rho |b| / |r|.
    Returns {("E"|"F"|"D", +1|-1): x}; CG is the oracle's plain CG on (Qhat^2 + mu^2)."""
    b = _c128(b)
    s2 = float(mu) * float(mu)
    qb = qhat(act, links, b)
    y, _ = cg(act, links, b, s2, rho)
    qy = qhat(act, links, y)
    out = {}
    bn = np.linalg.norm(b)
    for sg in (+1, -1):
        xe, _ = cg(act, links, qb - sg * 1j * mu * b, s2, rho)
        out[("E", sg)] = xe
        out[("F", sg)] = qy - sg * 1j * mu * y
        r = b - (qhat(act, links, xe) + sg * 1j * mu * xe)
        rn = np.linalg.norm(r)
        xd = xe.copy()
        if rn > rho * bn:
            d, _ = cg(act, links, r, s2, min(0.5, rho * bn / rn))
            xd = xd + (qhat(act, links, d) - sg * 1j * mu * d)
        out[("D", sg)] = xd
    return out


def equivalent_solutions(act: Action, links, b, mu, rho=1e-10):
    """The three solutions of (Qhat^2 + mu^2) x = b compared in App. A (squared
    twisted-mass operator):
      A: x_A = CG[b] (Eq. "direct");
      B: x_+ = (Qhat + i mu)^-1 b, then x_B = (Qhat - i mu)^-1 x_+, each single system solved
         as method D above, the second to |x_+ - (Qhat - i mu) x_B| <= rho |x_+| (Eq. "two-step");
      C: x_C = i/(2 mu) (x_+ - x_-), x_pm by method D (Eq. "linear-combination").
    Returns {"A", "B", "C", "p", "m"} (p, m = x_+, x_-)."""
    b = _c128(b)
    one = single_system_solves(act, links, b, mu, rho)
    xp, xm = one[("D", +1)], one[("D", -1)]
    xA, _ = cg(act, links, b, float(mu) * float(mu), rho)
    xB = single_system_solves(act, links, xp, -mu, rho)[("D", +1)]   # (Qhat - i mu)^-1 x_+
    xC = 1j / (2.0 * mu) * (xp - xm)
    return {"A": xA, "B": xB, "C": xC, "p": xp, "m": xm}


def equivalent_bounds(rho, bnorm, lmin, lmax, mu):
    """Upper limits of App. A for |r| and |e| of methods A, B, C (squared operator) and
    D, E, F (single systems), for sub-solves that meet their stopping criteria; lmin,
    lmax are the extreme eigenvalues of Qhat^2 (the paper's lambda^2_min, lambda^2_max)."""
    m2 = float(mu) ** 2
    lo, hi = lmin + m2, lmax + m2
    return {
        "A": (rho * bnorm, rho * bnorm / lo),
        "B": ((1.0 + np.sqrt(hi / lo)) * rho * bnorm, 2.0 * rho * bnorm / lo),
        "C": (rho * np.sqrt(hi) * bnorm / abs(mu), rho * bnorm / (abs(mu) * np.sqrt(lo))),
        "D": (rho * bnorm, rho * bnorm / np.sqrt(lo)),
        "E": (rho * bnorm * np.sqrt(hi / lo), rho * bnorm * np.sqrt(hi) / lo),
        "F": (rho * bnorm, rho * bnorm / np.sqrt(lo)),
    }
