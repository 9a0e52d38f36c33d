"""Pins for the oracle's operator: each checks the C oracle against something
other than itself (closed forms, symmetries the paper states, dense linear
algebra, gauge covariance), so that a dropped term, a wrong sign, a swapped
projector, a wrong link conjugation or a broken boundary fails one of them."""
import numpy as np
import pytest

import oracle
import synth

KAPPA, MU, EPS = 0.16, 0.1, 0.11
TAU1 = np.array([[0, 1], [1, 0]], np.complex128)
TAU3 = np.array([[1, 0], [0, -1]], np.complex128)


def _rand_vec(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


# ------------------------------------------------------------------ gammas
def test_gamma_clifford_and_gamma5(oracle_lib):
    """{gamma_mu, gamma_nu} = 2 delta_{mu nu}; gamma_5 = gamma_0 gamma_1 gamma_2
    gamma_3 = diag(1,1,-1,-1) in the chiral representation (Sec. 2)."""
    g = [oracle.gamma(m) for m in range(4)]
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T, atol=0)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2 * (a == b) * np.eye(4), atol=0)
    g5 = oracle.gamma(5)
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3], atol=0)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=0)


# -------------------------------------------------------- free-field spectra
def _free_full_closed_form(dims, kappa, mu, eps, apbc, paper_norm):
    """Free field (U = 1): D_ND at momentum p is
         M(p) + i sum_mu gamma_mu sin p_mu + i mu gamma_5 tau_3 - eps tau_1,
       M(p) = 1/(2 kappa) - 4 + sum_mu (1 - cos p_mu)   (paper's normalisation),
    and Q_ND^2 = D_ND^+ D_ND has eigenvalues (sqrt(M^2 + mu^2) +- eps)^2 + sum sin^2 p,
    each 4-fold in spin x flavour and 3-fold in colour.  Time momenta are
    (2n+1) pi / T for the antiperiodic boundary, 2 pi n / T otherwise."""
    T, X, Y, Z = dims
    m0 = 1.0 / (2 * kappa) - 4
    out = []
    for nt in range(T):
        pt = (2 * nt + 1) * np.pi / T if apbc else 2 * np.pi * nt / T
        for nx in range(X):
            for ny in range(Y):
                for nz in range(Z):
                    p = np.array([pt, 2 * np.pi * nx / X, 2 * np.pi * ny / Y, 2 * np.pi * nz / Z])
                    M = m0 + np.sum(1 - np.cos(p))
                    s2 = np.sum(np.sin(p) ** 2)
                    for sgn in (1, -1):
                        out += [(np.sqrt(M * M + mu * mu) + sgn * eps) ** 2 + s2] * 12
    scale = 1.0 if paper_norm else (2 * kappa) ** 2
    return np.sort(np.array(out)) * scale


@pytest.mark.parametrize("dims,apbc,paper_norm", [
    ((4, 2, 2, 2), True, True), ((4, 2, 2, 2), True, False),
    ((2, 2, 2, 4), False, False), ((2, 4, 2, 2), True, False)])
def test_free_field_full_spectrum(oracle_lib, dims, apbc, paper_norm):
    act = oracle.action(dims, KAPPA, MU, EPS, apbc=apbc, paper_norm=paper_norm)
    U = synth.unit_gauge_field(dims)
    V = int(np.prod(dims))
    D = oracle.dense(lambda v: oracle.dnd(act, U, v.reshape(V, 2, 4, 3)), V * 24)
    ev = np.sort(np.linalg.eigvalsh(D.conj().T @ D))
    cf = _free_full_closed_form(dims, KAPPA, MU, EPS, apbc, paper_norm)
    assert np.max(np.abs(ev - cf)) < 1e-12 * max(1.0, cf.max())


def _free_schur_closed_form(dims, kappa, mu, eps, apbc):
    """Hopping form, free field.  H(p) = sum_mu[(1-gamma_mu)e^{ip} + (1+gamma_mu)e^{-ip}]
    = 2 sum cos p - 2i sum gamma_mu sin p maps a plane wave on odd sites to the
    same wave on even sites (and back), so on odd sites the Schur complement
    A - kappa^2 H_oe A^-1 H_eo acts on the pair {p, p + (pi,pi,pi,pi)} as the
    8x8 matrix  Mhat(p) = A - kappa^2 H(p) A^-1 H(p)  (x colour identity),
    A = 1 + 2 i kappa mu gamma_5 tau_3 - 2 kappa eps tau_1."""
    T, X, Y, Z = dims
    g = [oracle.gamma(m) for m in range(4)]
    g5 = oracle.gamma(5)
    A = np.eye(8) + 2j * kappa * mu * np.kron(TAU3, g5) - 2 * kappa * eps * np.kron(TAU1, np.eye(4))
    Ainv = np.linalg.inv(A)
    seen = set()
    out = []
    for nt in range(T):
        for nx in range(X):
            for ny in range(Y):
                for nz in range(Z):
                    key = (nt, nx, ny, nz)
                    partner = ((nt + T // 2) % T, (nx + X // 2) % X, (ny + Y // 2) % Y, (nz + Z // 2) % Z)
                    if partner in seen:
                        continue
                    seen.add(key)
                    pt = (2 * nt + 1) * np.pi / T if apbc else 2 * np.pi * nt / T
                    p = [pt, 2 * np.pi * nx / X, 2 * np.pi * ny / Y, 2 * np.pi * nz / Z]
                    Hs = 2 * sum(np.cos(q) for q in p) * np.eye(4) - 2j * sum(gm * np.sin(q) for gm, q in zip(g, p))
                    H = np.kron(np.eye(2), Hs)
                    Mh = A - kappa ** 2 * H @ Ainv @ H
                    out += list(np.linalg.eigvalsh(Mh.conj().T @ Mh)) * 3
    return np.sort(np.array(out))


@pytest.mark.parametrize("dims,apbc", [((4, 2, 2, 2), True), ((2, 2, 2, 4), False), ((4, 4, 2, 2), True)])
def test_free_field_schur_spectrum(oracle_lib, dims, apbc):
    act = oracle.action(dims, KAPPA, MU, EPS, apbc=apbc)
    U = synth.unit_gauge_field(dims)
    Vh = int(np.prod(dims)) // 2
    Mh = oracle.dense(lambda v: oracle.schur(act, U, v.reshape(Vh, 2, 4, 3)), Vh * 24)
    ev = np.sort(np.linalg.eigvalsh(Mh.conj().T @ Mh))
    cf = _free_schur_closed_form(dims, KAPPA, MU, EPS, apbc)
    assert ev.shape == cf.shape
    assert np.max(np.abs(ev - cf)) < 1e-12


# --------------------------------------------------- rough-field symmetries
@pytest.fixture(scope="module")
def rough44():
    dims = (4, 4, 4, 4)
    return dims, synth.random_su3_field(dims, 0.5, 1234)


def test_qhat_hermitian_rough(oracle_lib, rough44):
    """Qhat = (Gamma_5 x tau_1) Mhat is hermitian (Sec. 2, Eq. "g5tau1-hermiticity"):
    <u, Qhat v> = <Qhat u, v> on a rough field."""
    dims, U = rough44
    act = oracle.action(dims, KAPPA, MU, EPS)
    Vh = 128
    u = _rand_vec((Vh, 2, 4, 3), 1)
    v = _rand_vec((Vh, 2, 4, 3), 2)
    lhs = np.vdot(u, oracle.qhat(act, U, v))
    rhs = np.vdot(oracle.qhat(act, U, u), v)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_schur_adjoint_rough(oracle_lib, rough44):
    """The oracle's Mhat^+ (built block by block from D^+) is the adjoint of Mhat:
    <u, Mhat v> = <Mhat^+ u, v>."""
    dims, U = rough44
    act = oracle.action(dims, KAPPA, MU, EPS)
    u = _rand_vec((128, 2, 4, 3), 3)
    v = _rand_vec((128, 2, 4, 3), 4)
    lhs = np.vdot(u, oracle.schur(act, U, v))
    rhs = np.vdot(oracle.schur(act, U, u, dagger=True), v)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_wilson_gamma5_hermitian_and_nd_spectrum_symmetric(oracle_lib):
    """Gamma_5-hermiticity of D_W (Sec. 2, Eq. "g5-hermiticity"): with mu = eps = 0
    the dense operator satisfies Gamma_5 D Gamma_5 = D^+.  For the ND operator
    the (Gamma_5 x tau_1)-hermiticity makes the spectrum symmetric about the
    real axis (Sec. 3.2)."""
    dims = (2, 2, 2, 4)
    U = synth.random_su3_field(dims, 0.7, 77)
    V = 32
    G5 = np.kron(np.eye(V * 2), np.kron(oracle.gamma(5), np.eye(3)))
    act0 = oracle.action(dims, KAPPA, 0.0, 0.0)
    D = oracle.dense(lambda v: oracle.dnd(act0, U, v.reshape(V, 2, 4, 3)), V * 24)
    assert np.max(np.abs(G5 @ D @ G5 - D.conj().T)) < 1e-14
    act = oracle.action(dims, KAPPA, MU, EPS)
    Dn = oracle.dense(lambda v: oracle.dnd(act, U, v.reshape(V, 2, 4, 3)), V * 24)
    G = np.kron(np.eye(V), np.kron(TAU1, np.kron(oracle.gamma(5), np.eye(3))))
    assert np.max(np.abs(G @ Dn @ G - Dn.conj().T)) < 1e-14
    ev = np.linalg.eigvals(Dn)
    evc = np.conj(ev)
    # every eigenvalue's conjugate is also an eigenvalue
    dist = np.min(np.abs(ev[:, None] - evc[None, :]), axis=1)
    assert dist.max() < 1e-8


def test_schur_matches_dense_block_elimination(oracle_lib):
    """Mhat = D_oo - D_oe D_ee^-1 D_eo computed from the dense full operator with
    numpy's inverse (Sec. 2, even-odd reduction) equals the oracle's Schur apply;
    this pins the odd-site ordering (half-index = lex >> 1) and the embedding."""
    dims = (2, 2, 2, 4)
    U = synth.random_su3_field(dims, 0.5, 5)
    act = oracle.action(dims, KAPPA, MU, EPS)
    V = 32
    D = oracle.dense(lambda v: oracle.dnd(act, U, v.reshape(V, 2, 4, 3)), V * 24)
    lex_odd = synth.odd_sites(dims)
    lex_even = np.setdiff1d(np.arange(V), lex_odd)
    io = (lex_odd[:, None] * 24 + np.arange(24)[None, :]).ravel()
    ie = (lex_even[:, None] * 24 + np.arange(24)[None, :]).ravel()
    Mh = D[np.ix_(io, io)] - D[np.ix_(io, ie)] @ np.linalg.inv(D[np.ix_(ie, ie)]) @ D[np.ix_(ie, io)]
    Mo = oracle.dense(lambda v: oracle.schur(act, U, v.reshape(V // 2, 2, 4, 3)), V // 2 * 24)
    assert np.max(np.abs(Mh - Mo)) < 1e-13
    assert np.all(np.diff(lex_odd // 2) == 1)  # odd half-index is lex >> 1


def test_gauge_covariance(oracle_lib):
    """D[U^g](g psi) = g D[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^+:
    pins the link direction and conjugation of both hops (Sec. 2, Eq. "Wilson")."""
    dims = (4, 2, 4, 2)
    T, X, Y, Z = dims
    U = synth.random_su3_field(dims, 0.6, 9)
    g = synth.random_gauge_transform(dims, 10)
    Ug = np.empty_like(U)
    for mu in range(4):
        gs = np.roll(g, -1, axis=mu)   # g(x + mu)
        Ug[mu] = np.einsum("...ij,...jk,...lk->...il", g, U[mu], np.conj(gs))
    act = oracle.action(dims, KAPPA, MU, EPS)
    V = T * X * Y * Z
    psi = _rand_vec((T, X, Y, Z, 2, 4, 3), 11)
    gpsi = np.einsum("txyzab,txyzfsb->txyzfsa", g, psi)
    lhs = oracle.dnd(act, Ug, gpsi.reshape(V, 2, 4, 3)).reshape(psi.shape)
    rhs = np.einsum("txyzab,txyzfsb->txyzfsa", g, oracle.dnd(act, U, psi.reshape(V, 2, 4, 3)).reshape(psi.shape))
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_flavour_structure(oracle_lib):
    """Eq. "non-degenerate": with eps = 0 the flavours decouple into D_TM(+mu) and
    D_TM(-mu); with mu = 0, w_pm = (v, +-v) is mapped to ((D_W -+ eps) v, +-(D_W -+ eps) v)
    (Sec. 3.2; with the -eps tau_1 sign of Eq. "non-degenerate")."""
    dims = (2, 2, 2, 4)
    V = 32
    U = synth.random_su3_field(dims, 0.5, 12)
    v = _rand_vec((V, 4, 3), 13)
    z = np.zeros_like(v)
    a_p = oracle.action(dims, KAPPA, MU, 0.0)
    a_m = oracle.action(dims, KAPPA, -MU, 0.0)
    up = oracle.dnd(a_p, U, np.stack([v, z], 1))
    dn = oracle.dnd(a_p, U, np.stack([z, v], 1))
    ref_m = oracle.dnd(a_m, U, np.stack([v, z], 1))
    assert np.max(np.abs(up[:, 1])) == 0 and np.max(np.abs(dn[:, 0])) == 0
    assert np.max(np.abs(dn[:, 1] - ref_m[:, 0])) < 1e-14
    a_w = oracle.action(dims, KAPPA, 0.0, 0.0)
    a_e = oracle.action(dims, KAPPA, 0.0, EPS)
    dw = oracle.dnd(a_w, U, np.stack([v, z], 1))[:, 0]
    e2 = 2 * KAPPA * EPS  # hopping form
    for s in (1, -1):
        w = oracle.dnd(a_e, U, np.stack([v, s * v], 1))
        assert np.max(np.abs(w[:, 0] - (dw - s * e2 * v))) < 1e-14
        assert np.max(np.abs(w[:, 1] - s * (dw - s * e2 * v))) < 1e-14
