"""Equivalent solutions of (Qhat^2 + mu^2) x = b (App. A: error and residual of
solutions that agree in exact arithmetic), on the GPU.

Host orchestration only: every arithmetic step runs in libtmnd (FP64 CG through
mms_cg_solve with one shift, Qhat through tm_nd_apply, complex combinations
through tmnd_lincomb_c, norms through tmnd_gram / tmnd_site_norm_range).

  A: x_A = CG[b]                                            (Eq. "direct")
  single systems (Qhat +- i mu) x = b, with (Qhat +- i mu)^-1 = (Qhat -+ i mu) (Qhat^2 + mu^2)^-1:
     E: x = CG[(Qhat -+ i mu) b], stopped at rho |(Qhat -+ i mu) b|
     F: x = (Qhat -+ i mu) CG[b]
     D: E, then one F step on its residual so that |b - (Qhat +- i mu) x| <= rho |b|
  B: x_B = (Qhat - i mu)^-1 x_+, both single systems by D    (Eq. "two-step")
  C: x_C = i/(2 mu) (x_+ - x_-), x_pm by D                  (Eq. "linear-combination")
"""
from __future__ import annotations

import numpy as np

import paper_1805_09584_gb300 as tm


def _norm(g, v) -> float:
    return float(np.sqrt(tm.tmnd_gram(g.handle, [v])[0, 0].real))


def _cg(g, b, s2, rho, maxiter=100000):
    x = g.spinor()
    tm.mms_cg_solve(g.handle, b, 1, [float(s2)], [x], rho=float(rho), maxiter=maxiter)
    return x


def qpm(g, x, mu, sg):
    """(Qhat + sg i mu) x."""
    t = g.spinor()
    tm.tm_nd_apply(g.handle, t, x, tm.OP_QHAT)
    tm.tmnd_lincomb_c(g.handle, [1.0, sg * 1j * mu], [t, x], t)
    return t


def solve_e(g, b, mu, sg, rho):
    """Method E for (Qhat + sg i mu) x = b: x = CG[(Qhat - sg i mu) b]."""
    return _cg(g, qpm(g, b, mu, -sg), float(mu) * float(mu), rho)


def solve_f(g, y, mu, sg):
    """Method F for (Qhat + sg i mu) x = b from y = CG[b]: x = (Qhat - sg i mu) y."""
    return qpm(g, y, mu, -sg)


def solve_d(g, b, mu, sg, rho, xe=None):
    """Method D for (Qhat + sg i mu) x = b: E (or the given E solution), then one F step
    on its residual r, x += (Qhat - sg i mu) CG[r] stopped at rho |b| / |r|."""
    if xe is None:
        xe = solve_e(g, b, mu, sg, rho)
    r = g.spinor()
    tm.tmnd_lincomb_c(g.handle, [1.0, -1.0], [b, qpm(g, xe, mu, sg)], r)
    bn, rn = _norm(g, b), _norm(g, r)
    xd = g.spinor()
    tm.tmnd_lincomb_c(g.handle, [1.0], [xe], xd)
    if rn > rho * bn:
        d = _cg(g, r, float(mu) * float(mu), min(0.5, rho * bn / rn))
        tm.tmnd_lincomb_c(g.handle, [1.0, 1.0], [xd, qpm(g, d, mu, -sg)], xd)
    return xd


def single_system_solves(g, b, mu, rho):
    """{("E"|"F"|"D", +1|-1): x} for (Qhat +- i mu) x = b (see the module docstring)."""
    y = _cg(g, b, float(mu) * float(mu), rho)
    out = {}
    for sg in (+1, -1):
        out[("E", sg)] = solve_e(g, b, mu, sg, rho)
        out[("F", sg)] = solve_f(g, y, mu, sg)
        out[("D", sg)] = solve_d(g, b, mu, sg, rho, out[("E", sg)])
    return out


def equivalent_solutions(g, b, mu, rho):
    """Methods A, B, C (device spinors "A", "B", "C"), x_+ and x_- ("p", "m"), and the single-
    system solutions of the + system by E, F, D ({("E"|"F"|"D", +1): x}); 7 CG solves."""
    s2 = float(mu) * float(mu)
    xa = _cg(g, b, s2, rho)
    xe = solve_e(g, b, mu, +1, rho)
    xp = solve_d(g, b, mu, +1, rho, xe)
    xm = solve_d(g, b, mu, -1, rho)
    xb = solve_d(g, xp, mu, -1, rho)
    xc = g.spinor()
    tm.tmnd_lincomb_c(g.handle, [1j / (2.0 * mu), -1j / (2.0 * mu)], [xp, xm], xc)
    one = {("E", +1): xe, ("F", +1): solve_f(g, xa, mu, +1), ("D", +1): xp}
    return {"A": xa, "B": xb, "C": xc, "p": xp, "m": xm}, one


def app_a_limits(rho, lmin, lmax, mu):
    """App. A's upper limits of |r| / |b| and |e| / |b| for methods A, B, C (squared
    operator) and D, E, F (single systems); lmin, lmax: extreme eigenvalues of Qhat^2."""
    m2 = float(mu) ** 2
    lo, hi = lmin + m2, lmax + m2
    return {"A": (rho, rho / lo), "B": ((1.0 + np.sqrt(hi / lo)) * rho, 2.0 * rho / lo),
            "C": (rho * np.sqrt(hi) / abs(mu), rho / (abs(mu) * np.sqrt(lo))),
            "D": (rho, rho / np.sqrt(lo)), "E": (rho * np.sqrt(hi / lo), rho * np.sqrt(hi) / lo),
            "F": (rho, rho / np.sqrt(lo))}


def residual_and_error(g, b, x_exact, x, mu, sg=None):
    """|b - A x| / |b|, |x_exact - x| / |b| (App. A's normalisation of the limits) and the
    smallest / largest site norm of the error relative to the largest site norm of b;
    A = Qhat^2 + mu^2, or Qhat + sg i mu."""
    Ax = g.spinor()
    if sg is None:
        tm.tm_nd_apply(g.handle, Ax, x, tm.OP_QHAT2, float(mu) * float(mu))
    else:
        Ax = qpm(g, x, mu, sg)
    r, e = g.spinor(), g.spinor()
    tm.tmnd_lincomb_c(g.handle, [1.0, -1.0], [b, Ax], r)
    tm.tmnd_lincomb_c(g.handle, [1.0, -1.0], [x_exact, x], e)
    lo, hi = tm.tmnd_site_norm_range(g.handle, e)
    bn, bmax = _norm(g, b), tm.tmnd_site_norm_range(g.handle, b)[1]
    return {"res": _norm(g, r) / bn, "err": _norm(g, e) / bn, "err_site_min": lo / bmax, "err_site_max": hi / bmax}
