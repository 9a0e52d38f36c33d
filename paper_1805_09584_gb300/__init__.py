"""GB300 (sm_103a) kernels for the shifted systems of the non-degenerate
twisted-mass operator (arXiv:1805.09584): the even-odd Schur stencil, the
multi-mass-shift CG and Lagrange-interpolated guesses.

This module is the thin Python binding of `libtmnd.so` (C ABI in
`include/tmnd.h`): argument marshalling only, every step runs in the CUDA
library.  PyTorch tensors (or raw integer device addresses) provide device
memory; streams are passed as `cudaStream_t` handles.  There is no CPU
fallback: if the library is missing the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtmnd.so")
MAX_SHIFTS = 32

TMND_F64, TMND_F32, TMND_S16 = 0, 1, 2
OP_MHAT, OP_MHAT_DAG, OP_QHAT2, OP_QHAT = 0, 1, 2, 3
OP_S16 = 16  # flag: sloppy operator on TMND_S16 spinors
OP_F32 = 32  # flag: FP32 operator on TMND_F32 spinors

STATUS = {0: "TMND_OK", 1: "TMND_ERR_ARG", 2: "TMND_ERR_CUDA", 3: "TMND_ERR_OOM", 4: "TMND_ERR_NOCONV",
          5: "TMND_ERR_NAN", 6: "TMND_ERR_TIMEOUT", 7: "TMND_ERR_NOTSU3"}

# every entry point declared in include/tmnd.h
EXPORTS = ("tmnd_gauge_create", "tmnd_gauge_destroy", "tmnd_spinor_bytes", "tmnd_spinor_bytes_prec",
           "tmnd_spinor_convert", "tmnd_spinor_pack",
           "tmnd_spinor_unpack", "tm_nd_apply", "tm_nd_apply_noalloc", "mms_cg_solve", "lagrange_guess",
           "tmnd_last_error", "tmnd_mg_create", "tmnd_mg_destroy", "tmnd_mg_coarse_bytes", "tmnd_mg_restrict",
           "tmnd_mg_prolong", "mg_coarse_apply", "tmnd_mg_export", "tmnd_dnd_full_apply", "tmnd_mg_solve",
           "tmnd_mg_smooth_vectors", "tmnd_hybrid_solve", "tmnd_mlp_num_params", "tmnd_mlp_create",
           "tmnd_mlp_destroy", "tmnd_mlp_params", "tmnd_mlp_fit_inputs", "tmnd_mlp_loss_grad", "tmnd_mlp_train_step", "tmnd_mlp_predict",
           "tmnd_mlp_features", "tmnd_gram", "tmnd_lincomb", "tmnd_zolotarev", "tmnd_rational_apply",
           "tmnd_hybrid_cost", "tmnd_fit_cg_time", "tmnd_fit_mg_time", "tmnd_lincomb_c", "tmnd_site_norm_range",
           "tmnd_lagrange_weights", "tmnd_lagrange_degree", "tmnd_guess_quadratic_form", "tmnd_mg_status",
           "tmnd_autotune", "tmnd_autotune_mms", "tmnd_s16_force_shape", "tmnd_s16_shape_info",
           "tmnd_mg_bootstrap")
S16_SHAPES = 16
TMND_MAX_BATCH = 16
NOALLOC_MAX_VH = 32768


class TmndError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Action(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("kappa", ctypes.c_double), ("mu_bar", ctypes.c_double),
                ("eps_bar", ctypes.c_double), ("antiperiodic_t", ctypes.c_int)]


class MGParams(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int * 4), ("nvec", ctypes.c_int), ("coarse_mu_factor", ctypes.c_double),
                ("coarse_simt", ctypes.c_int), ("wait_limit_s", ctypes.c_double), ("stall_test", ctypes.c_int),
                ("smoother", ctypes.c_int), ("sap_mr", ctypes.c_int)]


class HybridParams(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("maxiter", ctypes.c_int), ("prec", ctypes.c_int),
                ("rho_inner", ctypes.c_double), ("n_guess", ctypes.c_int), ("guess", ctypes.c_int),
                ("mg_tol", ctypes.c_double), ("mg_maxiter", ctypes.c_int), ("mg_restart", ctypes.c_int),
                ("mg_nu", ctypes.c_int), ("net", ctypes.c_void_p), ("lebesgue_max", ctypes.c_double)]


class HybridInfo(ctypes.Structure):
    _fields_ = [("mms_iters", ctypes.c_int), ("guess_res", ctypes.c_double * MAX_SHIFTS),
                ("mg_iters", ctypes.c_int * MAX_SHIFTS), ("true_res", ctypes.c_double * MAX_SHIFTS),
                ("fp64_applies", ctypes.c_int), ("refine_iters", ctypes.c_int),
                ("shift_ms", ctypes.c_double * MAX_SHIFTS), ("mms_ms", ctypes.c_double),
                ("lag_nodes", ctypes.c_int * MAX_SHIFTS), ("lebesgue", ctypes.c_double * MAX_SHIFTS),
                ("launches", ctypes.c_longlong), ("f32_applies", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("maxiter", ctypes.c_int), ("nsolve", ctypes.c_int),
                ("check_every", ctypes.c_int), ("profile", ctypes.c_int), ("prec", ctypes.c_int),
                ("rho_inner", ctypes.c_double), ("ab_hist", ctypes.POINTER(ctypes.c_double)),
                ("ab_hist_len", ctypes.c_int), ("batch", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("conv_iter", ctypes.c_int * MAX_SHIFTS),
                ("true_res", ctypes.c_double * MAX_SHIFTS), ("zeta", ctypes.c_double * MAX_SHIFTS),
                ("hop_ms", ctypes.c_double), ("update_ms", ctypes.c_double), ("launches", ctypes.c_longlong),
                ("refine_rounds", ctypes.c_int), ("refine_iters", ctypes.c_int), ("fp64_applies", ctypes.c_int),
                ("f32_applies", ctypes.c_int), ("mms_ms", ctypes.c_double), ("fp64_ms", ctypes.c_double),
                ("refine_ms", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libtmnd.so (built in-tree by `__graft_entry__.build()`); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.tmnd_gauge_create.argtypes = [vp, ctypes.POINTER(Action), i, ctypes.POINTER(vp)]
        L.tmnd_gauge_destroy.argtypes = [vp]
        L.tmnd_gauge_destroy.restype = None
        L.tmnd_spinor_bytes.argtypes = [vp]
        L.tmnd_spinor_bytes.restype = ctypes.c_size_t
        L.tmnd_spinor_bytes_prec.argtypes = [vp, i]
        L.tmnd_spinor_bytes_prec.restype = ctypes.c_size_t
        L.tmnd_spinor_convert.argtypes = [vp, vp, i, vp, i, i, vp]
        L.tmnd_spinor_convert.restype = ctypes.c_int
        L.tmnd_spinor_pack.argtypes = [vp, vp, vp, i, vp]
        L.tmnd_spinor_unpack.argtypes = [vp, vp, vp, i, vp]
        L.tm_nd_apply.argtypes = [vp, vp, vp, i, d, i, vp]
        L.tm_nd_apply_noalloc.argtypes = [vp, vp, vp, i, d, i, vp]
        L.mms_cg_solve.argtypes = [vp, vp, i, ctypes.POINTER(d), i, ctypes.POINTER(vp),
                                   ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), vp]
        L.lagrange_guess.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(vp), i, d, vp, i,
                                     ctypes.POINTER(d), vp]
        L.tmnd_last_error.argtypes = []
        L.tmnd_last_error.restype = ctypes.c_char_p
        L.tmnd_mg_create.argtypes = [vp, ctypes.POINTER(MGParams), vp, ctypes.POINTER(vp)]
        L.tmnd_mg_destroy.argtypes = [vp]
        L.tmnd_mg_destroy.restype = None
        L.tmnd_mg_coarse_bytes.argtypes = [vp]
        L.tmnd_mg_coarse_bytes.restype = ctypes.c_size_t
        L.tmnd_mg_restrict.argtypes = [vp, vp, vp, i, vp]
        L.tmnd_mg_prolong.argtypes = [vp, vp, vp, i, vp]
        L.mg_coarse_apply.argtypes = [vp, vp, vp, i, d, vp]
        L.tmnd_mg_export.argtypes = [vp, vp, vp, vp]
        L.tmnd_mg_status.argtypes = [vp]
        L.tmnd_mg_bootstrap.argtypes = [vp, ctypes.POINTER(MGParams), vp, i, ctypes.POINTER(vp), vp]
        L.tmnd_dnd_full_apply.argtypes = [vp, vp, vp, d, vp]
        L.tmnd_mg_solve.argtypes = [vp, vp, vp, d, d, i, i, i, ctypes.POINTER(i), ctypes.POINTER(d), vp]
        L.tmnd_mg_smooth_vectors.argtypes = [vp, vp, i, i, vp]
        L.tmnd_hybrid_solve.argtypes = [vp, vp, vp, i, ctypes.POINTER(d), i, i, ctypes.POINTER(vp),
                                        ctypes.POINTER(HybridParams), ctypes.POINTER(HybridInfo), vp]
        fp = ctypes.POINTER(ctypes.c_float)
        L.tmnd_mlp_num_params.argtypes = [i]
        L.tmnd_mlp_num_params.restype = ctypes.c_int
        L.tmnd_mlp_create.argtypes = [i, ctypes.c_ulonglong, ctypes.POINTER(vp)]
        L.tmnd_mlp_destroy.argtypes = [vp]
        L.tmnd_mlp_destroy.restype = None
        L.tmnd_mlp_params.argtypes = [vp, vp, vp]
        L.tmnd_mlp_fit_inputs.argtypes = [vp, vp, i, vp]
        L.tmnd_mlp_loss_grad.argtypes = [vp, vp, vp, vp, i, d, ctypes.POINTER(d), vp, vp]
        L.tmnd_mlp_train_step.argtypes = [vp, vp, vp, vp, i, d, d, ctypes.POINTER(d), vp]
        L.tmnd_mlp_predict.argtypes = [vp, vp, vp, i, vp, vp]
        L.tmnd_mlp_features.argtypes = [ctypes.POINTER(d), d, vp, i, d, fp]
        L.tmnd_gram.argtypes = [vp, ctypes.POINTER(vp), i, ctypes.POINTER(d), vp]
        L.tmnd_lincomb.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(vp), i, vp, i, vp]
        L.tmnd_lincomb_c.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(vp), i, vp, i, vp]
        L.tmnd_site_norm_range.argtypes = [vp, vp, i, ctypes.POINTER(d), vp]
        pd = ctypes.POINTER(d)
        L.tmnd_zolotarev.argtypes = [i, d, pd, pd, pd, pd]
        L.tmnd_hybrid_cost.argtypes = [pd, i, pd, pd, pd, ctypes.POINTER(i)]
        L.tmnd_fit_cg_time.argtypes = [pd, pd, i, d, d, pd, pd]
        L.tmnd_fit_mg_time.argtypes = [pd, pd, i, d, i, pd, pd, pd]
        L.tmnd_rational_apply.argtypes = [vp, vp, i, i, d, d, ctypes.POINTER(SolveParams), vp, pd,
                                          ctypes.POINTER(SolveInfo), vp]
        L.tmnd_lagrange_weights.argtypes = [pd, i, d, pd, pd]
        L.tmnd_autotune.argtypes = [vp, i, ctypes.POINTER(i), pd, vp]
        L.tmnd_autotune_mms.argtypes = [vp, i, ctypes.POINTER(i), pd, vp]
        L.tmnd_s16_force_shape.argtypes = [i]
        L.tmnd_s16_shape_info.argtypes = [i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                          ctypes.POINTER(i)]
        L.tmnd_lagrange_degree.argtypes = [pd, i, d, d, ctypes.POINTER(i), pd]
        L.tmnd_guess_quadratic_form.argtypes = [pd, pd, i, d, d, pd]
        for name in ("tmnd_mlp_create", "tmnd_mlp_params", "tmnd_mlp_fit_inputs", "tmnd_mlp_loss_grad",
                     "tmnd_mlp_train_step", "tmnd_zolotarev", "tmnd_rational_apply", "tmnd_hybrid_cost",
                     "tmnd_fit_cg_time", "tmnd_fit_mg_time",
                     "tmnd_mlp_predict", "tmnd_mlp_features", "tmnd_gram", "tmnd_lincomb", "tmnd_lincomb_c",
                     "tmnd_site_norm_range", "tmnd_lagrange_weights", "tmnd_lagrange_degree",
                     "tmnd_guess_quadratic_form", "tmnd_autotune", "tmnd_autotune_mms", "tmnd_s16_force_shape",
                     "tmnd_s16_shape_info"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("tmnd_mg_create", "tmnd_mg_restrict", "tmnd_mg_prolong", "mg_coarse_apply", "tmnd_mg_export",
                     "tmnd_mg_status", "tmnd_mg_bootstrap",
                     "tmnd_dnd_full_apply", "tmnd_mg_solve", "tmnd_mg_smooth_vectors", "tmnd_hybrid_solve"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("tmnd_gauge_create", "tmnd_spinor_pack", "tmnd_spinor_unpack", "tm_nd_apply",
                     "tm_nd_apply_noalloc", "mms_cg_solve", "lagrange_guess"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise TmndError(status, lib().tmnd_last_error().decode(errors="replace"))


def _ptr(t) -> int:
    """Device address of a tensor (anything with data_ptr()) or a raw integer."""
    if t is None:
        return 0
    return int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_action(dims, kappa, mu_bar, eps_bar, antiperiodic_t=True) -> Action:
    a = Action()
    for k in range(4):
        a.dims[k] = int(dims[k])
    a.kappa, a.mu_bar, a.eps_bar = float(kappa), float(mu_bar), float(eps_bar)
    a.antiperiodic_t = int(bool(antiperiodic_t))
    return a


# ------------------------------------------------------------ C-ABI mirror
def tmnd_gauge_create(host_links: np.ndarray, act: Action, prec: int = TMND_F64) -> ctypes.c_void_p:
    links = np.ascontiguousarray(host_links, dtype=np.complex128)
    h = ctypes.c_void_p()
    _check(lib().tmnd_gauge_create(links.ctypes.data, ctypes.byref(act), int(prec), ctypes.byref(h)))
    return h


def tmnd_gauge_destroy(h) -> None:
    lib().tmnd_gauge_destroy(h)


def tmnd_spinor_bytes(h) -> int:
    return int(lib().tmnd_spinor_bytes(h))


def tmnd_spinor_bytes_prec(h, prec: int) -> int:
    return int(lib().tmnd_spinor_bytes_prec(h, int(prec)))


def tmnd_spinor_convert(h, dst, dst_prec: int, src, src_prec: int, nrhs: int = 1, stream=None) -> None:
    _check(lib().tmnd_spinor_convert(h, _ptr(dst), int(dst_prec), _ptr(src), int(src_prec), int(nrhs),
                                     _stream(stream)))


def tmnd_spinor_pack(h, dev_internal, dev_canonical, nrhs: int = 1, stream=None) -> None:
    _check(lib().tmnd_spinor_pack(h, _ptr(dev_internal), _ptr(dev_canonical), int(nrhs), _stream(stream)))


def tmnd_spinor_unpack(h, dev_canonical, dev_internal, nrhs: int = 1, stream=None) -> None:
    _check(lib().tmnd_spinor_unpack(h, _ptr(dev_canonical), _ptr(dev_internal), int(nrhs), _stream(stream)))


def tm_nd_apply(h, out, inp, op: int, sigma: float = 0.0, nrhs: int = 1, stream=None) -> None:
    _check(lib().tm_nd_apply(h, _ptr(out), _ptr(inp), int(op), float(sigma), int(nrhs), _stream(stream)))


def tm_nd_apply_noalloc(h, out, inp, op: int, sigma: float = 0.0, nrhs: int = 1, stream=None) -> None:
    """tm_nd_apply with its temporaries in the library's fixed device array: never
    allocates (for callers whose device memory is owned by another allocator or
    that cannot take cudaMalloc's synchronisation); V/2 <= NOALLOC_MAX_VH."""
    _check(lib().tm_nd_apply_noalloc(h, _ptr(out), _ptr(inp), int(op), float(sigma), int(nrhs), _stream(stream)))


def mms_cg_solve(h, b, nrhs: int, sigma, x, rho: float = 1e-10, maxiter: int = 100000, nsolve: int = 0,
                 check_every: int = 0, profile: bool = False, prec: int = TMND_F64, rho_inner: float = 0.0,
                 ab_hist=None, batch: int = 0, stream=None) -> dict:
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    ns = len(sig)
    xs = (ctypes.c_void_p * ns)(*[_ptr(v) for v in x])
    p = SolveParams(float(rho), int(maxiter), int(nsolve), int(check_every), int(bool(profile)), int(prec),
                    float(rho_inner))
    if ab_hist is not None:
        assert ab_hist.dtype == np.float64 and ab_hist.flags["C_CONTIGUOUS"]
        p.ab_hist = ab_hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.ab_hist_len = int(ab_hist.size)
    p.batch = int(batch)
    info = SolveInfo()
    st = lib().mms_cg_solve(h, _ptr(b), int(nrhs), sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ns, xs,
                            ctypes.byref(p), ctypes.byref(info), _stream(stream))
    out = {"status": st, "iters": info.iters, "conv_iter": list(info.conv_iter[:ns]),
           "true_res": list(info.true_res[:ns]), "zeta": list(info.zeta[:ns]),
           "hop_ms": info.hop_ms, "update_ms": info.update_ms, "launches": info.launches,
           "refine_rounds": info.refine_rounds, "refine_iters": info.refine_iters,
           "fp64_applies": info.fp64_applies, "f32_applies": info.f32_applies,
           "phase_ms": {"multi_shift": info.mms_ms, "fp64_defects": info.fp64_ms, "refinement": info.refine_ms}}
    _check(st)
    return out


def lagrange_guess(h, nodes, xs, target: float, out, nrhs: int = 1, stream=None) -> float:
    nd = np.ascontiguousarray(nodes, dtype=np.float64)
    k = len(nd)
    arr = (ctypes.c_void_p * k)(*[_ptr(v) for v in xs])
    leb = ctypes.c_double()
    _check(lib().lagrange_guess(h, nd.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), arr, k, float(target),
                                _ptr(out), int(nrhs), ctypes.byref(leb), _stream(stream)))
    return leb.value


def mg_params(block, nvec: int, coarse_mu_factor: float = 1.0, coarse_simt: bool = False, wait_limit_s: float = 0.0,
              stall_test: int = 0, smoother: int = 0, sap_mr: int = 0) -> MGParams:
    p = MGParams()
    for k in range(4):
        p.block[k] = int(block[k])
    p.nvec, p.coarse_mu_factor, p.coarse_simt = int(nvec), float(coarse_mu_factor), int(bool(coarse_simt))
    p.wait_limit_s, p.stall_test = float(wait_limit_s), int(stall_test)
    p.smoother, p.sap_mr = int(smoother), int(sap_mr)
    return p


def tmnd_mg_bootstrap(mg, test_vectors, iters: int, block, nvec: int, stream=None, **kw):
    """A new hierarchy from the test vectors improved by `iters` outer iterations of mg's
    two-level method (the vectors are updated in place); the caller destroys both handles."""
    p = mg_params(block, nvec, **kw)
    out = ctypes.c_void_p()
    _check(lib().tmnd_mg_bootstrap(mg, ctypes.byref(p), _ptr(test_vectors), int(iters), ctypes.byref(out),
                                   _stream(stream)))
    return out


def tmnd_mg_create(h, block, nvec: int, test_vectors, coarse_mu_factor: float = 1.0, coarse_simt: bool = False,
                   wait_limit_s: float = 0.0, stall_test: int = 0, smoother: int = 0, sap_mr: int = 0):
    p = MGParams()
    for k in range(4):
        p.block[k] = int(block[k])
    p.nvec, p.coarse_mu_factor, p.coarse_simt = int(nvec), float(coarse_mu_factor), int(bool(coarse_simt))
    p.wait_limit_s, p.stall_test = float(wait_limit_s), int(stall_test)
    p.smoother, p.sap_mr = int(smoother), int(sap_mr)
    out = ctypes.c_void_p()
    _check(lib().tmnd_mg_create(h, ctypes.byref(p), _ptr(test_vectors), ctypes.byref(out)))
    return out


def tmnd_mg_destroy(mg) -> None:
    lib().tmnd_mg_destroy(mg)


def tmnd_mg_coarse_bytes(mg) -> int:
    return int(lib().tmnd_mg_coarse_bytes(mg))


def tmnd_mg_restrict(mg, out_c, in_fine, nrhs: int = 1, stream=None) -> None:
    _check(lib().tmnd_mg_restrict(mg, _ptr(out_c), _ptr(in_fine), int(nrhs), _stream(stream)))


def tmnd_mg_prolong(mg, out_fine, in_c, nrhs: int = 1, stream=None) -> None:
    _check(lib().tmnd_mg_prolong(mg, _ptr(out_fine), _ptr(in_c), int(nrhs), _stream(stream)))


def mg_coarse_apply(mg, out_c, in_c, nrhs: int = 1, odd_shift_s: float = 0.0, stream=None) -> None:
    _check(lib().mg_coarse_apply(mg, _ptr(out_c), _ptr(in_c), int(nrhs), float(odd_shift_s), _stream(stream)))


def tmnd_mg_status(mg) -> None:
    """Raise TmndError(TMND_ERR_TIMEOUT) if a tensor-core apply gave up a wait since the last check."""
    _check(lib().tmnd_mg_status(mg))


def tmnd_mg_export(mg, P_host=None, Dc_host=None, Godd_host=None) -> None:
    _check(lib().tmnd_mg_export(mg, _hp(P_host), _hp(Dc_host), _hp(Godd_host)))


def tmnd_dnd_full_apply(h, out, inp, s: float = 0.0, stream=None) -> None:
    _check(lib().tmnd_dnd_full_apply(h, _ptr(out), _ptr(inp), float(s), _stream(stream)))


def tmnd_mg_solve(mg, x, b, s: float = 0.0, tol: float = 1e-6, maxiter: int = 200, restart: int = 24, nu: int = 4,
                  stream=None) -> dict:
    it = ctypes.c_int()
    res = ctypes.c_double()
    _check(lib().tmnd_mg_solve(mg, _ptr(x), _ptr(b), float(s), float(tol), int(maxiter), int(restart), int(nu),
                               ctypes.byref(it), ctypes.byref(res), _stream(stream)))
    return {"iters": it.value, "res": res.value}


def tmnd_mg_smooth_vectors(h, vecs, nvec: int, iters: int, stream=None) -> None:
    _check(lib().tmnd_mg_smooth_vectors(h, _ptr(vecs), int(nvec), int(iters), _stream(stream)))


def tmnd_hybrid_solve(h, mg, b, nrhs: int, sigma, n_mms: int, x, rho: float = 1e-10, maxiter: int = 100000,
                      prec: int = TMND_F64, rho_inner: float = 0.0, n_guess: int = 2, guess: int = 1,
                      mg_tol: float = 0.0, mg_maxiter: int = 0, mg_restart: int = 0, mg_nu: int = 0,
                      net=None, lebesgue_max: float = 0.0, stream=None) -> dict:
    """mg may be None (no multigrid: guesses go straight to the FP64 defect correction);
    guess = 2 with a trained network `net` (tmnd_mlp_create) uses learned weights."""
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    ns = len(sig)
    xs = (ctypes.c_void_p * ns)(*[_ptr(v) for v in x])
    p = HybridParams(float(rho), int(maxiter), int(prec), float(rho_inner), int(n_guess), int(guess), float(mg_tol),
                     int(mg_maxiter), int(mg_restart), int(mg_nu), net, float(lebesgue_max))
    info = HybridInfo()
    st = lib().tmnd_hybrid_solve(h, mg, _ptr(b), int(nrhs), sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ns,
                                 int(n_mms), xs, ctypes.byref(p), ctypes.byref(info), _stream(stream))
    out = {"status": st, "mms_iters": info.mms_iters, "guess_res": list(info.guess_res[:ns]),
           "mg_iters": list(info.mg_iters[:ns]), "true_res": list(info.true_res[:ns]),
           "fp64_applies": info.fp64_applies, "refine_iters": info.refine_iters,
           "shift_ms": list(info.shift_ms[:ns]), "mms_ms": info.mms_ms,
           "lag_nodes": list(info.lag_nodes[:ns]), "lebesgue": list(info.lebesgue[:ns]),
           "launches": info.launches, "f32_applies": info.f32_applies}
    _check(st)
    return out


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def tmnd_autotune(h, nrhs: int, stream=None):
    """(chosen shape, per-shape ms) of the 16-bit stencil's Qhat^2 + sigma application for
    this lattice and nrhs per launch."""
    sh = ctypes.c_int()
    ms = np.zeros(S16_SHAPES)
    _check(lib().tmnd_autotune(h, int(nrhs), ctypes.byref(sh), _pd(ms), _stream(stream)))
    return sh.value, ms


def tmnd_autotune_mms(h, nrhs: int, stream=None):
    """(chosen shape, per-shape ms) of the 16-bit stencil's sloppy multi-shift iteration (the
    4 launches, the last with the residual-update epilogue) for this lattice and nrhs."""
    sh = ctypes.c_int()
    ms = np.zeros(S16_SHAPES)
    _check(lib().tmnd_autotune_mms(h, int(nrhs), ctypes.byref(sh), _pd(ms), _stream(stream)))
    return sh.value, ms


def tmnd_s16_force_shape(shape: int) -> None:
    _check(lib().tmnd_s16_force_shape(int(shape)))


def tmnd_s16_shape_info(shape: int):
    """(threads per block, resident blocks per SM, prefetch, loop order 0..3) of a launch variant."""
    t, b, p, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().tmnd_s16_shape_info(int(shape), ctypes.byref(t), ctypes.byref(b), ctypes.byref(p), ctypes.byref(o)))
    return t.value, b.value, bool(p.value), o.value


def tmnd_lagrange_weights(nodes, target: float):
    """(w, gamma): Lagrange weights over `nodes` at `target` and their Lebesgue function."""
    nd = np.ascontiguousarray(nodes, np.float64)
    w = np.zeros(len(nd))
    gam = ctypes.c_double()
    _check(lib().tmnd_lagrange_weights(_pd(nd), len(nd), float(target), _pd(w), ctypes.byref(gam)))
    return w, gam.value


def tmnd_lagrange_degree(nodes, target: float, gamma_max: float):
    """(k_used, gamma): the longest prefix of `nodes` (nearest first) with gamma <= gamma_max."""
    nd = np.ascontiguousarray(nodes, np.float64)
    ku = ctypes.c_int()
    gam = ctypes.c_double()
    _check(lib().tmnd_lagrange_degree(_pd(nd), len(nd), float(target), float(gamma_max), ctypes.byref(ku),
                                      ctypes.byref(gam)))
    return ku.value, gam.value


def tmnd_guess_quadratic_form(G, nodes, target: float, bb: float) -> np.ndarray:
    """H [k, k] = Re((t - s_j) G_jq (t - s_q)) / bb for a complex Gram matrix G [k, k]."""
    nd = np.ascontiguousarray(nodes, np.float64)
    k = len(nd)
    Gi = np.empty(2 * k * k)
    Gc = np.asarray(G, np.complex128).ravel()
    Gi[0::2], Gi[1::2] = Gc.real, Gc.imag
    H = np.zeros(k * k)
    _check(lib().tmnd_guess_quadratic_form(_pd(Gi), _pd(nd), k, float(target), float(bb), _pd(H)))
    return H.reshape(k, k)


def tmnd_mlp_num_params(F: int) -> int:
    return int(lib().tmnd_mlp_num_params(int(F)))


def tmnd_mlp_create(F: int = 20, seed: int = 0):
    out = ctypes.c_void_p()
    _check(lib().tmnd_mlp_create(int(F), ctypes.c_ulonglong(int(seed)), ctypes.byref(out)))
    return out


def tmnd_mlp_destroy(m) -> None:
    lib().tmnd_mlp_destroy(m)


def tmnd_mlp_params(m, get: np.ndarray = None, set_: np.ndarray = None) -> None:
    for a in (get, set_):
        if a is not None:
            assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    _check(lib().tmnd_mlp_params(m, None if get is None else get.ctypes.data,
                                 None if set_ is None else set_.ctypes.data))


def tmnd_mlp_fit_inputs(m, X, N: int, stream=None) -> None:
    _check(lib().tmnd_mlp_fit_inputs(m, _ptr(X), int(N), _stream(stream)))


def tmnd_mlp_loss_grad(m, X, S, H, N: int, floor: float = 0.0, grad: np.ndarray = None, stream=None) -> float:
    loss = ctypes.c_double()
    if grad is not None:
        assert grad.dtype == np.float32 and grad.flags["C_CONTIGUOUS"]
    _check(lib().tmnd_mlp_loss_grad(m, _ptr(X), _ptr(S), _ptr(H), int(N), float(floor), ctypes.byref(loss),
                                    None if grad is None else grad.ctypes.data, _stream(stream)))
    return loss.value


def tmnd_mlp_train_step(m, X, S, H, N: int, lr: float, floor: float = 0.0, stream=None) -> float:
    loss = ctypes.c_double()
    _check(lib().tmnd_mlp_train_step(m, _ptr(X), _ptr(S), _ptr(H), int(N), float(lr), float(floor),
                                     ctypes.byref(loss), _stream(stream)))
    return loss.value


def tmnd_mlp_predict(m, X, S, N: int, W, stream=None) -> None:
    _check(lib().tmnd_mlp_predict(m, _ptr(X), _ptr(S), int(N), _ptr(W), _stream(stream)))


def tmnd_mlp_features(nodes, target: float, ab_hist, niter: int, sigma0: float) -> np.ndarray:
    nd = np.ascontiguousarray(nodes, np.float64)
    out = np.zeros(20, np.float32)
    hist = None if ab_hist is None else np.ascontiguousarray(ab_hist, np.float64)
    _check(lib().tmnd_mlp_features(nd.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(target),
                                   None if hist is None else hist.ctypes.data, int(niter), float(sigma0),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def tmnd_gram(h, xs, stream=None) -> np.ndarray:
    k = len(xs)
    arr = (ctypes.c_void_p * k)(*[_ptr(v) for v in xs])
    G = np.zeros(2 * k * k, np.float64)
    _check(lib().tmnd_gram(h, arr, k, G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)))
    return (G[0::2] + 1j * G[1::2]).reshape(k, k)


def tmnd_lincomb(h, w, xs, out, nrhs: int = 1, stream=None) -> None:
    ww = np.ascontiguousarray(w, np.float64)
    k = len(xs)
    arr = (ctypes.c_void_p * k)(*[_ptr(v) for v in xs])
    _check(lib().tmnd_lincomb(h, ww.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), arr, k, _ptr(out), int(nrhs),
                              _stream(stream)))


def tmnd_lincomb_c(h, w, xs, out, nrhs: int = 1, stream=None) -> None:
    """out = sum_j w_j xs[j] with complex weights w (App. A combinations)."""
    w = np.asarray(w, np.complex128)
    ww = np.ascontiguousarray(np.stack([w.real, w.imag], axis=1).ravel(), np.float64)
    k = len(xs)
    arr = (ctypes.c_void_p * k)(*[_ptr(v) for v in xs])
    _check(lib().tmnd_lincomb_c(h, ww.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), arr, k, _ptr(out),
                                int(nrhs), _stream(stream)))


def tmnd_site_norm_range(h, x, nrhs: int = 1, stream=None):
    """(smallest, largest) site norm of internal FP64 spinors x (App. A local deviations)."""
    mm = np.zeros(2, np.float64)
    _check(lib().tmnd_site_norm_range(h, _ptr(x), int(nrhs), mm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      _stream(stream)))
    return float(mm[0]), float(mm[1])


def _hp(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------ conveniences
class Gauge:
    """Owns a tmnd_gauge handle (created from canonical host links)."""

    def __init__(self, host_links, dims, kappa, mu_bar, eps_bar, antiperiodic_t=True, prec=TMND_F64):
        self.dims = tuple(int(d) for d in dims)
        self.vh = int(np.prod(self.dims)) // 2
        self.act = make_action(dims, kappa, mu_bar, eps_bar, antiperiodic_t)
        self.handle = tmnd_gauge_create(host_links, self.act, prec)

    def close(self):
        if self.handle is not None and self.handle.value:
            tmnd_gauge_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spinor(self, nrhs: int = 1, device="cuda", prec: int = TMND_F64):
        """A new internal-layout spinor buffer: complex128 (TMND_F64), complex64
        (TMND_F32) or raw 16-byte words (TMND_S16), nrhs right-hand sides."""
        import torch
        if prec == TMND_F64:
            return torch.empty(nrhs * 24 * self.vh, dtype=torch.complex128, device=device)
        if prec == TMND_F32:
            return torch.empty(nrhs * 24 * self.vh, dtype=torch.complex64, device=device)
        nbytes = tmnd_spinor_bytes_prec(self.handle, prec) * nrhs
        return torch.empty(nbytes // 4, dtype=torch.int32, device=device)

    def convert(self, src, src_prec: int, dst_prec: int, nrhs: int = 1, stream=None):
        out = self.spinor(nrhs, src.device, dst_prec)
        tmnd_spinor_convert(self.handle, out, dst_prec, src, src_prec, nrhs, stream)
        return out

    def pack(self, canonical, nrhs: int = 1, stream=None):
        out = self.spinor(nrhs, canonical.device)
        tmnd_spinor_pack(self.handle, out, canonical, nrhs, stream)
        return out

    def unpack(self, internal, nrhs: int = 1, stream=None):
        import torch
        out = torch.empty((nrhs, self.vh, 2, 4, 3), dtype=torch.complex128, device=internal.device)
        tmnd_spinor_unpack(self.handle, out, internal, nrhs, stream)
        return out


def tmnd_zolotarev(n: int, eps: float):
    """(a, c[2n], q[n], delta) of Zolotarev's approximation of 1/sqrt(y) on (eps, 1)."""
    a, delta = ctypes.c_double(), ctypes.c_double()
    c = np.zeros(2 * n)
    q = np.zeros(n)
    pd = ctypes.POINTER(ctypes.c_double)
    _check(lib().tmnd_zolotarev(int(n), float(eps), ctypes.byref(a), c.ctypes.data_as(pd), q.ctypes.data_as(pd),
                                ctypes.byref(delta)))
    return a.value, c, q, delta.value


def tmnd_rational_apply(h, b, nrhs: int, n: int, lambda_min: float, lambda_max: float, out, rho: float = 1e-10,
                        prec: int = TMND_F64, maxiter: int = 100000, stream=None) -> dict:
    """out = R(Qhat^2/lambda_max) b / sqrt(lambda_max) ~ (Qhat^2)^(-1/2) b."""
    p = SolveParams(float(rho), int(maxiter), 0, 0, 0, int(prec), 0.0)
    info = SolveInfo()
    delta = ctypes.c_double()
    _check(lib().tmnd_rational_apply(h, _ptr(b), int(nrhs), int(n), float(lambda_min), float(lambda_max),
                                     ctypes.byref(p), _ptr(out), ctypes.byref(delta), ctypes.byref(info),
                                     _stream(stream)))
    return {"delta": delta.value, "iters": info.iters, "true_res": list(info.true_res[:n])}


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def tmnd_hybrid_cost(sigma, cg, mg):
    """(c_HY(n) for n = 1..N, n_opt); cg = (a, b, lmin, lmax), mg = (A, B, C, L)."""
    s = np.ascontiguousarray(sigma, np.float64)
    c1 = np.ascontiguousarray(cg, np.float64)
    m1 = np.ascontiguousarray(mg, np.float64)
    cost = np.zeros(len(s))
    n = ctypes.c_int()
    _check(lib().tmnd_hybrid_cost(_pd(s), len(s), _pd(c1), _pd(m1), _pd(cost), ctypes.byref(n)))
    return cost, n.value


def tmnd_fit_cg_time(sigma, t, lmin: float, lmax: float):
    s = np.ascontiguousarray(sigma, np.float64)
    tt = np.ascontiguousarray(t, np.float64)
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().tmnd_fit_cg_time(_pd(s), _pd(tt), len(s), float(lmin), float(lmax), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def tmnd_fit_mg_time(sigma, t, L: float, grid: int = 2001):
    s = np.ascontiguousarray(sigma, np.float64)
    tt = np.ascontiguousarray(t, np.float64)
    A, B, C = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().tmnd_fit_mg_time(_pd(s), _pd(tt), len(s), float(L), int(grid), ctypes.byref(A), ctypes.byref(B),
                                  ctypes.byref(C)))
    return A.value, B.value, C.value
