"""Write the stored expected values under tests/golden/ by running the FP64
oracle (and nothing else).  Usage: python tests/golden/make_golden.py [name]

mms_16x16x16x32.json: the oracle's multi-shift CG on the 16^3x32 workload
(kappa 0.16, mu_bar 0.1, eps_bar 0.11, antiperiodic time, roughness 0.5,
gauge seed 1002, RHS seed 2032, 12 shifts log-spaced in 1e-5..2, rho 1e-10):
iteration count, per-shift freezing iterations, final zeta, and the
oracle-computed true residual of every shift.  Takes about three minutes on 8 cores.

mms_32x32x32x64.json: the same for the first right-hand side of the 32^3x64
workload (gauge seed 1004, RHS seed 2004, right-hand side 0 of 8; otherwise as
above).  Its iteration count scales the timed sample of the CPU baseline at that
size.  Takes about an hour on 8 cores and ~13 GB of memory."""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def _mms_workload(name, dims, gseed, bseed, nrhs, lattice):
    U = synth.random_su3_field(dims, 0.5, gseed)
    b = synth.gaussian_rhs(dims, bseed, nrhs=nrhs)[0]
    act = oracle.action(dims, 0.16, 0.1, 0.11)
    sig = synth.shift_set(12, 1e-5, 2.0)
    t = time.time()
    res = oracle.mms_cg(act, U, b, sig, rho=1e-10)
    el = time.time() - t
    tr = [oracle.true_residual(act, U, b, res["x"][i], s) for i, s in enumerate(sig)]
    out = {"workload": f"{lattice} ND twisted mass, kappa 0.16, mu_bar 0.1, eps_bar 0.11, APBC, "
                       f"roughness 0.5, gauge seed {gseed}, rhs seed {bseed} (right-hand side 0 of {nrhs}), "
                       "12 shifts 1e-5..2, rho 1e-10",
           "sigma": list(map(float, sig)), "iters": int(res["iters"]),
           "conv_iter": [int(v) for v in res["conv_iter"]], "zeta": [float(v) for v in res["zeta"]],
           "true_res": tr, "oracle_seconds": el, "oracle_threads": oracle.nthreads()}
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


def mms_bench_workload():
    _mms_workload("mms_16x16x16x32", (32, 16, 16, 16), 1002, 2032, 1, "16^3x32")


def mms_32_workload():
    _mms_workload("mms_32x32x32x64", (64, 32, 32, 32), 1004, 2004, 8, "32^3x64")


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "mms_16x16x16x32"
    {"mms_16x16x16x32": mms_bench_workload, "mms_32x32x32x64": mms_32_workload}[which]()
