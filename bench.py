"""Benchmark: shift-system solves/s at relative residual 1e-10 on one GB300.

Workload (N = 1): the 16^3x32 FP64 multi-shift solve of the ND twisted-mass
doublet (kappa 0.16, mu_bar 0.1, eps_bar 0.11, antiperiodic time, seeded
SU(3) links with roughness 0.5), 12 shifts log-spaced in 1e-5..2, one
Gaussian right-hand side, rho = 1e-10.  A step is one complete multi-shift CG
solve (all shifts, with the FP64 true-residual certification).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tmnd|reference]
                    [--form fp64|mixed|batched|hybrid|learned]

--form selects one of the solver forms on its own workload (the default, fp64,
is the headline above); every form certifies each shift at 1e-10 by its FP64
true residual:
  mixed    24^3x48, 12 shifts, 2 RHS one at a time: sloppy FP32/16-bit multi-shift
           CG + FP64 defect correction
  batched  32^3x64, 12 shifts, 8 RHS: the same with all 8 RHS in every 16-bit
           stencil launch
  hybrid   32^3x64, 12 shifts, 8 RHS: mixed multi-shift CG for the 8 largest,
           Lagrange guesses and case-C two-level MG (4^4 aggregates, 24 vectors
           per chirality, coarse operator on the tensor cores) for the 4 smallest
           (the MG setup is built once per gauge field, outside the timed region)
  learned  24^3x48, 12 shifts, 1 RHS on an unseen field: mixed multi-shift CG for
           the 8 largest, learned guesses for the 4 smallest finished by defect
           correction; the network is trained first on solves of other fields
           (outside the timed region); the same with Lagrange guesses is reported
  rational 24^3x48, 2 RHS: x = R(Qhat^2) b ~ (Qhat^2)^(-1/2) b with Zolotarev's n = 10
           approximation on the spectrum bounds from a Lanczos estimate (mixed
           multi-shift CG over the 10 Zolotarev shifts + one combination)
Each form's line also times the plain FP64 multi-shift CG on its workload
("fp64_same_workload") and reports a roofline for its dominant kernel.

--study errors runs App. A's comparison of equivalent solutions (methods A-F) on the
16^3x32 field against a known solution, rho = 1e-2 .. 1e-10.
--study learned runs config 5: train on solves of 20 fields, evaluate on 5 unseen
fields (CG iterations for the 4 smallest shifts from zero, Lagrange and learned guesses).
--study hybrid measures the hybrid cost model of Sec. 4.3 on GB300 (24^3x48):
per-shift CG and MG times, their fits, the model's optimal n and the measured
hybrid time for every n, without and with Lagrange guesses.

--kernel fp64|s16|coarse times one kernel family alone (CUDA events, L2 flushed
between applications) and prints its achieved rate against the roofline:
  fp64    FP64 Qhat^2 + sigma (4 stencil launches), 16^3x32
  s16     16-bit Qhat^2 + sigma (4 stencil launches), 24^3x48, 1 and 8 RHS per launch
  coarse  coarse doublet operator, tensor cores and CUDA cores, 24^3x48 with 4^4
          aggregates and 24 vectors per chirality, 1 and 8 RHS

--impl reference times the FP64 CPU oracle (the only other implementation of
this method here) on the host cores, on a bounded sample of the same workload.
Under torchrun (N > 1) every rank solves its own right-hand side (replicas: the
path has no data exchange between independent solves); value = all ranks'
solves / max-over-ranks time.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (32, 16, 16, 16)            # T, X, Y, Z
KAPPA, MU_BAR, EPS_BAR = 0.16, 0.1, 0.11
ROUGHNESS = 0.5
GAUGE_SEED, RHS_SEED = 1002, 2032
NSHIFT, SIG_LO, SIG_HI = 12, 1e-5, 2.0
RHO = 1e-10
METRIC = "shift-system solves/sec at rel. residual 1e-10"
WORKLOAD = "16^3x32 ND twisted-mass doublet, FP64 multi-shift CG, 12 shifts 1e-5..2, 1 RHS, rho 1e-10"
L2_FLUSH_BYTES = 512 << 20         # > 129 MB L2

# Algorithmic counts per odd site for ONE stencil launch (both flavours):
#   flops: 2 x 1320 (Wilson hop with spin projection, 8 directions) + 240 (A^-1 or A site term)
#   bytes (FP64, 18-real links): even launch 240 reals (in 48, links 144, out 48),
#   odd launch 288 reals (t 48, psi 48, links 144, out 48)
HOP_FLOP_PER_SITE = 2 * 1320 + 240
HOP_BYTES_PER_SITE = (240 + 288) / 2 * 8
# DRAM bytes of one odd-site FP64 stencil launch at 16^3x32, one ncu capture of this kernel
# (dram__bytes_read.sum + dram__bytes_write.sum: 132.87 MB + 9.04 MB)
FP64_ODD_LAUNCH_TRAFFIC = 132.866816e6 + 9.036288e6
# DRAM bytes of the 16-bit stencil at 24^3x48 (V/2 = 331776), one ncu capture: even launch
# 98.22 + 3.71 MB, odd launch 134.10 + 7.79 MB; Qhat^2 = 2 even + 2 odd launches
# DRAM bytes (read + write) of one 16-bit Qhat^2 + sigma at 24^3x48: the 4 launches of one ncu capture
S16_Q2_TRAFFIC_24 = (97.503232e6 + 3.967232e6) + (132.547840e6 + 8.404480e6) + (97.519360e6 + 3.632896e6) \
    + (169.893632e6 + 15.372288e6)
S16_TRAFFIC_VH = 331776


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_rhs_seed(rank: int) -> int:
    """Seed of rank `rank`'s right-hand side: every replica solves its own system."""
    return RHS_SEED + rank


def max_over_ranks(ms: float, ws: int, device="cuda") -> float:
    """The slowest rank's time (all ranks' work is done only when it is)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, ws: int, ms_max: float) -> float:
    """Units all ranks processed divided by the max-over-ranks time (per second)."""
    return units_per_rank * ws / (ms_max / 1e3)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_tmnd(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1805_09584_gb300 as tm
    import synth
    from paper_1805_09584_gb300 import _build

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    _build.build()

    U = synth.random_su3_field(DIMS, ROUGHNESS, GAUGE_SEED)
    b_host = synth.gaussian_rhs(DIMS, replica_rhs_seed(rank))[0]
    sig = synth.shift_set(NSHIFT, SIG_LO, SIG_HI)
    g = tm.Gauge(U, DIMS, KAPPA, MU_BAR, EPS_BAR)
    stream = torch.cuda.current_stream()
    b_dev = g.pack(torch.from_numpy(b_host).cuda())
    xs = [g.spinor() for _ in sig]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(profile=False):
        return tm.mms_cg_solve(g.handle, b_dev, 1, sig, xs, rho=RHO, profile=profile, stream=stream)

    # nvidia-smi starts before the warm-up, so that its start-up does not overlap the timed region
    sampler = ClockSampler(local)
    for _ in range(args.warmup):
        info = step()
    # ---- timed region: K solves, L2 flushed between solves
    infos = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        flush.fill_(1.0)
        infos.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ms_all = max_over_ranks(ms, ws)
    solves = args.steps * NSHIFT * ws
    value = whole_job_rate(args.steps * NSHIFT, ws, ms_all)
    worst_res = max(max(i["true_res"]) for i in infos)
    iters = infos[-1]["iters"]

    # ---- e2e: the public API with host buffers (pinned b in, all x_i out, per step)
    b_pin = torch.from_numpy(b_host).pin_memory()
    x_pin = torch.empty((NSHIFT, g.vh, 2, 4, 3), dtype=torch.complex128).pin_memory()
    b_can = torch.empty((1, g.vh, 2, 4, 3), dtype=torch.complex128, device="cuda")
    x_can = torch.empty((1, g.vh, 2, 4, 3), dtype=torch.complex128, device="cuda")
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        flush.fill_(1.0)
        b_can.copy_(b_pin, non_blocking=True)
        tm.tmnd_spinor_pack(g.handle, b_dev, b_can, 1, stream)
        tm.mms_cg_solve(g.handle, b_dev, 1, sig, xs, rho=RHO, stream=stream)
        for i in range(NSHIFT):
            tm.tmnd_spinor_unpack(g.handle, x_can, xs[i], 1, stream)
            x_pin[i].copy_(x_can[0], non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), ws)
    e2e_value = whole_job_rate(args.steps * NSHIFT, ws, e2e_ms)
    h2d = b_host.nbytes
    d2h = NSHIFT * b_host.nbytes

    # ---- roofline of the dominant kernel (the FP64 stencil launches): one more
    # solve, identical to the timed ones, with CUDA events recorded around the
    # stencil and update launches of every iteration (event nodes in the graph;
    # kept out of the timed region so that they do not slow the headline number)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    pinfo = step(profile=True)
    p1.record(stream)
    torch.cuda.synchronize()
    prof_ms = p0.elapsed_time(p1)
    hop_ms = pinfo["hop_ms"]
    n_hop_launch = 4 * pinfo["iters"]
    hop_avg_s = hop_ms / 1e3 / n_hop_launch
    flop_per_launch = HOP_FLOP_PER_SITE * g.vh
    achieved_tflops = flop_per_launch / hop_avg_s / 1e12
    fp64_peak = FP64_PEAK_TFLOPS
    upd_ms = pinfo["update_ms"]
    launches = sum(i["launches"] for i in infos)

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": "16^3x32", "nshift": NSHIFT, "nrhs": 1,
                       "rho": RHO, "kappa": KAPPA, "mu_bar": MU_BAR, "eps_bar": EPS_BAR, "roughness": ROUGHNESS,
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "flushed between steps (512 MB write); solve working set > L2"},
            "iters": iters, "max_true_rel_residual": worst_res,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "alu", "kernel": "k_hop_even/k_hop_odd (FP64 stencil)",
                         "achieved": achieved_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved_tflops / fp64_peak, "traffic": FP64_ODD_LAUNCH_TRAFFIC,
                         "traffic_note": "DRAM bytes per odd-site launch (ncu capture of this kernel, this workload)",
                         "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)",
                         "hop_share_of_step": hop_ms / prof_ms,
                         "measured": "CUDA events around every iteration's 4 stencil launches of a profiled "
                                     "solve run right after the timed steps",
                         "hop_achieved_gbs": HOP_BYTES_PER_SITE * g.vh / hop_avg_s / 1e9,
                         "hbm_peak_gbs": _peaks().get("hbm_gbs")},
            "update_share_of_step": upd_ms / prof_ms,
            "gpu_launches": launches,
            "clocks": clocks,
        }
    g.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out



FORMS = {
    "mixed": dict(dims=(48, 24, 24, 24), nrhs=2, seeds=(1003, 2003), lattice="24^3x48"),
    "batched": dict(dims=(64, 32, 32, 32), nrhs=8, seeds=(1004, 2004), lattice="32^3x64"),
    "hybrid": dict(dims=(64, 32, 32, 32), nrhs=8, seeds=(1004, 2004), lattice="32^3x64"),
    "learned": dict(dims=(48, 24, 24, 24), nrhs=1, seeds=(1005, 2005), lattice="24^3x48"),
    "rational": dict(dims=(48, 24, 24, 24), nrhs=2, seeds=(1003, 2003), lattice="24^3x48"),
}
# 16-bit stencil, algorithmic bytes per odd site: even launch 392 (in 100, 12-real
# 16-bit links 192, out 100), odd launch 492 (+ psi 100); Qhat^2 + sigma adds aux 100
S16_Q2_BYTES_PER_SITE = 2 * (392 + 492) + 100


def _timed(step, steps, flush, stream):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    e0.record(stream)
    for _ in range(steps):
        flush.fill_(1.0)
        out.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def s16_roofline(tm, g, flush, stream, reps=20):
    """CUDA-event time of the sloppy Qhat^2 (4 stencil launches) on the form's lattice."""
    import torch
    q = g.spinor(1, prec=tm.TMND_S16)
    tm.tmnd_spinor_convert(g.handle, q, tm.TMND_S16, g.pack(torch.randn(g.vh * 24, dtype=torch.complex128,
                                                                          device="cuda").view(1, g.vh, 2, 4, 3)),
                           tm.TMND_F64)
    o = g.spinor(1, prec=tm.TMND_S16)
    for _ in range(3):
        tm.tm_nd_apply(g.handle, o, q, tm.OP_QHAT2 | tm.OP_S16, 0.01, stream=stream)
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tm.tm_nd_apply(g.handle, o, q, tm.OP_QHAT2 | tm.OP_S16, 0.01, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    peak = _peaks().get("hbm_gbs") or 6800.0
    gbs = S16_Q2_BYTES_PER_SITE * g.vh / (ms / 1e3) / 1e9
    scaled = g.vh != S16_TRAFFIC_VH
    return {"bound": "hbm", "kernel": "k_hop_even_s16/k_hop_odd_s16 (16-bit stencil, Qhat^2 + sigma: 4 launches)",
            "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "traffic": S16_Q2_TRAFFIC_24 * g.vh / S16_TRAFFIC_VH,
            "traffic_note": "DRAM bytes per Qhat^2 from an ncu capture at 24^3x48 (its 4 launches; below the "
                            "algorithmic bytes because each launch's output is still in L2 when the next reads it)"
                            + (", scaled by the number of sites" if scaled else ""),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs" if _peaks().get("hbm_gbs") else "fallback 6.8 TB/s",
            "measured": f"median of {reps} CUDA-event timings of tm_nd_apply(Qhat^2, 16-bit), L2 flushed",
            "ms_per_qhat2": ms}


def run_form(args):
    """One solver form on its own workload (see the module docstring)."""
    import numpy as np
    import torch

    import paper_1805_09584_gb300 as tm
    import synth
    from paper_1805_09584_gb300 import _build, learned

    ws, rank, local = _dist()
    if ws > 1:
        raise SystemExit("--form runs on one GPU")
    torch.cuda.set_device(local)
    _build.build()
    F = FORMS[args.form]
    dims, nrhs = F["dims"], F["nrhs"]
    gseed, bseed = F["seeds"]
    sig = synth.shift_set(NSHIFT, SIG_LO, SIG_HI)
    U = synth.random_su3_field(dims, ROUGHNESS, gseed)
    g = tm.Gauge(U, dims, KAPPA, MU_BAR, EPS_BAR)
    stream = torch.cuda.current_stream()
    b_host = synth.gaussian_rhs(dims, bseed, nrhs=nrhs)
    b_dev = g.pack(torch.from_numpy(b_host).cuda(), nrhs=nrhs)
    xs = [g.spinor(nrhs) for _ in sig]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    extra = {}
    mg = net = None
    if args.form == "hybrid":
        t0 = time.perf_counter()
        nv = 24
        tv = torch.randn(nv * 2 * 12 * g.vh, dtype=torch.complex64, device="cuda")
        tm.tmnd_mg_smooth_vectors(g.handle, tv, nv, 4)
        mg = tm.tmnd_mg_create(g.handle, (4, 4, 4, 4), nv, tv)
        torch.cuda.synchronize()
        extra["mg_setup_s"] = time.perf_counter() - t0
        del tv
    if args.form == "learned":
        t0 = time.perf_counter()
        Xs, Ss, Hs = [], [], []
        for fs in range(4):   # training fields (roughness 0.3..0.7), 2 RHS each
            gt = tm.Gauge(synth.random_su3_field(dims, 0.3 + 0.1 * fs, 100 + fs), dims, KAPPA, MU_BAR, EPS_BAR)
            for bk in synth.gaussian_rhs(dims, 200 + fs, nrhs=2):
                bd = gt.pack(torch.from_numpy(bk[None]).cuda())
                xn, info, hist = learned.solve_nodes(gt, bd, sig, prec=tm.TMND_S16)
                X, S, H = learned.samples(gt, bd, sig, xn, info, hist)
                Xs.append(X); Ss.append(S); Hs.append(H)
                del xn
            gt.close()
        net, losses = learned.train(np.concatenate(Xs), np.concatenate(Ss), np.concatenate(Hs), epochs=600)
        extra["training"] = {"solves": 8, "samples": 32, "fields": 4, "s": time.perf_counter() - t0,
                             "loss_first_last": [losses[0], losses[-1]]}

    if args.form == "rational":
        # spectrum bounds of Qhat^2 from the Ritz values of one FP64 CG history (10 % margins)
        hist = np.zeros(8192)
        xb = [g.spinor(1)]
        inf = tm.mms_cg_solve(g.handle, b_dev[: 24 * g.vh], 1, [1e-5], xb, rho=1e-8, ab_hist=hist)
        f = tm.tmnd_mlp_features(sig[:8], float(sig[8]), hist, inf["iters"], 1e-5)
        lmin, lmax = 0.9 * 10 ** float(f[17]), 1.1 * 10 ** float(f[18])
        a_z, c_z, q_z, delta = tm.tmnd_zolotarev(10, lmin / lmax)
        sig = lmax * c_z[1::2]                 # the shifts the multi-shift solve sees
        out_r = g.spinor(nrhs)
        extra["rational"] = {"n": 10, "lambda_min": lmin, "lambda_max": lmax, "delta": delta,
                             "shifts": [float(v) for v in sig]}
        del xb

    def step():
        if args.form == "rational":
            return tm.tmnd_rational_apply(g.handle, b_dev, nrhs, 10, lmin, lmax, out_r, rho=RHO, prec=tm.TMND_S16,
                                          stream=stream)
        if args.form in ("mixed", "batched"):
            return tm.mms_cg_solve(g.handle, b_dev, nrhs, sig, xs, rho=RHO, prec=tm.TMND_S16,
                                   batch=1 if args.form == "mixed" else 0, stream=stream)
        if args.form == "hybrid":
            return tm.tmnd_hybrid_solve(g.handle, mg, b_dev, nrhs, sig, 8, xs, rho=RHO, prec=tm.TMND_S16,
                                        n_guess=0, guess=1, stream=stream)
        return tm.tmnd_hybrid_solve(g.handle, None, b_dev, nrhs, sig, 8, xs, rho=RHO, prec=tm.TMND_S16,
                                    n_guess=0, guess=2, net=net, stream=stream)

    sampler = ClockSampler(local)
    for _ in range(args.warmup):
        step()
    ms, infos = _timed(step, args.steps, flush, stream)
    clocks = sampler.stop()
    solves = args.steps * len(sig) * nrhs
    value = solves / (ms / 1e3)
    worst = max(max(i["true_res"]) for i in infos)
    if args.form == "learned":   # the same with Lagrange guesses (the method without the network)
        def step_lag():
            return tm.tmnd_hybrid_solve(g.handle, None, b_dev, nrhs, sig, 8, xs, rho=RHO, prec=tm.TMND_S16,
                                        n_guess=0, guess=1, stream=stream)
        step_lag()
        ms_l, inf_l = _timed(step_lag, args.steps, flush, stream)
        extra["lagrange_guesses"] = {"value": solves / (ms_l / 1e3), "ms_per_step": ms_l / args.steps,
                                     "guess_res": inf_l[-1]["guess_res"][8:],
                                     "refine_iters": inf_l[-1]["refine_iters"],
                                     "fp64_applies": inf_l[-1]["fp64_applies"]}
        extra["learned_guesses"] = {"guess_res": infos[-1]["guess_res"][8:], "refine_iters": infos[-1]["refine_iters"],
                                    "fp64_applies": infos[-1]["fp64_applies"]}
    # e2e: host buffers in and out through the public API
    b_pin = torch.from_numpy(b_host).pin_memory()
    x_pin = torch.empty((NSHIFT, nrhs, g.vh, 2, 4, 3), dtype=torch.complex128).pin_memory()
    b_can = torch.empty((nrhs, g.vh, 2, 4, 3), dtype=torch.complex128, device="cuda")
    x_can = torch.empty((nrhs, g.vh, 2, 4, 3), dtype=torch.complex128, device="cuda")

    outs = [out_r] if args.form == "rational" else xs

    def step_e2e():
        b_can.copy_(b_pin, non_blocking=True)
        tm.tmnd_spinor_pack(g.handle, b_dev, b_can, nrhs, stream)
        step()
        for i, v in enumerate(outs):
            tm.tmnd_spinor_unpack(g.handle, x_can, v, nrhs, stream)
            x_pin[i].copy_(x_can, non_blocking=True)
    e2e_ms, _ = _timed(step_e2e, args.steps, flush, stream)
    # the plain FP64 multi-shift CG on the same workload (one step), and each form's solutions
    # against its solutions: max over shifts of |x_form - x_FP64| / |x_FP64| (all RHS together)
    keep = [v.clone() for v in xs[:len(sig)]] if args.form != "rational" else None
    f64 = lambda: tm.mms_cg_solve(g.handle, b_dev, nrhs, sig, xs[:len(sig)], rho=RHO, stream=stream)
    f64()
    f64_ms, _ = _timed(f64, 1, flush, stream)
    if keep is not None:
        dx = [float(torch.linalg.vector_norm(k - v) / torch.linalg.vector_norm(v)) for k, v in zip(keep, xs)]
        extra["rel_diff_vs_fp64"] = {"max": max(dx), "per_shift": [float("%.3g" % d) for d in dx]}
        del keep
    roof = s16_roofline(tm, g, flush, stream)
    if mg is not None:   # the coarse operator on the tensor cores, all 8 RHS at once
        nb = g.vh * 2 // 256
        xc = torch.randn(nrhs * nb * 4 * 24, dtype=torch.complex64, device="cuda")
        yc = torch.empty_like(xc)
        tm.mg_coarse_apply(mg, yc, xc, nrhs, 0.0, stream=stream)
        c_ms, _ = _timed(lambda: tm.mg_coarse_apply(mg, yc, xc, nrhs, 0.0, stream=stream), 10, flush, stream)
        byts = nb * 9 * 48 * 48 * 8 + 2 * nrhs * nb * 4 * 24 * 8
        extra["coarse_tc"] = {"ms": c_ms / 10, "GBs": byts / (c_ms / 10 / 1e3) / 1e9, "nrhs": nrhs,
                              "kernel": "k_coarse_apply_tc (tcgen05 TF32, 48x48 blocks)"}
    launches = sum(i.get("launches", 0) for i in infos) or None
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/16-bit sloppy + f64 defect correction", "data": "synthetic",
        "config": {"workload": f"{F['lattice']} ND twisted-mass doublet, {args.form} form, "
                               + ("Zolotarev n = 10 shifts" if args.form == "rational" else "12 shifts 1e-5..2")
                               + f", {nrhs} RHS, rho 1e-10", "form": args.form, "lattice": F["lattice"],
                   "nshift": len(sig), "nrhs": nrhs, "rho": RHO, "kappa": KAPPA, "mu_bar": MU_BAR,
                   "eps_bar": EPS_BAR, "roughness": ROUGHNESS, "parallelism": "single GPU",
                   "l2": "flushed between steps (512 MB write); solve working set > L2"},
        "max_true_rel_residual": worst,
        "fp64_same_workload": {"value": nrhs * len(sig) / (f64_ms / 1e3), "ms_per_step": f64_ms},
        "e2e": {"value": solves / (e2e_ms / 1e3), "unit": "solves/s", "h2d_bytes_per_step": b_host.nbytes,
                "d2h_bytes_per_step": len(outs) * b_host.nbytes},
        "roofline": roof, "gpu_launches": launches, "clocks": clocks, **extra,
    }
    if net is not None:
        tm.tmnd_mlp_destroy(net)
    if mg is not None:
        tm.tmnd_mg_destroy(mg)
    g.close()
    return out



def run_kernel(args):
    """One kernel family alone on its workload lattice (see the module docstring)."""
    import torch

    import paper_1805_09584_gb300 as tm
    import synth
    from paper_1805_09584_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    peak_hbm = _peaks().get("hbm_gbs") or 6800.0
    reps = max(args.steps, 10)

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    out = {"kernel": args.kernel, "reps": reps, "timing": "median of CUDA-event timings, L2 flushed between"}
    if args.kernel == "fp64":
        dims = DIMS
        g = tm.Gauge(synth.random_su3_field(dims, ROUGHNESS, GAUGE_SEED), dims, KAPPA, MU_BAR, EPS_BAR)
        x = g.pack(torch.from_numpy(synth.gaussian_rhs(dims, RHS_SEED)).cuda())
        y = g.spinor()
        ms = timed(lambda: tm.tm_nd_apply(g.handle, y, x, tm.OP_QHAT2, 0.01, stream=stream))
        tf = 4 * HOP_FLOP_PER_SITE * g.vh / (ms / 1e3) / 1e12
        out.update(lattice="16^3x32", ms_qhat2=ms, tflops=tf, fp64_peak_tflops=FP64_PEAK_TFLOPS,
                   frac=tf / FP64_PEAK_TFLOPS, gbs=4 * HOP_BYTES_PER_SITE * g.vh / (ms / 1e3) / 1e9)
    elif args.kernel == "s16":
        for dims, name, rs in (((48, 24, 24, 24), "24^3x48", (1, 8)), ((64, 32, 32, 32), "32^3x64", (1,))):
            g = tm.Gauge(synth.random_su3_field(dims, ROUGHNESS, 1003), dims, KAPPA, MU_BAR, EPS_BAR)
            for R in rs:
                b = g.pack(torch.from_numpy(synth.gaussian_rhs(dims, 2003, nrhs=R)).cuda(), nrhs=R)
                q = g.convert(b, tm.TMND_F64, tm.TMND_S16, nrhs=R)
                o = g.spinor(R, prec=tm.TMND_S16)
                del b
                ms = timed(lambda: tm.tm_nd_apply(g.handle, o, q, tm.OP_QHAT2 | tm.OP_S16, 0.01, nrhs=R,
                                                  stream=stream))
                # links are read once per launch for all R right-hand sides
                byts = g.vh * (R * (2 * (200 + 300) + 100) + 4 * 192)
                out[f"{name}_nrhs{R}"] = {"ms_qhat2": ms, "ms_per_rhs": ms / R, "gbs": byts / (ms / 1e3) / 1e9,
                                          "frac_hbm": byts / (ms / 1e3) / 1e9 / peak_hbm}
                del q, o
            g.close()
        out.update(hbm_peak_gbs=peak_hbm)
        return out
    else:
        dims, nv = (48, 24, 24, 24), 24
        g = tm.Gauge(synth.random_su3_field(dims, ROUGHNESS, 1003), dims, KAPPA, MU_BAR, EPS_BAR)
        tv = torch.randn(nv * 2 * 12 * g.vh, dtype=torch.complex64, device="cuda")
        tm.tmnd_mg_smooth_vectors(g.handle, tv, nv, 4)
        mg = tm.tmnd_mg_create(g.handle, (4, 4, 4, 4), nv, tv)
        mgs = tm.tmnd_mg_create(g.handle, (4, 4, 4, 4), nv, tv, coarse_simt=True)
        del tv
        nb = 2 * g.vh // 256
        for R in (1, 8):
            xc = torch.randn(R * nb * 4 * nv, dtype=torch.complex64, device="cuda")
            yc = torch.empty_like(xc)
            byts = nb * 9 * (2 * nv) ** 2 * 8 + 2 * R * nb * 4 * nv * 8
            for name, h in (("tc", mg), ("simt", mgs)):
                ms = timed(lambda: tm.mg_coarse_apply(h, yc, xc, R, 0.0, stream=stream))
                out[f"{name}_nrhs{R}"] = {"ms": ms, "gbs": byts / (ms / 1e3) / 1e9,
                                          "frac_hbm": byts / (ms / 1e3) / 1e9 / peak_hbm}
        out.update(lattice="24^3x48, 4^4 aggregates, 24 vectors per chirality", hbm_peak_gbs=peak_hbm)
        tm.tmnd_mg_destroy(mg)
        tm.tmnd_mg_destroy(mgs)
    g.close()
    return out



def run_study(args):
    """Hybrid cost model on GB300 (Sec. 4.3): per shift the mixed CG time t_CG and the
    case-C MG time t_MG (zero start), fits of Eqs. "CGtime2" / "MGtime2", the model's
    c_HY(n) and n_opt, and the measured hybrid time for every n, without and with guesses."""
    import numpy as np
    import torch

    import paper_1805_09584_gb300 as tm
    import synth
    from paper_1805_09584_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    dims = (48, 24, 24, 24)
    g = tm.Gauge(synth.random_su3_field(dims, ROUGHNESS, 1003), dims, KAPPA, MU_BAR, EPS_BAR)
    sig = synth.shift_set(NSHIFT, SIG_LO, SIG_HI)
    b = g.pack(torch.from_numpy(synth.gaussian_rhs(dims, 2003)).cuda())
    xs = [g.spinor() for _ in sig]
    nv = 24
    tv = torch.randn(nv * 2 * 12 * g.vh, dtype=torch.complex64, device="cuda")
    tm.tmnd_mg_smooth_vectors(g.handle, tv, nv, 4)
    mg = tm.tmnd_mg_create(g.handle, (4, 4, 4, 4), nv, tv)
    del tv
    hist = np.zeros(8192)
    inf = tm.mms_cg_solve(g.handle, b, 1, [SIG_LO], xs[:1], rho=1e-8, ab_hist=hist)
    f = tm.tmnd_mlp_features(sig[:8], float(sig[8]), hist, inf["iters"], SIG_LO)
    lmin, lmax = 10 ** float(f[17]), 10 ** float(f[18])

    def wall(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) * 1e3, out

    wall(lambda: tm.mms_cg_solve(g.handle, b, 1, sig[-1:], xs[:1], rho=RHO, prec=tm.TMND_S16))
    t_cg = [wall(lambda s=s: tm.mms_cg_solve(g.handle, b, 1, [s], xs[:1], rho=RHO, prec=tm.TMND_S16))[0]
            for s in sig]
    hyb = lambda n, guess: tm.tmnd_hybrid_solve(g.handle, mg, b, 1, sig, n, xs, rho=RHO, prec=tm.TMND_S16,
                                                n_guess=0, guess=guess)
    hyb(1, 0)
    _, h0 = wall(lambda: hyb(1, 0))
    t_mg = h0["shift_ms"][1:]                       # shifts 1..N-1 by MG from zero
    a, bb = tm.tmnd_fit_cg_time(sig, t_cg, lmin, lmax)
    A, B, C = tm.tmnd_fit_mg_time(sig[1:], t_mg, lmax)
    cost, n_opt = tm.tmnd_hybrid_cost(sig, (a, bb, lmin, lmax), (A, B, C, lmax))
    meas0 = [wall(lambda n=n: hyb(n, 0))[0] for n in range(1, NSHIFT + 1)]
    meas1 = [wall(lambda n=n: hyb(n, 1))[0] for n in range(1, NSHIFT + 1)]
    tm.tmnd_mg_destroy(mg)
    g.close()
    r = lambda v: [round(float(x), 2) for x in v]
    return {"study": "hybrid cost model (Sec. 4.3) on GB300", "lattice": "24^3x48", "shifts": r(sig),
            "spectrum": {"lambda_min": lmin, "lambda_max": lmax, "source": "Ritz values of a CG history"},
            "t_cg_ms": r(t_cg), "t_mg_ms": r(t_mg),
            "fit_cg": {"a": a, "b": bb}, "fit_mg": {"A": A, "B": B, "C": C, "L": lmax},
            "model_cost_ms": r(cost), "model_n_opt": n_opt,
            "measured_ms_no_guess": r(meas0), "measured_n_opt_no_guess": int(np.argmin(meas0)) + 1,
            "measured_ms_lagrange": r(meas1), "measured_n_opt_lagrange": int(np.argmin(meas1)) + 1,
            "note": "n = shifts by the mixed multi-shift CG; the rest by case-C MG + FP64 defect correction"}



def run_study_learned(args):
    """Config 5: network trained on solves of 20 seeded fields (roughness 0.3..0.7,
    RHS_PER_FIELD each), evaluated on 5 unseen fields (roughness 0.3, 0.4, ..., 0.7):
    CG iterations to 1e-10 for the 4 smallest shifts from the zero vector, from the
    Lagrange guess (Sec. 4.2.1) and from the learned guess, over the 8 solved shifts
    just above each target."""
    import numpy as np
    import torch

    import paper_1805_09584_gb300 as tm
    import synth
    from paper_1805_09584_gb300 import _build, learned

    _build.build()
    torch.cuda.set_device(0)
    dims = (48, 24, 24, 24)
    sig = synth.shift_set(NSHIFT, SIG_LO, SIG_HI)
    per_field = int(os.environ.get("RHS_PER_FIELD", "10"))
    t0 = time.perf_counter()
    Xs, Ss, Hs = [], [], []
    for f in range(20):
        r = 0.3 + 0.4 * ((f * 37) % 100) / 100.0
        g = tm.Gauge(synth.random_su3_field(dims, r, f), dims, KAPPA, MU_BAR, EPS_BAR)
        for bk in synth.gaussian_rhs(dims, 3000 + 16 * f, nrhs=per_field):
            bd = g.pack(torch.from_numpy(bk[None]).cuda())
            xn, info, hist = learned.solve_nodes(g, bd, sig, prec=tm.TMND_S16)
            X, S, H = learned.samples(g, bd, sig, xn, info, hist)
            Xs.append(X); Ss.append(S); Hs.append(H)
            del xn
        g.close()
    t_data = time.perf_counter() - t0
    net, losses = learned.train(np.concatenate(Xs), np.concatenate(Ss), np.concatenate(Hs), epochs=800)
    t_train = time.perf_counter() - t0 - t_data
    it = {"zero": np.zeros((5, 4), int), "lagrange": np.zeros((5, 4), int), "learned": np.zeros((5, 4), int)}
    gres = {"lagrange": np.zeros((5, 4)), "learned": np.zeros((5, 4))}
    for e in range(5):
        r = 0.3 + 0.1 * e
        g = tm.Gauge(synth.random_su3_field(dims, r, 100 + e), dims, KAPPA, MU_BAR, EPS_BAR)
        b = synth.gaussian_rhs(dims, 5000 + e)
        bd = g.pack(torch.from_numpy(b).cuda())
        xn, info, hist = learned.solve_nodes(g, bd, sig, prec=tm.TMND_S16)
        X, S, H = learned.samples(g, bd, sig, xn, info, hist)
        w_net = learned.predict(net, X, S)
        for q in range(4):
            t = float(sig[8 + q])
            nodes_x = xn[q:q + 8]
            wl = learned.lagrange_weights(sig[q:q + 8], t)
            z = tm.mms_cg_solve(g.handle, bd, 1, [t], [g.spinor()], rho=RHO)
            it["zero"][e, q] = z["iters"]
            it["lagrange"][e, q], gres["lagrange"][e, q] = learned.iterations_from_guess(g, bd, nodes_x, wl, t)
            it["learned"][e, q], gres["learned"][e, q] = learned.iterations_from_guess(g, bd, nodes_x, w_net[q], t)
        g.close()
    tm.tmnd_mlp_destroy(net)
    tot = {k: int(v.sum()) for k, v in it.items()}
    return {"study": "learned guesses (config 5)", "lattice": "24^3x48",
            "training": {"fields": 20, "rhs_per_field": per_field, "solves": 20 * per_field,
                         "samples": int(sum(len(x) for x in Xs)), "data_s": t_data, "train_s": t_train,
                         "loss_first_last": [losses[0], losses[-1]]},
            "evaluation": "5 unseen fields (roughness 0.3..0.7), 1 RHS each; FP64 CG iterations to rel. residual "
                          "1e-10 for shifts 8..11 (the 4 smallest) from each guess",
            "iterations": {k: v.tolist() for k, v in it.items()}, "iterations_total": tot,
            "guess_rel_residual": {k: [[float("%.3g" % x) for x in row] for row in v] for k, v in gres.items()},
            "saved_vs_lagrange": tot["lagrange"] - tot["learned"], "saved_vs_zero": tot["zero"] - tot["learned"]}



def run_study_errors(args):
    """App. A (error and residual of equivalent solutions) on the 16^3x32 field: a known
    Gaussian x, b = (Qhat^2 + mu^2) x, methods A (direct), B (two consecutive single
    systems), C (i/(2 mu) (x_+ - x_-)) and, for (Qhat + i mu) x_+ = b, methods D, E, F,
    each stopped at rho; |r|/|b|, |e|/|b|, the smallest / largest site norm of e and
    App. A's upper limits (extreme eigenvalues of Qhat^2 from Ritz values)."""
    import numpy as np
    import torch

    import paper_1805_09584_gb300 as tm
    import synth
    from paper_1805_09584_gb300 import _build, equivalent

    _build.build()
    torch.cuda.set_device(0)
    dims = DIMS
    g = tm.Gauge(synth.random_su3_field(dims, ROUGHNESS, GAUGE_SEED), dims, KAPPA, MU_BAR, EPS_BAR)
    x = g.pack(torch.from_numpy(synth.gaussian_rhs(dims, 4000)).cuda())
    hist = np.zeros(8192)
    xr = [g.spinor()]
    inf = tm.mms_cg_solve(g.handle, x, 1, [1e-6], xr, rho=1e-8, ab_hist=hist)
    f = tm.tmnd_mlp_features(synth.shift_set(8, 1e-4, 1.0), 1e-5, hist, inf["iters"], 1e-6)
    lmin, lmax = 10 ** float(f[17]), 10 ** float(f[18])
    t0 = time.perf_counter()
    rows = []
    for mu2 in (1e-1, 1e-3, 1e-5):
        mu = float(np.sqrt(mu2))
        b = g.spinor()
        tm.tm_nd_apply(g.handle, b, x, tm.OP_QHAT2, mu2)
        xp_exact = equivalent.qpm(g, x, mu, -1)          # (Qhat + i mu)^-1 b = (Qhat - i mu) x
        for rho in (1e-2, 1e-4, 1e-6, 1e-8, 1e-10):
            sols, one = equivalent.equivalent_solutions(g, b, mu, rho)
            lim = equivalent.app_a_limits(rho, lmin, lmax, mu)
            row = {"mu2": mu2, "rho": rho}
            for c in "ABC":
                row[c] = equivalent.residual_and_error(g, b, x, sols[c], mu)
                row[c]["limits"] = list(lim[c])
            for m in "DEF":
                row[m] = equivalent.residual_and_error(g, b, xp_exact, one[(m, +1)], mu, +1)
                row[m]["limits"] = list(lim[m])
            rows.append(row)
            del sols, one
    g.close()
    return {"study": "App. A equivalent solutions", "lattice": "16^3x32", "kappa": KAPPA, "mu_bar": MU_BAR,
            "eps_bar": EPS_BAR, "x": "complex Gaussian, seed 4000", "lambda_min": lmin, "lambda_max": lmax,
            "spectrum": "extreme Ritz values of an FP64 CG history (sigma = 1e-6)",
            "normalisation": "|r| and |e| divided by |b|; site norms of e divided by the largest site norm of b",
            "single_systems": "(Qhat + i mu) x_+ = b, exact x_+ = (Qhat - i mu) x", "seconds": time.perf_counter() - t0,
            "rows": rows}


# FP64 peak of a GB300 (sm_103a): 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def cpu_baseline(iters_full: int, sample_iters: int = 6):
    """The oracle, as it stands, on the host cores: `sample_iters` MMS-CG
    iterations of the same workload, scaled to a full solve of `iters_full`
    iterations (the oracle's own count for this workload, tests/golden)."""
    import oracle
    import synth
    U = synth.random_su3_field(DIMS, ROUGHNESS, GAUGE_SEED)
    b = synth.gaussian_rhs(DIMS, RHS_SEED)[0]
    sig = synth.shift_set(NSHIFT, SIG_LO, SIG_HI)
    act = oracle.action(DIMS, KAPPA, MU_BAR, EPS_BAR)
    t = time.perf_counter()
    oracle.mms_cg(act, U, b, sig, rho=RHO, maxiter=sample_iters)
    el = time.perf_counter() - t
    per_iter = el / sample_iters
    out = {"value": NSHIFT / (per_iter * iters_full), "unit": "solves/s", "cores": oracle.nthreads(),
           "kind": "oracle",
           "sample": f"{sample_iters} MMS-CG iterations of the full 16^3x32 12-shift solve "
                     f"({el:.1f} s), scaled to the oracle's full solve of {iters_full} iterations"}
    # the same on one thread (OpenMP fixes its thread count at start-up: a child process)
    code = ("import sys, time; sys.path.insert(0, %r); import oracle, synth; "
            "U = synth.random_su3_field(%r, %r, %r); b = synth.gaussian_rhs(%r, %r)[0]; "
            "sig = synth.shift_set(%r, %r, %r); act = oracle.action(%r, %r, %r, %r); "
            "t = time.perf_counter(); oracle.mms_cg(act, U, b, sig, rho=%r, maxiter=2); "
            "print(time.perf_counter() - t)") % (ROOT, DIMS, ROUGHNESS, GAUGE_SEED, DIMS, RHS_SEED, NSHIFT, SIG_LO,
                                                 SIG_HI, DIMS, KAPPA, MU_BAR, EPS_BAR, RHO)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, OMP_NUM_THREADS="1"),
                           capture_output=True, text=True, timeout=300)
        el1 = float(r.stdout.strip().splitlines()[-1])
        out["single_thread"] = {"value": NSHIFT / (el1 / 2 * iters_full), "unit": "solves/s", "cores": 1,
                                "sample": f"2 MMS-CG iterations on one thread ({el1:.1f} s), scaled likewise"}
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        out["single_thread"] = {"value": None, "error": str(e)[:200]}
    return out


def oracle_full_iters():
    p = os.path.join(ROOT, "tests", "golden", "mms_16x16x16x32.json")
    try:
        with open(p) as f:
            return int(json.load(f)["iters"])
    except (OSError, KeyError, ValueError):
        return None


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    iters_full = oracle_full_iters()
    if iters_full is None:
        return {"impl": "reference", "unavailable": "oracle iteration count for the workload not recorded"}
    import oracle
    import synth
    U = synth.random_su3_field(DIMS, ROUGHNESS, GAUGE_SEED)
    b = synth.gaussian_rhs(DIMS, RHS_SEED)[0]
    sig = synth.shift_set(NSHIFT, SIG_LO, SIG_HI)
    act = oracle.action(DIMS, KAPPA, MU_BAR, EPS_BAR)
    sample = 2
    for _ in range(args.warmup):
        oracle.mms_cg(act, U, b, sig, rho=RHO, maxiter=1)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.mms_cg(act, U, b, sig, rho=RHO, maxiter=sample)
    el = time.perf_counter() - t
    per_iter = el / (args.steps * sample)
    value = NSHIFT / (per_iter * iters_full)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_iter * iters_full * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": "16^3x32", "nshift": NSHIFT, "nrhs": 1, "rho": RHO},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": oracle.nthreads(), "kind": "oracle",
                             "sample": f"each step: {sample} MMS-CG iterations of the full workload, scaled to "
                                       f"the oracle's {iters_full}-iteration solve"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tmnd", choices=["tmnd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="fp64", choices=["fp64", "mixed", "batched", "hybrid", "learned", "rational"])
    ap.add_argument("--kernel", default=None, choices=["fp64", "s16", "coarse"])
    ap.add_argument("--study", default=None, choices=["hybrid", "learned", "errors"])
    args = ap.parse_args()
    if args.study:
        fn = {"hybrid": run_study, "learned": run_study_learned, "errors": run_study_errors}[args.study]
        print(json.dumps(fn(args)))
        return
    if args.kernel:
        print(json.dumps(run_kernel(args)))
        return
    if args.impl == "reference":
        out = run_reference(args)
        if out is not None:
            print(json.dumps(out))
        return
    if args.form != "fp64":
        print(json.dumps(run_form(args)))
        return
    out = run_tmnd(args)
    ws, rank, _ = _dist()
    if rank == 0 and out is not None:
        if ws == 1 and not args.no_cpu_baseline:
            itf = oracle_full_iters() or out["iters"]
            out["cpu_baseline"] = cpu_baseline(itf)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
