"""Benchmark: shift-system solves/s at relative residual 1e-10 on one GB300, and the
16-bit Dslash's GB/s against the measured HBM peak.

Workload (N = 1, the default): the 32^3x64 hybrid solve of the ND twisted-mass
doublet (kappa 0.16, mu_bar 0.1, eps_bar 0.11, antiperiodic time, seeded SU(3)
links with roughness 0.5), 12 shifts log-spaced in 1e-5..2, 8 Gaussian
right-hand sides, rho = 1e-10: mixed-precision multi-shift CG (FP32 arithmetic on
16-bit stencil data, all 8 right-hand sides in every stencil launch) for the 8
largest shifts, Lagrange guesses and case-C two-level multigrid (4^4 aggregates,
24 test vectors per chirality, coarse operator on the tensor cores) for the 4
smallest, every (shift, right-hand side) pair finished by FP64 defect correction
and certified by its FP64 true residual.  A step is one complete solve of the 96
systems (the multigrid setup is built once per gauge field, outside the timed
region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tmnd|reference]
                    [--form hybrid|fp64|mixed|batched|learned|rational]

--form selects a solver form on its own workload (every form certifies each shift
at 1e-10 by its FP64 true residual):
  hybrid   the headline above
  fp64     16^3x32, 12 shifts, 1 RHS: plain FP64 multi-shift CG (its oracle baseline is
           the oracle's full solve of the same system, timed)
  mixed    24^3x48, 12 shifts, 2 RHS one at a time: sloppy FP32/16-bit multi-shift
           CG + FP64 defect correction
  batched  32^3x64, 12 shifts, 8 RHS: the same with all 8 RHS in every 16-bit
           stencil launch, no multigrid
  learned  24^3x48, 12 shifts, 1 RHS on an unseen field: mixed multi-shift CG for
           the 8 largest, learned guesses for the 4 smallest finished by defect
           correction; the network is trained first on solves of other fields
           (outside the timed region); the same with Lagrange guesses is reported
  rational 24^3x48, 2 RHS: x = R(Qhat^2) b ~ (Qhat^2)^(-1/2) b with Zolotarev's n = 10
           approximation on the spectrum bounds from a Lanczos estimate (mixed
           multi-shift CG over the 10 Zolotarev shifts + one combination)
Each form's line also times the plain FP64 multi-shift CG on its workload
("fp64_same_workload") and reports the rooflines of its stencils.

--study errors runs App. A's comparison of equivalent solutions (methods A-F) on the
16^3x32 field against a known solution, rho = 1e-2 .. 1e-10.
--study learned runs config 5: train on solves of 20 fields, evaluate on 5 unseen
fields (CG iterations for the 4 smallest shifts from zero, Lagrange and learned guesses).
--study mg compares the case-C multigrid's smoothers and setups at small shifts (24^3x48).
--study hybrid measures the hybrid cost model of Sec. 4.3 on GB300 (24^3x48):
per-shift CG and MG times, their fits, the model's optimal n and the measured
hybrid time for every n, without and with Lagrange guesses.

--kernel fp64|s16|coarse times one kernel family alone (CUDA events, L2 flushed
between applications) and prints its achieved rate against the roofline:
  fp64    FP64 Qhat^2 + sigma (4 stencil launches), 16^3x32
  s16     16-bit Qhat^2 + sigma (4 stencil launches), 24^3x48 (1 and 8 RHS per launch)
          and 32^3x64 (1 and 8 RHS)
  f32     FP32-operator Qhat^2 + sigma (4 launches), 24^3x48 and 32^3x64
  coarse  coarse doublet operator, tensor cores and CUDA cores, 24^3x48 with 4^4
          aggregates and 24 vectors per chirality, 1 and 8 RHS

--impl reference times the FP64 CPU oracle (the only other implementation of
this method here) on the host cores, on a bounded sample of the same workload.
Under torchrun (N > 1) every rank solves its own right-hand sides (replicas: the
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

KAPPA, MU_BAR, EPS_BAR = 0.16, 0.1, 0.11
ROUGHNESS = 0.5
NSHIFT, SIG_LO, SIG_HI = 12, 1e-5, 2.0
RHO = 1e-10
METRIC = "shift-system solves/sec at rel. residual 1e-10; Dslash GB/s vs HBM peak"
L2_FLUSH_BYTES = 512 << 20         # > 129 MB L2

# 16^3x32 workload of the plain FP64 form (and of --kernel fp64, --study errors)
DIMS = (32, 16, 16, 16)            # T, X, Y, Z
GAUGE_SEED, RHS_SEED = 1002, 2032

# Algorithmic counts per odd site for ONE FP64 stencil launch (both flavours):
#   flops: 2 x 1320 (Wilson hop with spin projection, 8 directions) + 240 (A^-1 or A site term)
#   bytes (FP64, 18-real links): even launch 240 reals (in 48, links 144, out 48),
#   odd launch 288 reals (t 48, psi 48, links 144, out 48)
HOP_FLOP_PER_SITE = 2 * 1320 + 240
HOP_BYTES_PER_SITE = (240 + 288) / 2 * 8
# DRAM bytes of one odd-site FP64 stencil launch at 16^3x32, one ncu capture of this kernel
# (dram__bytes_read.sum + dram__bytes_write.sum: 132.87 MB + 9.04 MB)
FP64_ODD_LAUNCH_TRAFFIC = 132.866816e6 + 9.036288e6
FP64_TRAFFIC_VH = 65536
# 16-bit stencil, algorithmic bytes per odd site and right-hand side: even launch 200 (in 100,
# out 100) + 192 links, odd launch 300 (+ psi 100) + 192 links; a Qhat^2 + sigma is 2 even +
# 2 odd launches and the sigma term's 100; with R right-hand sides per launch the links
# (4 x 192) are read once: R (2 (200 + 300) + 100) + 4 x 192 bytes per odd site
S16_SPINOR_BYTES_PER_SITE = 2 * (200 + 300) + 100
# FP32 operator (FP32 planes, 18-real FP32 links), per odd site per Qhat^2 + sigma: even launch
# 192 + 8 x 72 + 192, odd launch + psi 192, the sigma term's 192
F32_Q2_BYTES_PER_SITE = 2 * ((192 + 576 + 192) + (192 + 192 + 576 + 192)) + 192
S16_LINK_BYTES_PER_SITE = 4 * 192
# DRAM bytes (read + write) of one 16-bit Qhat^2 + sigma, one ncu capture of its 4 launches:
# {(lattice V/2, RHS per launch): bytes}
# (the 8-RHS entry: the grid-stride variant the autotuner keeps there, 64 threads x 6 blocks per SM)
S16_Q2_TRAFFIC = {(331776, 1): (97.503232e6 + 3.967232e6) + (132.547840e6 + 8.404480e6)
                  + (97.519360e6 + 3.632896e6) + (169.893632e6 + 15.372288e6),
                  (1048576, 8): (3218.8e6 + 820.7e6) + (4144.8e6 + 821.5e6)
                  + (3223.5e6 + 816.4e6) + (4910.6e6 + 823.1e6)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_rhs_seed(rank: int, base: int = 2004, nrhs: int = 8) -> int:
    """Seed of rank `rank`'s right-hand sides: every replica solves its own systems
    (right-hand side k of the rank draws from seed + k)."""
    return base + 1000 * rank


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


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of this machine, else the fallback."""
    v = _peaks().get("hbm_gbs")
    return (float(v), "MEASURED_PEAKS.json hbm_gbs (measured)") if v else (6800.0, "fallback 6.8 TB/s")


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
        # nvidia-smi's start-up (NVML initialisation) stalls the GPU's work for a few hundred ms:
        # wait for its first sample, so that the start-up overlaps neither warm-up nor timing
        t0 = time.time()
        while self.p is not None and self.p.poll() is None and time.time() - t0 < 10:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.05)

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


def kernel_base_name(name):
    """A kernel's bare function name from a demangled signature, e.g.
    "void <unnamed>::k_hop_odd_s16<1, 3, 1, 128, 3>(Geom, ...)" -> "k_hop_odd_s16" (CUPTI writes
    the anonymous namespace as "(anonymous namespace)::" or "<unnamed>::")."""
    nm = name.replace("(anonymous namespace)::", "").replace("<unnamed>::", "")
    return nm.split("(")[0].split("<")[0].split(" ")[-1]


def count_kernels(fn, prefix=("k_",)):
    """Kernels of this library that one call of fn launches, counted from the CUDA
    activity trace of torch's profiler (CUPTI; kernels replayed inside CUDA graphs
    included), and their names.  None if the profiler is unavailable."""
    import torch
    try:
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
        n, names = 0, {}
        for ev in prof.events():
            dev = str(getattr(ev, "device_type", ""))
            base = kernel_base_name(ev.name or "")
            if "CUDA" in dev and any(base.startswith(p) for p in prefix):
                n += 1
                names[base] = names.get(base, 0) + 1
        return n, names
    except Exception as e:  # noqa: BLE001
        return None, {"error": str(e)[:200]}


def fp64_peak_measured():
    """FP64 throughput of this GPU measured in this run: cuBLAS DGEMM 8192^3 through torch
    (best of 5, CUDA events) -- the denominator of the FP64 stencil's roofline."""
    import torch
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    bm = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = a @ bm
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ bm
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, bm, c
    torch.cuda.empty_cache()
    return 2 * n ** 3 / (best / 1e3) / 1e12


def _median_ms(fn, flush, stream, reps):
    import torch
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


def s16_roofline(tm, g, flush, stream, nrhs=1, reps=20):
    """The 16-bit stencil of the sloppy solves: median CUDA-event time of one 16-bit
    Qhat^2 + sigma (its 4 stencil launches, nrhs right-hand sides per launch, as the
    solve launches them) on the form's lattice, L2 flushed, against the HBM peak."""
    import torch
    src = g.pack(torch.randn(nrhs * g.vh * 24, dtype=torch.complex128, device="cuda").view(nrhs, g.vh, 2, 4, 3),
                 nrhs=nrhs)
    q = g.convert(src, tm.TMND_F64, tm.TMND_S16, nrhs=nrhs)
    del src
    o = g.spinor(nrhs, prec=tm.TMND_S16)
    ms = _median_ms(lambda: tm.tm_nd_apply(g.handle, o, q, tm.OP_QHAT2 | tm.OP_S16, 0.01, nrhs=nrhs, stream=stream),
                    flush, stream, reps)
    peak, src_peak = hbm_peak()
    byts = g.vh * (nrhs * S16_SPINOR_BYTES_PER_SITE + S16_LINK_BYTES_PER_SITE)
    gbs = byts / (ms / 1e3) / 1e9
    tr = None
    note = "no ncu capture of this launch shape"
    for (vh, r), t in S16_Q2_TRAFFIC.items():
        if r == nrhs:
            tr = t * g.vh / vh
            note = (f"DRAM bytes of one Qhat^2 from an ncu capture of its 4 launches at V/2 = {vh}, {r} RHS per launch"
                    + (", scaled by the number of sites" if vh != g.vh else ""))
            break
    del q, o
    return {"bound": "hbm", "kernel": f"k_hop_even_s16/k_hop_odd_s16 (16-bit stencil, Qhat^2 + sigma: 4 launches, "
                                      f"{nrhs} RHS per launch)",
            "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "traffic": tr,
            "traffic_note": note, "algorithmic_bytes": byts, "peak_source": src_peak,
            "measured": f"median of {reps} CUDA-event timings of tm_nd_apply(Qhat^2 + sigma, 16-bit), L2 flushed",
            "ms_per_qhat2": ms, "nrhs": nrhs}


def fp64_roofline(tm, g, flush, stream, peak_tflops, reps=10):
    """The FP64 stencil of the true residuals and defect corrections: median CUDA-event
    time of one FP64 Qhat^2 + sigma (4 launches, 1 RHS) on the form's lattice, against
    the FP64 throughput measured in this run (FP64-pipe bound on GB300)."""
    import torch
    x = g.pack(torch.randn(g.vh * 24, dtype=torch.complex128, device="cuda").view(1, g.vh, 2, 4, 3))
    y = g.spinor()
    ms = _median_ms(lambda: tm.tm_nd_apply(g.handle, y, x, tm.OP_QHAT2, 0.01, stream=stream), flush, stream, reps)
    tf = 4 * HOP_FLOP_PER_SITE * g.vh / (ms / 1e3) / 1e12
    del x, y
    return {"bound": "alu", "kernel": "k_hop_even/k_hop_odd (FP64 stencil, Qhat^2 + sigma: 4 launches)",
            "achieved": tf, "peak": peak_tflops, "unit": "TFLOP/s", "frac": tf / peak_tflops,
            "traffic": FP64_ODD_LAUNCH_TRAFFIC * g.vh / FP64_TRAFFIC_VH,
            "traffic_note": "DRAM bytes of one odd-site launch from an ncu capture at 16^3x32, scaled by the "
                            "number of sites",
            "peak_source": "cuBLAS DGEMM 8192^3 (torch, best of 5) measured in this run",
            "algorithmic_flop_per_launch": HOP_FLOP_PER_SITE * g.vh,
            "measured": f"median of {reps} CUDA-event timings of tm_nd_apply(Qhat^2 + sigma, FP64), L2 flushed",
            "ms_per_qhat2": ms, "gbs": 4 * HOP_BYTES_PER_SITE * g.vh / (ms / 1e3) / 1e9}


FORMS = {
    "fp64": dict(dims=(32, 16, 16, 16), nrhs=1, seeds=(1002, 2032), lattice="16^3x32", batch=1),
    "mixed": dict(dims=(48, 24, 24, 24), nrhs=2, seeds=(1003, 2003), lattice="24^3x48", batch=1),
    "batched": dict(dims=(64, 32, 32, 32), nrhs=8, seeds=(1004, 2004), lattice="32^3x64", batch=8),
    "hybrid": dict(dims=(64, 32, 32, 32), nrhs=8, seeds=(1004, 2004), lattice="32^3x64", batch=8),
    "learned": dict(dims=(48, 24, 24, 24), nrhs=1, seeds=(1005, 2005), lattice="24^3x48", batch=1),
    "rational": dict(dims=(48, 24, 24, 24), nrhs=2, seeds=(1003, 2003), lattice="24^3x48", batch=2),
}
# the multigrid of the hybrid form: 4^4 aggregates, 24 test vectors per chirality relaxed by
# 4 minimal-residual steps on D_TM(mu_bar) x = 0
MG_BLOCK, MG_NV, MG_RELAX = (4, 4, 4, 4), 24, 4
N_MMS = 8


def workload_name(form, F, nrhs):
    desc = {
        "fp64": "plain FP64 multi-shift CG",
        "mixed": "mixed-precision multi-shift CG (FP32 on 16-bit data + FP64 defect correction), RHS one at a time",
        "batched": "mixed-precision multi-shift CG with all RHS in every 16-bit stencil launch + batched FP64 "
                   "defect correction",
        "hybrid": "hybrid solve: batched mixed multi-shift CG for the 8 largest shifts, Lagrange guesses for the "
                  "4 smallest, batched FP64 defect correction of every shift; case-C two-level multigrid (4^4 "
                  "aggregates, 24 vectors per chirality, tensor-core coarse operator) set up and entered for a shift "
                  "whose guess residual exceeds 1e-4 (none at this workload: mg_iters in the line)",
        "learned": "mixed multi-shift CG for the 8 largest shifts, learned guesses for the 4 smallest",
        "rational": "Zolotarev n = 10 rational approximation of (Qhat^2)^(-1/2) over a mixed multi-shift solve",
    }[form]
    shifts = "Zolotarev shifts" if form == "rational" else "12 shifts 1e-5..2"
    return f"{F['lattice']} ND twisted-mass doublet, {desc}, {shifts}, {nrhs} RHS, rho 1e-10"


def _timed(step, steps, flush, stream, nvtx=None, per_step=None):
    """CUDA-event time of `steps` calls of step (L2 flushed before each); each call inside an
    NVTX range named `nvtx` if given (profilers can select the timed steps by it).  With a
    list `per_step`, it receives each step's own event time (ms, flush included)."""
    import torch
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    out = []
    ev[0].record(stream)
    for i in range(steps):
        flush.fill_(1.0)
        if nvtx:
            torch.cuda.nvtx.range_push(nvtx)
        out.append(step())
        if nvtx:
            torch.cuda.nvtx.range_pop()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    if per_step is not None:
        per_step.extend(ev[i].elapsed_time(ev[i + 1]) for i in range(steps))
    return ev[0].elapsed_time(ev[steps]), out


def run_form(args):
    """One solver form on its own workload (see the module docstring); the default form,
    hybrid, is the headline.  Under torchrun every rank solves its own right-hand sides."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1805_09584_gb300 as tm
    import synth
    from paper_1805_09584_gb300 import _build, learned

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    _build.build()
    F = FORMS[args.form]
    dims, nrhs = F["dims"], F["nrhs"]
    gseed, bseed = F["seeds"]
    sig = synth.shift_set(NSHIFT, SIG_LO, SIG_HI)
    U = synth.random_su3_field(dims, ROUGHNESS, gseed)
    g = tm.Gauge(U, dims, KAPPA, MU_BAR, EPS_BAR)
    del U
    stream = torch.cuda.current_stream()
    b_host = synth.gaussian_rhs(dims, bseed if ws == 1 else replica_rhs_seed(rank, bseed, nrhs), nrhs=nrhs)
    b_dev = g.pack(torch.from_numpy(b_host).cuda(), nrhs=nrhs)
    xs = [g.spinor(nrhs) for _ in sig]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    extra = {}
    mg = net = None
    if args.form != "fp64":
        # launch shapes of the 16-bit stencil for every batch size a solve may launch (1..16
        # right-hand sides), tuned here so that no timed step pays for it
        t0 = time.perf_counter()
        per = {}
        for R in range(1, tm.TMND_MAX_BATCH + 1):
            sh, tms = tm.tmnd_autotune(g.handle, R, stream)
            shm, tmm = tm.tmnd_autotune_mms(g.handle, R, stream)
            per[R] = {"shape": sh, "ms": [round(float(v), 4) for v in tms],
                      "shape_mms": shm, "ms_mms": [round(float(v), 4) for v in tmm]}
        extra["autotune"] = {"shapes": [tm.tmnd_s16_shape_info(i) for i in range(tm.S16_SHAPES)],
                             "shape_fields": ["threads per block", "blocks per SM", "next-direction prefetch",
                                              "loop order (0 chunk, sites outside; 1 chunk, RHS outside; "
                                              "2 grid stride, sites outside; 3 grid stride over (32-site group, RHS) per warp)"],
                             "per_nrhs": per, "s": time.perf_counter() - t0}
    if args.form == "hybrid":
        t0 = time.perf_counter()
        tv = torch.randn(MG_NV * 2 * 12 * g.vh, dtype=torch.complex64, device="cuda")
        tm.tmnd_mg_smooth_vectors(g.handle, tv, MG_NV, MG_RELAX)
        mg = tm.tmnd_mg_create(g.handle, MG_BLOCK, MG_NV, tv)
        torch.cuda.synchronize()
        extra["mg_setup_s"] = time.perf_counter() - t0
        del tv
    if args.form == "learned":
        t0 = time.perf_counter()
        Xs, Ss, Hs = [], [], []
        for fs in range(4):   # training fields (roughness 0.3..0.6), 2 RHS each
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
        if args.form == "fp64":
            return tm.mms_cg_solve(g.handle, b_dev, nrhs, sig, xs, rho=RHO, stream=stream)
        if args.form == "rational":
            return tm.tmnd_rational_apply(g.handle, b_dev, nrhs, 10, lmin, lmax, out_r, rho=RHO, prec=tm.TMND_S16,
                                          stream=stream)
        if args.form in ("mixed", "batched"):
            return tm.mms_cg_solve(g.handle, b_dev, nrhs, sig, xs, rho=RHO, prec=tm.TMND_S16,
                                   batch=F["batch"], stream=stream)
        if args.form == "hybrid":
            return tm.tmnd_hybrid_solve(g.handle, mg, b_dev, nrhs, sig, N_MMS, xs, rho=RHO, prec=tm.TMND_S16,
                                        n_guess=0, guess=1, stream=stream)
        return tm.tmnd_hybrid_solve(g.handle, None, b_dev, nrhs, sig, N_MMS, xs, rho=RHO, prec=tm.TMND_S16,
                                    n_guess=0, guess=2, net=net, stream=stream)

    # nvidia-smi starts before the warm-up, so that its start-up does not overlap the timed region
    sampler = ClockSampler(local)
    for _ in range(args.warmup):
        step()
    if ws > 1:
        dist.barrier()
    step_ms = []
    ms, infos = _timed(step, args.steps, flush, stream, nvtx="timed_step", per_step=step_ms)
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms_all = max_over_ranks(ms, ws)
    solves = args.steps * len(sig) * nrhs
    value = whole_job_rate(args.steps * len(sig) * nrhs, ws, ms_all)
    worst = max(max(i["true_res"]) for i in infos)
    if args.form == "learned":   # the same with Lagrange guesses (the method without the network)
        def step_lag():
            return tm.tmnd_hybrid_solve(g.handle, None, b_dev, nrhs, sig, N_MMS, xs, rho=RHO, prec=tm.TMND_S16,
                                        n_guess=0, guess=1, stream=stream)
        step_lag()
        ms_l, inf_l = _timed(step_lag, args.steps, flush, stream)
        extra["lagrange_guesses"] = {"value": solves / (ms_l / 1e3), "ms_per_step": ms_l / args.steps,
                                     "guess_res": inf_l[-1]["guess_res"][8:],
                                     "refine_iters": inf_l[-1]["refine_iters"],
                                     "fp64_applies": inf_l[-1]["fp64_applies"]}
        extra["learned_guesses"] = {"guess_res": infos[-1]["guess_res"][8:], "refine_iters": infos[-1]["refine_iters"],
                                    "fp64_applies": infos[-1]["fp64_applies"]}
    if args.form == "batched":   # the same solve one RHS at a time (batching's gain): the multi-shift
        # solve of each RHS alone, its defect corrections batched over its own 12 shifts only
        def step_one():
            return tm.mms_cg_solve(g.handle, b_dev, nrhs, sig, xs, rho=RHO, prec=tm.TMND_S16, batch=1,
                                   stream=stream)
        step_one()
        ms_1, _ = _timed(step_one, 1, flush, stream)
        extra["one_rhs_at_a_time"] = {"value": len(sig) * nrhs / (ms_1 / 1e3), "ms_per_step": ms_1}
    # solver statistics of the last timed step
    last = infos[-1]
    stats = {k: last[k] for k in ("iters", "mms_iters", "refine_iters", "fp64_applies", "f32_applies",
                                  "refine_rounds", "mg_iters", "guess_res", "lag_nodes", "phase_ms", "mms_ms",
                                  "shift_ms") if k in last}
    # e2e: host buffers in and out through the public API: the canonical right-hand sides
    # from pinned host memory, packed, solved, and every shift's solutions unpacked and read
    # back into pinned host memory (one buffer, reused shift by shift)
    e2e_steps = min(args.steps, 3)
    outs = [out_r] if args.form == "rational" else xs
    b_pin = torch.from_numpy(b_host).pin_memory()
    x_pin = torch.empty((nrhs, g.vh, 2, 4, 3), dtype=torch.complex128).pin_memory()
    b_can = torch.empty((nrhs, g.vh, 2, 4, 3), dtype=torch.complex128, device="cuda")
    x_can = torch.empty((nrhs, g.vh, 2, 4, 3), dtype=torch.complex128, device="cuda")

    def step_e2e():
        b_can.copy_(b_pin, non_blocking=True)
        tm.tmnd_spinor_pack(g.handle, b_dev, b_can, nrhs, stream)
        r = step()
        for v in outs:
            tm.tmnd_spinor_unpack(g.handle, x_can, v, nrhs, stream)
            x_pin.copy_(x_can, non_blocking=True)
        return r
    if ws > 1:
        dist.barrier()
    e2e_ms, _ = _timed(step_e2e, e2e_steps, flush, stream)
    e2e_all = max_over_ranks(e2e_ms, ws)
    del b_pin, x_pin, b_can, x_can
    # kernels launched per step (torch profiler's CUDA activity trace of one more step)
    nk, knames = count_kernels(step)
    # the plain FP64 multi-shift CG on the same workload (one step), and each form's solutions
    # against its solutions: max over shifts of |x_form - x_FP64| / |x_FP64| (all RHS together)
    if args.form != "fp64":
        keep = [v.clone() for v in xs[:len(sig)]] if args.form != "rational" else None
        f64 = lambda: tm.mms_cg_solve(g.handle, b_dev, nrhs, sig, xs[:len(sig)], rho=RHO, stream=stream)
        f64()
        f64_ms, f64_inf = _timed(f64, 1, flush, stream)
        extra["fp64_same_workload"] = {"value": nrhs * len(sig) / (f64_ms / 1e3), "ms_per_step": f64_ms,
                                       "iters": f64_inf[0]["iters"]}
        if keep is not None:
            dx = [float(torch.linalg.vector_norm(k - v) / torch.linalg.vector_norm(v)) for k, v in zip(keep, xs)]
            extra["rel_diff_vs_fp64"] = {"max": max(dx), "per_shift": [float("%.3g" % d) for d in dx]}
            del keep
    # rooflines of the two stencils on this lattice
    fp64_peak = fp64_peak_measured()
    roof = s16_roofline(tm, g, flush, stream, nrhs=F["batch"])
    roof64 = fp64_roofline(tm, g, flush, stream, fp64_peak)
    if mg is not None:   # the coarse operator on the tensor cores, all RHS at once
        nb = g.vh * 2 // 256
        xc = torch.randn(nrhs * nb * 4 * MG_NV, dtype=torch.complex64, device="cuda")
        yc = torch.empty_like(xc)
        c_ms = _median_ms(lambda: tm.mg_coarse_apply(mg, yc, xc, nrhs, 0.0, stream=stream), flush, stream, 10)
        byts = nb * 9 * (2 * MG_NV) ** 2 * 8 + 2 * nrhs * nb * 4 * MG_NV * 8
        extra["coarse_tc"] = {"ms": c_ms, "GBs": byts / (c_ms / 1e3) / 1e9, "nrhs": nrhs,
                              "frac_hbm": byts / (c_ms / 1e3) / 1e9 / hbm_peak()[0],
                              "kernel": "k_coarse_apply_tc (tcgen05 TF32, 48x48 blocks)"}
    launches_claim = nk * args.steps if nk else (sum(i.get("launches", 0) for i in infos) or None)
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if args.form == "fp64" else "f32 (16-bit storage) + f64 (true residuals, defect correction)",
            "data": "synthetic",
            "config": {"workload": workload_name(args.form, F, nrhs), "form": args.form, "lattice": F["lattice"],
                       "nshift": len(sig), "nrhs": nrhs, "rho": RHO, "kappa": KAPPA, "mu_bar": MU_BAR,
                       "eps_bar": EPS_BAR, "roughness": ROUGHNESS,
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "flushed between steps (512 MB write); solve working set > L2"},
            "max_true_rel_residual": worst,
            "step_ms": [round(v, 3) for v in step_ms],
            "e2e": {"value": whole_job_rate(e2e_steps * len(sig) * nrhs, ws, e2e_all), "unit": "solves/s",
                    "h2d_bytes_per_step": b_host.nbytes, "d2h_bytes_per_step": len(outs) * b_host.nbytes,
                    "steps": e2e_steps},
            "roofline": roof, "roofline_fp64": roof64, "solver": stats,
            "gpu_launches": launches_claim,
            "gpu_launches_note": ("kernels per step counted from torch.profiler's CUDA activity trace of one "
                                  "step, times the timed steps" if nk else "the library's own launch count"),
            **({"kernels_per_step": knames} if knames else {}), "clocks": clocks, **extra,
        }
    if net is not None:
        tm.tmnd_mlp_destroy(net)
    if mg is not None:
        tm.tmnd_mg_destroy(mg)
    g.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
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

    def timed(fn, nvtx=None):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if nvtx:   # profilers can select the timed applications by this range
                torch.cuda.nvtx.range_push(nvtx)
            e0.record(stream)
            fn()
            e1.record(stream)
            if nvtx:
                torch.cuda.nvtx.range_pop()
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
    elif args.kernel == "f32":
        for dims, name in (((48, 24, 24, 24), "24^3x48"), ((64, 32, 32, 32), "32^3x64")):
            g = tm.Gauge(synth.random_su3_field(dims, ROUGHNESS, 1003), dims, KAPPA, MU_BAR, EPS_BAR)
            b = g.pack(torch.from_numpy(synth.gaussian_rhs(dims, 2003)).cuda())
            q = g.convert(b, tm.TMND_F64, tm.TMND_F32)
            o = g.spinor(prec=tm.TMND_F32)
            del b
            ms = timed(lambda: tm.tm_nd_apply(g.handle, o, q, tm.OP_QHAT2 | tm.OP_F32, 0.01, stream=stream))
            byts = g.vh * F32_Q2_BYTES_PER_SITE
            out[f"{name}"] = {"ms_qhat2": ms, "gbs": byts / (ms / 1e3) / 1e9,
                              "frac_hbm": byts / (ms / 1e3) / 1e9 / peak_hbm,
                              "tflops": 4 * HOP_FLOP_PER_SITE * g.vh / (ms / 1e3) / 1e12}
            del q, o
            g.close()
        out.update(hbm_peak_gbs=peak_hbm, bytes_per_site=F32_Q2_BYTES_PER_SITE)
        return out
    elif args.kernel == "s16":
        tm.tmnd_s16_force_shape(args.variant)  # -1: the autotuner's choice
        out.update(forced_variant=args.variant if args.variant >= 0 else None)
        for dims, name, rs in (((48, 24, 24, 24), "24^3x48", (1, 8)), ((64, 32, 32, 32), "32^3x64", (1, 8))):
            g = tm.Gauge(synth.random_su3_field(dims, ROUGHNESS, 1003), dims, KAPPA, MU_BAR, EPS_BAR)
            for R in rs:
                b = g.pack(torch.from_numpy(synth.gaussian_rhs(dims, 2003, nrhs=R)).cuda(), nrhs=R)
                q = g.convert(b, tm.TMND_F64, tm.TMND_S16, nrhs=R)
                o = g.spinor(R, prec=tm.TMND_S16)
                del b
                ms = timed(lambda: tm.tm_nd_apply(g.handle, o, q, tm.OP_QHAT2 | tm.OP_S16, 0.01, nrhs=R,
                                                  stream=stream), nvtx=f"s16_{name.replace('^', '')}_nrhs{R}")
                # links are read once per launch for all R right-hand sides
                byts = g.vh * (R * (2 * (200 + 300) + 100) + 4 * 192)
                sh, tms = tm.tmnd_autotune(g.handle, R, stream)
                if args.variant >= 0:
                    sh = args.variant
                out[f"{name}_nrhs{R}"] = {"ms_qhat2": ms, "ms_per_rhs": ms / R, "gbs": byts / (ms / 1e3) / 1e9,
                                          "frac_hbm": byts / (ms / 1e3) / 1e9 / peak_hbm, "variant": sh,
                                          "variant_ms": [round(float(v), 4) for v in tms]}
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



def run_study_mg(args):
    """Case-C multigrid at small shifts (Sec. 3: DD-alphaAMG smooths with SAP and builds its
    prolongator adaptively), 24^3x48, 4^4 aggregates, 24 test vectors per chirality: for
    s^2 = sigma in (0.07, 7.8e-3, 2.8e-4, 1e-5) the outer iterations and the time to reach
    1e-4 from a zero start (at most 100 outer iterations, GCR(24), 2 smoothing steps) of
    D_ND + i s gamma_5 tau_1 Pi_odd on a Gaussian full-lattice right-hand side, for minimal-
    residual smoothing (test vectors relaxed by 4 MR steps), SAP smoothing with the same
    vectors, and SAP after one round of adaptive setup; next to the mixed CG on the same shift.
    With --kappa k1 k2 ..., the same for each hopping parameter (the spectrum of Qhat^2 moves
    with kappa: the Wilson hops and the twisted-mass terms 2 kappa mu_bar, 2 kappa eps_bar all
    scale with it), SAP after the adaptive setup only, with the extreme Ritz values of Qhat^2
    from an FP64 CG history."""
    import numpy as np
    import torch

    import paper_1805_09584_gb300 as tm
    import synth
    from paper_1805_09584_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    dims = (48, 24, 24, 24)
    nv, blk = 24, (4, 4, 4, 4)
    kappas = args.kappa or [KAPPA]
    out = {"study": "case-C multigrid at small shifts (SAP, adaptive setup)", "lattice": "24^3x48",
           "aggregates": "4^4", "test_vectors": nv,
           "solve": "GCR(24), 2 pre/post smoothing steps, tol 1e-4, at most 100 outer iterations, zero start, "
                    "Gaussian full-lattice right-hand side", "per_kappa": []}
    for kappa in kappas:
        g = tm.Gauge(synth.random_su3_field(dims, ROUGHNESS, 1003), dims, kappa, MU_BAR, EPS_BAR)
        gen = torch.Generator(device="cuda").manual_seed(7)
        tv = torch.randn(nv * 2 * 12 * g.vh, dtype=torch.complex64, device="cuda", generator=gen)
        tm.tmnd_mg_smooth_vectors(g.handle, tv, nv, 4)
        t0 = time.perf_counter()
        mg_mr = tm.tmnd_mg_create(g.handle, blk, nv, tv) if not args.kappa else None
        mg_sap = tm.tmnd_mg_create(g.handle, blk, nv, tv, smoother=1)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        mg_boot = tm.tmnd_mg_bootstrap(mg_sap, tv, 3, blk, nv, smoother=1)
        torch.cuda.synchronize()
        t_boot = time.perf_counter() - t0
        del tv
        rhs = torch.randn(2 * 24 * g.vh, dtype=torch.complex64, device="cuda", generator=gen)
        b_odd = g.pack(torch.from_numpy(synth.gaussian_rhs(dims, 2003)).cuda())
        variants = (("mr", mg_mr), ("sap", mg_sap), ("sap_bootstrap", mg_boot)) if not args.kappa else \
            (("sap_bootstrap", mg_boot),)
        rows = []
        for sigma in (0.07, 7.8e-3, 2.8e-4, 1e-5):
            s = float(sigma) ** 0.5
            row = {"sigma": sigma}
            for name, mg in variants:
                x = torch.zeros_like(rhs)
                torch.cuda.synchronize()
                t = time.perf_counter()
                info = tm.tmnd_mg_solve(mg, x, rhs, s, tol=1e-4, maxiter=100, restart=24, nu=2)
                torch.cuda.synchronize()
                row[name] = {"iters": info["iters"], "res": info["res"], "s": time.perf_counter() - t}
            xs = [g.spinor()]
            torch.cuda.synchronize()
            t = time.perf_counter()
            inf = tm.mms_cg_solve(g.handle, b_odd, 1, [sigma], xs, rho=1e-10, prec=tm.TMND_S16)
            torch.cuda.synchronize()
            row["mixed_cg_1e-10"] = {"iters": inf["iters"] + inf["refine_iters"], "s": time.perf_counter() - t}
            rows.append(row)
        # extreme Ritz values of Qhat^2 (FP64 CG history at the smallest shift)
        hist = np.zeros(2 * 8192)
        xb = [g.spinor()]
        inf = tm.mms_cg_solve(g.handle, b_odd, 1, [1e-5], xb, rho=1e-8, ab_hist=hist)
        sg = synth.shift_set(NSHIFT, SIG_LO, SIG_HI)
        f = tm.tmnd_mlp_features(sg[:8], float(sg[8]), hist, inf["iters"], 1e-5)
        rec = {"kappa": kappa, "setup_s": t_setup, "bootstrap_s": t_boot, "rows": rows,
               "ritz_min_max": [10 ** float(f[17]), 10 ** float(f[18])], "fp64_cg_iters_1e-8": inf["iters"]}
        out["per_kappa"].append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
        for mg in (mg_boot, mg_sap, mg_mr):
            if mg is not None:
                tm.tmnd_mg_destroy(mg)
        del xs, xb, b_odd, rhs
        g.close()
    if not args.kappa:   # the single-kappa study's original layout
        rec = out.pop("per_kappa")[0]
        out.update(setup_s=rec["setup_s"], bootstrap_s=rec["bootstrap_s"], rows=rec["rows"],
                   ritz_min_max=rec["ritz_min_max"])
    return out


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




# nominal FP64 rate of a GB300 (sm_103a): 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz;
# the headline's FP64 roofline uses the DGEMM rate measured in the run instead
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def oracle_full_iters(name):
    """The oracle's own iteration count for a workload (tests/golden/make_golden.py)."""
    p = os.path.join(ROOT, "tests", "golden", name + ".json")
    try:
        with open(p) as f:
            return int(json.load(f)["iters"])
    except (OSError, KeyError, ValueError):
        return None


GOLDEN = {"fp64": "mms_16x16x16x32", "hybrid": "mms_32x32x32x64", "batched": "mms_32x32x32x64"}


def _oracle_inputs(form):
    import oracle
    import synth
    F = FORMS[form]
    dims = F["dims"]
    U = synth.random_su3_field(dims, ROUGHNESS, F["seeds"][0])
    b = synth.gaussian_rhs(dims, F["seeds"][1], nrhs=F["nrhs"])[0]
    act = oracle.action(dims, KAPPA, MU_BAR, EPS_BAR)
    return oracle, U, b, synth.shift_set(NSHIFT, SIG_LO, SIG_HI), act


def cpu_baseline(form, sample_iters=3):
    """The oracle, as it stands, on the host cores (all of them: OpenMP over sites).
    fp64 form: the oracle's complete 12-shift solve of the same system, timed.
    32^3x64 forms: one right-hand side, a bounded sample -- the solve's set-up alone
    (maxiter 0) and `sample_iters` iterations -- scaled to the oracle's own iteration
    count for that system (tests/golden) and to the workload's 8 right-hand sides."""
    oracle, U, b, sig, act = _oracle_inputs(form)
    nrhs = FORMS[form]["nrhs"]
    if form == "fp64":
        t = time.perf_counter()
        res = oracle.mms_cg(act, U, b, sig, rho=RHO)
        el = time.perf_counter() - t
        return {"value": NSHIFT / el, "unit": "solves/s", "cores": oracle.nthreads(), "kind": "oracle",
                "sample": f"the oracle's complete 16^3x32 12-shift solve ({res['iters']} iterations, {el:.1f} s)"}
    iters_full = oracle_full_iters(GOLDEN[form])
    if iters_full is None:
        return {"value": None, "unavailable": "the oracle's iteration count for this workload is not recorded"}
    t = time.perf_counter()
    oracle.mms_cg(act, U, b, sig, rho=RHO, maxiter=0)
    t_setup = time.perf_counter() - t
    t = time.perf_counter()
    oracle.mms_cg(act, U, b, sig, rho=RHO, maxiter=sample_iters)
    t_k = time.perf_counter() - t
    per_iter = max(t_k - t_setup, 1e-9) / sample_iters
    full = t_setup + iters_full * per_iter
    return {"value": NSHIFT * nrhs / (nrhs * full), "unit": "solves/s", "cores": oracle.nthreads(), "kind": "oracle",
            "sample": f"1 of the {nrhs} right-hand sides: the oracle's set-up ({t_setup:.1f} s) and {sample_iters} "
                      f"multi-shift CG iterations ({t_k:.1f} s with set-up) of its 12-shift FP64 solve, scaled to "
                      f"the oracle's {iters_full}-iteration solve of that system and to {nrhs} right-hand sides",
            "projected_s_per_step": nrhs * full}


def run_reference(args, form=None):
    """--impl reference: the FP64 oracle on the host cores, on the default form's workload
    (rank 0 only).  Each step is one call of the oracle's multi-shift CG on one of the
    right-hand sides, stopped after one iteration; the warm-up steps time the solve's
    set-up alone (maxiter 0).  The value scales the median step to the oracle's full
    iteration count for that system and to all right-hand sides of the workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    form = form or args.form
    if form not in GOLDEN:
        form = "hybrid"
    iters_full = oracle_full_iters(GOLDEN[form])
    if iters_full is None:
        return {"impl": "reference", "unavailable": "oracle iteration count for the workload not recorded"}
    oracle, U, b, sig, act = _oracle_inputs(form)
    F = FORMS[form]
    nrhs = F["nrhs"]
    setup = []
    for _ in range(max(args.warmup, 1)):
        t = time.perf_counter()
        oracle.mms_cg(act, U, b, sig, rho=RHO, maxiter=0)
        setup.append(time.perf_counter() - t)
    steps = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.mms_cg(act, U, b, sig, rho=RHO, maxiter=1)
        steps.append(time.perf_counter() - t)
    el = time.perf_counter() - t_all
    t_setup = statistics.median(setup)
    per_iter = max(statistics.median(steps) - t_setup, 1e-9)
    full = t_setup + iters_full * per_iter          # one right-hand side, seconds
    value = NSHIFT / full
    sample = (f"each step: one oracle multi-shift CG call on 1 of the {nrhs} right-hand sides, stopped after 1 "
              f"iteration (median {statistics.median(steps):.2f} s; set-up alone {t_setup:.2f} s), scaled to the "
              f"oracle's {iters_full}-iteration solve of that system; value = {NSHIFT * nrhs} solves / "
              f"({nrhs} x that time)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / max(args.steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(form, F, nrhs), "form": form, "lattice": F["lattice"],
                       "nshift": NSHIFT, "nrhs": nrhs, "rho": RHO},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": oracle.nthreads(), "kind": "oracle",
                             "sample": sample},
            "projected_s_per_workload": nrhs * full,
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tmnd", choices=["tmnd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="hybrid", choices=list(FORMS))
    ap.add_argument("--kernel", default=None, choices=["fp64", "s16", "f32", "coarse"])
    ap.add_argument("--variant", type=int, default=-1,
                    help="--kernel s16: time this launch variant of the 16-bit stencil (tmnd_s16_force_shape) "
                         "instead of the autotuner's choice")
    ap.add_argument("--study", default=None, choices=["hybrid", "learned", "errors", "mg"])
    ap.add_argument("--kappa", type=float, nargs="+", default=None,
                    help="--study mg: hopping parameters to run the study at (default: the configs' kappa)")
    args = ap.parse_args()
    if args.study:
        fn = {"hybrid": run_study, "learned": run_study_learned, "errors": run_study_errors,
              "mg": run_study_mg}[args.study]
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
    out = run_form(args)
    ws, rank, _ = _dist()
    if rank == 0 and out is not None:
        if args.form == "fp64":
            out["roofline"], out["roofline_s16"] = out.pop("roofline_fp64"), out.pop("roofline")
        if ws == 1 and not args.no_cpu_baseline and args.form in GOLDEN:
            out["cpu_baseline"] = cpu_baseline(args.form)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
