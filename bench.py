"""Benchmark of the time-domain BEM hot path on one GB300.

One "step" is one marching-on-in-time step (Eq. linear): the history sum
that forms b^{a-1} over every stored element pair and lag, the incident-wave
term, and the zero-lag solve.  The workload is the seeded synthetic
scattering problem with Ns = 20480: a sound-hard ellipsoid (icosphere
subdivision 5 mapped by axes ~ U[0.5, 1.5], seed 3), Burton-Miller BIE,
B-spline order d = 2, c dt = 0.5 x mean edge, Gaussian plane pulse (sigma =
0.3, seeded direction).  The path is the direct (all-pairs) FP64 history
sum; the space-time FMM is not built yet, so the workload name says
"direct".

Before the W warm-up steps the run marches gamma_max steps untimed, so that
every timed step uses the full lag window of every pair (steady state).
The coefficient stream (~14 GB) is far larger than the 129 MB L2, so no
flush is needed between steps.

Output: one JSON line (see the keys below).  ``--impl reference`` times the
FP64 CPU oracle on a bounded sample of the same workload instead.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ellipsoid20480_bmbie_d2_hard_plane"
METRIC = "time-steps/sec FMM-TDBEM Ns=20480 (mixed vs FP64 form, ≤1e-3 rel L2); M2L TC util"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for k, n in enumerate(names):
                    if r[3 + k].lower().startswith("active"):
                        reasons.add(n)
            except Exception:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _excitation(w, xc, n, alphas):
    """Host-side excitation e_i(t_a) of the sound-hard Burton-Miller problem:
    (d/dn_x - c^-1 d/dt) of the Gaussian plane pulse, the caller's input in
    the end-to-end measurement."""
    k = np.asarray(w.direction, dtype=np.float64)
    kx = xc @ k
    kn = n @ k
    out = np.empty((len(alphas), len(xc)))
    for r, a in enumerate(alphas):
        s = (a * w.dt - w.t0 - kx / w.c) / w.sigma
        df = -2.0 * s / w.sigma * np.exp(-s * s)
        out[r] = -(1.0 + kn) / w.c * df
    return out


def _geometry(w):
    v = w.xyz[w.tri]
    xc = (v[:, 0] + v[:, 1] + v[:, 2]) / 3.0
    g = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    return xc, -g / np.linalg.norm(g, axis=1, keepdims=True)


def _unknown(s, w, n):
    u, q = s.solution(0, n)
    return u if w.bc == "neumann" else q


def _timed(abi, torch, ctx, nsteps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    abi.tdbem_step(ctx, nsteps)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def max_over_ranks(ms, dist, device):
    """The slowest rank's time: the whole job is done only when every rank
    is (dist = torch.distributed, or None for one process)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch
    from paper_2111_05205_gb300 import Solver, abi, build
    from synth import workload

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()

    w = workload(args.workload)
    fmm = args.algo == "fmm"
    spin = 260  # untimed steps before the warm-up: every lag window in use
    need = spin + 2 * (args.warmup + args.steps) + 2
    w.nt = max(w.nt, need)
    stream = torch.cuda.current_stream().cuda_stream
    phi = np.full(w.ns, 1 if w.bc == "neumann" else 0, np.int8)
    inc = (w.direction, w.t0, w.sigma)

    def make(precision, algo_fmm):
        kw = dict(depth=args.depth, fmm=(args.ps, args.pt, 0)) if algo_fmm else {}
        return Solver(w.xyz, w.tri, w.c, w.dt, w.nt, w.d, w.bie, phi=phi, incident=inc, stream=stream,
                      precision=precision, **kw)

    t0 = time.time()
    s = make(args.precision, fmm)
    setup_s = time.time() - t0
    st0 = s.stats()
    gmax = st0["gamma_max"]
    ctx = s.ctx
    abi.tdbem_step(ctx, spin)
    abi.tdbem_step(ctx, args.warmup)
    abi.tdbem_sync(ctx)
    abi.tdbem_reset_stats(ctx)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        ms = _timed(abi, torch, ctx, args.steps)
        torch.cuda.nvtx.range_pop()
    if dist is not None:
        dist.barrier()
    st = s.stats()
    abi.tdbem_sync(ctx)
    ms = max_over_ranks(ms, dist, "cuda")
    ms_step = ms / args.steps

    # end to end through the C ABI with host buffers: per step, the
    # excitation goes host -> device and the solution device -> host
    a_start = abi.tdbem_steps_done(ctx) + 1
    n_e2e = args.warmup + args.steps
    xc, nrm = _geometry(w)
    exc = torch.from_numpy(_excitation(w, xc, nrm, range(a_start, a_start + n_e2e))).pin_memory()
    xout = torch.empty((n_e2e, w.ns), dtype=torch.float64).pin_memory()
    for r in range(args.warmup):
        abi.tdbem_step_io(ctx, 1, exc[r], xout[r], on_device=False)
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    for r in range(args.warmup, n_e2e):
        abi.tdbem_step_io(ctx, 1, exc[r], xout[r], on_device=False)
    e2e_s = time.perf_counter() - t_e
    assert np.isfinite(xout.numpy()).all()
    n_done = abi.tdbem_steps_done(ctx)
    X = _unknown(s, w, n_done)
    s.close()

    hbm, peak_kind = _peaks()
    near_ms = st["ms_near"] / max(st["launches_near"], 1)
    near_gbs = st["near_bytes_per_step"] / (near_ms * 1e-3) / 1e9
    launches = st["launches_near"] + st["launches_solve"]
    out = {
        "metric": METRIC,
        "value": world * 1000.0 / ms_step,
        "unit": "time-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "e2e": {"value": world * args.steps / e2e_s, "unit": "time-steps/s",
                "h2d_bytes_per_step": w.ns * 8, "d2h_bytes_per_step": w.ns * 8},
        "clocks": clk.summary(),
    }
    phases = {"near_ms": near_ms, "solve_ms": st["ms_solve"] / max(st["steps"], 1),
              "solve_sweeps": st["solve_iters"]}
    if fmm:
        bf16, bf_kind = _bf16_peak()
        emu = 9.0  # FP32 products emulated by nine BF16 products
        peak = bf16 / emu if args.precision != "fp64" else FP64_TFLOPS
        m2l_tf = st["m2l_flops"] / (st["ms_m2l"] * 1e-3) / 1e12 if st["ms_m2l"] > 0 else 0.0
        phases.update({"far_ms": st["ms_far"] / args.steps, "m2l_ms": st["ms_m2l"] / args.steps,
                       "m2l_tflops": m2l_tf, "Lt": st["fmm_lt"], "mu": st["fmm_mu"]})
        launches += st["launches_far"] * 8 + st["launches_m2l"] * 3
        out["config"] = {"workload": args.workload + "_fmm_L%d_p%dx%d_%s" % (args.depth, args.ps, args.pt,
                                                                              args.precision),
                         "ns": w.ns, "d": w.d, "bie": w.bie, "bc": w.bc, "depth": args.depth, "ps": args.ps,
                         "pt": args.pt, "mu": st["fmm_mu"], "Lt": st["fmm_lt"],
                         "precision": ("FP64 throughout" if args.precision == "fp64" else
                                       "M2L FP32 on tensor cores (cuBLAS BF16x9 emulation), FP64 locals and "
                                       "recurrence, near-field history sum on FP32 pairs in double-float, FP64 "
                                       "coefficients and solve"),
                         "l2": "near coefficients + operator bank read every step exceed the 129 MB L2 only "
                               "partly; no flush", "setup_s": round(setup_s, 2),
                         "parallelism": "replicas" if world > 1 else "single-gpu"}
        out["roofline"] = {"bound": "tensor", "achieved": m2l_tf, "peak": peak, "unit": "TFLOP/s",
                           "frac": m2l_tf / peak, "traffic": None, "kernel": "M2L GEMM (cuBLAS, all offsets)",
                           "peak_source": ("measured bf16 / 9" if args.precision != "fp64" else
                                           "FP64 FMA probe (measured)"), "flops_per_step": st["m2l_flops"] / args.steps}
        out["near_roofline"] = {"bound": "hbm", "achieved": near_gbs, "peak": hbm, "frac": near_gbs / hbm}
    else:
        out["config"] = {"workload": args.workload + "_direct_" + args.precision, "ns": w.ns, "d": w.d,
                         "bie": w.bie, "bc": w.bc, "gamma_max": gmax, "spinup_steps": spin,
                         "coefficients_per_kind": st["n_coef"],
                         "precision": ("FP64 coefficients, histories, FMA and solve" if args.precision == "fp64" else
                                       "FP64 coefficients and solve; history sum on FP32 pairs (48-bit) in "
                                       "double-float arithmetic"),
                         "l2": "working set (%.1f GB per step) larger than L2; no flush" %
                               (st["near_bytes_per_step"] / 1e9),
                         "parallelism": "replicas" if world > 1 else "single-gpu", "setup_s": round(setup_s, 2)}
        out["roofline"] = {"bound": "hbm", "achieved": near_gbs, "peak": hbm, "unit": "GB/s", "frac": near_gbs / hbm,
                           "traffic": _traffic(st), "kernel": "k_near_sum", "peak_source": peak_kind,
                           "bytes_per_launch": st["near_bytes_per_step"], "avg_launch_ms": near_ms}
    out["phases_ms_per_step"] = phases
    out["gpu_launches"] = int(launches)

    if fmm:
        if args.accuracy:
            # accuracy: the direct path (parity-checked against the FP64 oracle)
            # over the same steps, and the FMM's FP64 form
            d = make("split", False)
            abi.tdbem_step(d.ctx, spin)
            Xd = _unknown(d, w, spin)
            d.close()
            X = X[:spin]
            out["accuracy"] = {"rel_l2_vs_direct": float(np.linalg.norm(X - Xd) / np.linalg.norm(Xd)),
                               "steps": spin, "target": 1e-3,
                               "reference": "direct history sum, parity 1e-11 with the FP64 oracle"}
            if args.fp64_form and args.precision != "fp64":
                f64 = make("fp64", True)
                abi.tdbem_step(f64.ctx, spin)
                Xf = _unknown(f64, w, spin)
                abi.tdbem_reset_stats(f64.ctx)
                msf = _timed(abi, torch, f64.ctx, min(args.steps, 40))
                f64.close()
                out["fp64_form"] = {"value": 1000.0 * min(args.steps, 40) / msf, "unit": "time-steps/s",
                                    "rel_l2_vs_direct": float(np.linalg.norm(Xf - Xd) / np.linalg.norm(Xd)),
                                    "mixed_rel_l2_vs_this": float(np.linalg.norm(X - Xf) / np.linalg.norm(Xf))}
            if args.direct_form:
                dd = make("split", False)
                abi.tdbem_step(dd.ctx, spin)
                msd = _timed(abi, torch, dd.ctx, args.steps)
                dd.close()
                out["direct_form"] = {"value": 1000.0 * args.steps / msd, "unit": "time-steps/s",
                                      "precision": "split", "note": "exact path (no FMM), all element pairs"}
    else:
        if args.fp64_form and args.precision != "fp64":
            out["fp64_form"] = fp64_form(args, w, phi, stream)
        if args.fmm_form:
            # the space-time FMM (mixed form) on the same workload and steps:
            # throughput and its error against this direct history
            t1 = time.time()
            f = make(args.precision, True)
            fsetup = time.time() - t1
            abi.tdbem_step(f.ctx, spin + args.warmup)
            abi.tdbem_sync(f.ctx)
            abi.tdbem_reset_stats(f.ctx)
            msf = _timed(abi, torch, f.ctx, args.steps)
            stf = f.stats()
            rest = n_done - abi.tdbem_steps_done(f.ctx)
            if rest > 0:
                abi.tdbem_step(f.ctx, rest)
            Xf = _unknown(f, w, n_done)
            f.close()
            m2l_tf = stf["m2l_flops"] / (stf["ms_m2l"] * 1e-3) / 1e12 if stf["ms_m2l"] > 0 else 0.0
            marks = [n for n in (60, 120, 240, n_done) if n <= n_done]
            err = [float(np.linalg.norm(Xf[:n] - X[:n]) / np.linalg.norm(X[:n])) for n in marks]
            # the same FMM with every pass in FP64: the mixed form's own error
            f64 = make("fp64", True)
            abi.tdbem_step(f64.ctx, n_done)
            X64 = _unknown(f64, w, n_done)
            f64.close()
            err64 = [float(np.linalg.norm(Xf[:n] - X64[:n]) / np.linalg.norm(X64[:n])) for n in marks]
            err64d = [float(np.linalg.norm(X64[:n] - X[:n]) / np.linalg.norm(X[:n])) for n in marks]
            out["fmm_form"] = {"value": 1000.0 * args.steps / msf, "unit": "time-steps/s",
                               "config": "depth %d, ps=pt=%d, mu=%d, Lt=%d, %s" % (
                                   args.depth, args.ps, stf["fmm_mu"], stf["fmm_lt"],
                                   "M2L FP32 on tensor cores (BF16x9)" if args.precision != "fp64" else "FP64"),
                               "rel_l2_vs_direct_after_steps": dict(zip([str(n) for n in (60, 120, 240, n_done)
                                                                         if n <= n_done], err)),
                               "meets_1e-3": bool(max(err) <= 1e-3),
                               "mixed_vs_fp64_fmm_after_steps": dict(zip([str(n) for n in marks], err64)),
                               "mixed_meets_1e-3_vs_fp64_fmm": bool(max(err64) <= 1e-3),
                               "fp64_fmm_vs_direct_after_steps": dict(zip([str(n) for n in marks], err64d)),
                               "m2l_tflops": m2l_tf,
                               "m2l_ms_per_step": stf["ms_m2l"] / args.steps,
                               "near_ms_per_step": stf["ms_near"] / args.steps,
                               "far_ms_per_step": stf["ms_far"] / args.steps, "setup_s": round(fsetup, 2),
                               "m2l_tile_n_by_level": stf["m2l_tile_n"][:args.depth + 1]}
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, rows=args.cpu_rows)
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


FP64_TFLOPS = 1.19  # FP64 FMA-chain probe on this machine's GB300 (0.596 TFMA/s)


def _traffic(st):
    """DRAM bytes (read + write) of one history-sum launch, from the ncu
    counters summarised in profiles/near_sum_traffic.txt: their ratio to the
    algorithmic bytes on the capture's workload, times this launch's
    algorithmic bytes.  None unless the summary is for the kernel as built
    (same source revision)."""
    tr_path = os.path.join(ROOT, "profiles", "near_sum_traffic.txt")
    if not os.path.exists(tr_path):
        return None
    try:
        kv = {}
        with open(tr_path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_rev") != _kernel_rev():
            return None
        return float(kv["bytes_per_algorithmic_byte"]) * st["near_bytes_per_step"]
    except Exception:
        return None


def fp64_form(args, w, phi, stream):
    """The same workload with the FP64 history sum (device steps/s only)."""
    import torch
    from paper_2111_05205_gb300 import Solver, abi
    s = Solver(w.xyz, w.tri, w.c, w.dt, w.nt, w.d, w.bie, phi=phi, incident=(w.direction, w.t0, w.sigma),
               stream=stream, precision="fp64")
    try:
        ctx = s.ctx
        g = s.stats()["gamma_max"]
        abi.tdbem_step(ctx, g + args.warmup)
        abi.tdbem_sync(ctx)
        abi.tdbem_reset_stats(ctx)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        abi.tdbem_step(ctx, args.steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        st = s.stats()
        near = st["ms_near"] / max(st["launches_near"], 1)
        hbm, _ = _peaks()
        return {"value": 1000.0 / ms, "unit": "time-steps/s", "ms_per_step": ms, "near_avg_ms": near,
                "near_hbm_frac": st["near_bytes_per_step"] / (near * 1e-3) / 1e9 / hbm}
    finally:
        s.close()


def _kernel_rev():
    """Source revision of the history-sum kernel: a hash of the code (line
    comments and blank lines dropped) of its part of csrc/march.cu (the file
    up to the end of its launcher: constants, incident term, double-float
    helpers, kernel) and of csrc/tdbem_internal.cuh."""
    import hashlib
    import re

    def code(text):
        lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.split("\n"))
        return "\n".join(ln for ln in lines if ln)

    h = hashlib.sha1()
    with open(os.path.join(ROOT, "paper_2111_05205_gb300", "csrc", "march.cu")) as fh:
        src = fh.read()
    b = src.index("cudaError_t launch_near_sum(")
    b = src.index("\n}\n", b)
    h.update(code(src[:b]).encode())
    with open(os.path.join(ROOT, "paper_2111_05205_gb300", "csrc", "tdbem_internal.cuh")) as fh:
        h.update(code(fh.read()).encode())
    return h.hexdigest()[:12]


class _OracleSample:
    """The FP64 oracle on the host cores on a bounded sample of the
    workload: the history sum (its step loop, Eq. linear) of `rows`
    observation rows over every lag and every source element; the rows'
    coefficients are the oracle's (computed once, untimed); one step of the
    sample is scaled by Ns / rows to a full step."""

    def __init__(self, w, rows):
        from oracle import coeffs as oc
        cdt = w.c * w.dt
        self.gm = oc.gamma_max(w.xyz, w.tri, w.d, cdt)
        rng = np.random.default_rng(0)
        self.rows = np.sort(rng.choice(w.ns, size=rows, replace=False))
        kind = "wb" if w.bc == "neumann" else "ub"
        self.C = oc.rows(w.xyz, w.tri, w.d, cdt, self.rows, kinds=(kind,), gmax=self.gm)[kind]  # [r, g, j]
        self.hist = np.random.default_rng(1).standard_normal((self.gm + 1, w.ns))
        self.ns = w.ns
        self.cores = oc.num_threads()
        self.sample = ("history sum of %d of %d rows over all %d lags (oracle dense rows, numpy), scaled x%.0f"
                       % (rows, w.ns, self.gm, w.ns / rows))

    def step_seconds(self):
        t = time.perf_counter()
        b = np.zeros(len(self.rows))
        for g in range(1, self.gm + 1):
            b += self.C[:, g, :] @ self.hist[self.gm - g]
        return (time.perf_counter() - t) * self.ns / len(self.rows)


def cpu_baseline(w, rows=2, repeats=3):
    o = _OracleSample(w, rows)
    per_step = min(o.step_seconds() for _ in range(repeats))
    return {"value": 1.0 / per_step, "unit": "time-steps/s", "cores": o.cores, "kind": "oracle", "sample": o.sample}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synth import workload
    w = workload(args.workload)
    o = _OracleSample(w, args.cpu_rows)
    for _ in range(args.warmup):
        o.step_seconds()
    per_step = float(np.mean([o.step_seconds() for _ in range(args.steps)]))
    out = {"metric": METRIC, "value": 1.0 / per_step, "unit": "time-steps/s", "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload + "_direct_" + args.precision, "ns": w.ns,
                      "oracle": "direct FP64 history sum (the same workload and steps)"},
           "cpu_baseline": {"value": 1.0 / per_step, "unit": "time-steps/s", "cores": o.cores,
                            "kind": "oracle", "sample": o.sample},
           "e2e": {"value": 1.0 / per_step, "unit": "time-steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_batch(args):
    """Batched driver on a mix shaped like the batched workload: N independent
    instances (seeded ellipsoids; Ns alternating 1280 / 5120; Nt drawn from
    U{256..1024}; OBIE d=1 and BMBIE d=2 alternating; sound-hard; split
    precision).  From the same start (a checkpoint after the warm-up steps)
    every instance is marched to its own last step Nt-1 by (a) plain
    launches, one instance after another, (b) one graph per instance, (c) one
    graph for all instances, replayed until the longest is done (shorter ones
    stop at their end on the device).  Timed with the host clock around each
    mode, device synchronised."""
    import torch
    from paper_2111_05205_gb300 import abi, build
    from synth import workload
    from tests.gpu_cases import gpu_solver
    build.build()
    n = args.batch
    rng = np.random.default_rng(2024)
    nts = [int(v) for v in rng.integers(256, 1025, size=n)]
    ws = [workload("ellipsoid%d_%s_hard_plane_s%d" % ((1280, 5120)[i % 2], ("bmbie_d2", "obie_d1")[(i // 2) % 2], i + 1),
                   nt=nts[i]) for i in range(n)]
    t0 = time.time()
    sols = [gpu_solver(w, precision=1) for w in ws]
    setup_s = time.time() - t0
    try:
        for s in sols:
            abi.tdbem_step(s.ctx, args.warmup)
        blobs = [abi.tdbem_checkpoint(s.ctx) for s in sols]
        todo = [nt - 1 - args.warmup for nt in nts]
        tot = sum(todo)

        def reset():
            for s, b in zip(sols, blobs):
                abi.tdbem_restore(s.ctx, b)
            torch.cuda.synchronize()

        torch.cuda.synchronize()
        t = time.perf_counter()
        for s, m in zip(sols, todo):
            abi.tdbem_step(s.ctx, m)
        torch.cuda.synchronize()
        t_plain = time.perf_counter() - t
        X_plain = [s.solution(0, nt - 1)[0] for s, nt in zip(sols, nts)]
        reset()
        t = time.perf_counter()
        for s, m in zip(sols, todo):
            abi.tdbem_step_graph(s.ctx, m)
        torch.cuda.synchronize()
        t_graph = time.perf_counter() - t
        reset()
        B = abi.tdbem_batch_create([s.ctx for s in sols])
        try:
            t = time.perf_counter()
            abi.tdbem_batch_step(B, max(todo))
            abi.tdbem_batch_sync(B)
            t_batch = time.perf_counter() - t
        finally:
            abi.tdbem_batch_destroy(B)
        same = all(np.array_equal(s.solution(0, nt - 1)[0], x) for s, nt, x in zip(sols, nts, X_plain))
        launches = sum(m * (1 + s.stats()["solve_iters"] + 1) for s, m in zip(sols, todo))
    finally:
        for s in sols:
            s.close()
    print(json.dumps({"metric": "instance-steps/sec, batched driver", "value": tot / t_batch,
                      "unit": "instance-steps/s", "n_gpus": 1, "steps": max(todo), "warmup": args.warmup,
                      "higher_is_better": True, "dtype": "f64+f32", "data": "synthetic",
                      "config": {"workload": "batch%d_ellipsoids_ns1280-5120_nt256-1024_obie-d1_bmbie-d2" % n,
                                 "instances": n, "ns": [w.ns for w in ws], "nt": nts,
                                 "instance_steps": tot, "setup_s": round(setup_s, 1),
                                 "excluded": "Ns=20480 instances: the direct form needs 15 GB of coefficients "
                                             "each, and FMM steps are not graph-replayed"},
                      "plain_launches": tot / t_plain, "graph_per_instance": tot / t_graph,
                      "batch_equals_plain": bool(same), "gpu_launches_plain": int(launches),
                      "timing": "host clock around each mode, device synchronised"}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-rows", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="split", choices=["split", "fp64"])
    ap.add_argument("--no-fp64-form", dest="fp64_form", action="store_false")
    ap.add_argument("--algo", default="direct", choices=["direct", "fmm"])
    ap.add_argument("--depth", type=int, default=4)
    ap.add_argument("--ps", type=int, default=4)
    ap.add_argument("--pt", type=int, default=4)
    ap.add_argument("--direct-form", action="store_true")
    ap.add_argument("--no-fmm-form", dest="fmm_form", action="store_false")
    ap.add_argument("--no-accuracy", dest="accuracy", action="store_false",
                    help="--algo fmm: skip the comparison runs against the direct path and the FP64 form")
    ap.add_argument("--batch", type=int, default=0, help="measure the batched driver with N instances")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.batch:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
