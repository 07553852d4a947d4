"""Benchmark of the time-domain BEM hot path on one GB300.

One "step" is one marching-on-in-time step (Eq. linear): the right-hand
side b^{a-1} (near-field history sum over the leaf neighbours' element
pairs, the incident-wave term and, at leaf-interval boundaries, the
space-time FMM's far field: P2M, M2M, M2L by symmetry class on the tcgen05
tensor cores, the Formula 1 recurrence, L2L, L2P) and the zero-lag solve.
The workload is the seeded synthetic scattering problem with Ns = 20480: a
sound-hard ellipsoid (icosphere subdivision 5 mapped by axes ~ U[0.5, 1.5],
seed 3), Burton-Miller BIE, B-spline order d = 2, c dt = 0.5 x mean edge,
Gaussian plane pulse (sigma = 0.3, seeded direction), Nt = 1024.  The FMM
runs at octree depth 3 with ps = 7, pt = 8 interpolation points and the M2L
in two scaled FP16 terms by default (the fastest configuration measured
whose whole march stays within 1e-3 of the direct path); the configuration
table's depth 5 with orders 5/5, depth 4 with 6/6, depth 3 with 8/8 and 5/5,
and the FFT form of the M2L (equispaced nodes) at depth 3 with 5/5 and 7/8
are measured beside it.

The timed steps are whole cycles of the FMM's interval pattern (the leaf
interval times 2^(depth-2) steps, so that every level's M2L occurs in its
true proportion), after a warm-up; the operator terms and coefficients read
per cycle are far larger than the 129 MB L2, so no flush is needed.  The
accuracy of the march (the whole Nt) is measured against the direct path,
which is parity-checked with the FP64 oracle, and against the same FMM in
FP64.  ``--algo direct`` times the direct (all-pairs) path instead.

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


PREC = {"fp64": 0, "split": 1, "bf16x3": 2, "bf16": 3, "f16x2": 4, "fft": 5}
PREC_NAME = {v: k for k, v in PREC.items()}
PREC_TEXT = {
    0: "FP64 throughout (M2L as FP64 GEMMs)",
    1: "M2L on tcgen05 tensor cores, operators and moments split into three BF16 terms with the six leading "
       "products (FP32-grade), FP32 accumulation in TMEM; FP64 locals and recurrence; near field on FP32 pairs "
       "(48-bit double-float); FP64 coefficients and zero-lag solve",
    2: "M2L on tcgen05 tensor cores, BF16x3 (two terms, three products); otherwise as the FP32-grade form",
    3: "M2L on tcgen05 tensor cores, single BF16 products; otherwise as the FP32-grade form",
    4: "M2L on tcgen05 tensor cores, operators and moments split into two FP16 terms scaled by powers of two "
       "per operator row and per cell's moment (about 22 bits), three products, FP32 accumulation in TMEM; "
       "otherwise as the FP32-grade form",
    5: "M2L near-future blocks by the FFT on equispaced nodes (observation box = source box): Toeplitz blocks as "
       "circular convolutions on a 2ps x 2ps x 2ps x 2pt grid, FP32 transforms and products on the CUDA cores, "
       "summed over each interaction list between the transforms; otherwise as the FP32-grade form",
}


def _solver(w, phi, stream, precision, fmm=None, depth=0):
    from paper_2111_05205_gb300 import Solver
    kw = dict(depth=depth, fmm=fmm) if fmm else {}
    return Solver(w.xyz, w.tri, w.c, w.dt, w.nt, w.d, w.bie, phi=phi, incident=(w.direction, w.t0, w.sigma, w.shape),
                  stream=stream, precision=precision, **kw)


def _e2e(abi, torch, ctx, w, n_warm, n_timed):
    """Steps through the C ABI with host buffers: every step copies its
    excitation host -> device and its solution device -> host."""
    a_start = abi.tdbem_steps_done(ctx) + 1
    xc, nrm = _geometry(w)
    exc = torch.from_numpy(_excitation(w, xc, nrm, range(a_start, a_start + n_warm + n_timed))).pin_memory()
    xout = torch.empty((n_warm + n_timed, w.ns), dtype=torch.float64).pin_memory()
    for r in range(n_warm):
        abi.tdbem_step_io(ctx, 1, exc[r], xout[r], on_device=False)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for r in range(n_warm, n_warm + n_timed):
        abi.tdbem_step_io(ctx, 1, exc[r], xout[r], on_device=False)
    s = time.perf_counter() - t
    assert np.isfinite(xout.numpy()).all()
    return n_timed / s


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_ours(args):
    if args.algo == "direct":
        return run_direct(args)
    return run_fmm(args)


def _rooflines(st, nsteps, prec):
    """Roofline objects of the history sum (HBM) and of the tcgen05 GEMM
    (tensor pipe) from one timed region's stats; the first of the returned
    triple is the kernel with the most device time per step."""
    bf16, bf_kind = _bf16_peak()
    gemm_ms = st["ms_gemm"] / max(st["launches_gemm"], 1)
    nprod = max(st["m2l_products"], 1)
    if prec:
        tc = st["gemm_tc_flops"] / (st["ms_gemm"] * 1e-3) / 1e12 if st["ms_gemm"] > 0 else 0.0
        gemm_obj = {
            "bound": "tensor", "achieved": tc, "peak": bf16, "unit": "TFLOP/s", "frac": tc / bf16,
            "traffic": None, "kernel": "k_tc_gemm (M2L, tcgen05)",
            "peak_source": bf_kind + " bf16 burst" + (" (FP16 has the same nominal dense rate)" if prec == 4 else ""),
            "flops_per_launch": st["gemm_tc_flops"] / max(st["launches_gemm"], 1), "avg_launch_ms": gemm_ms,
            "flops": "16-bit tensor-pipe flops the split needs: %d products x 2 P per kept operator row and pair "
                     "(K and tile padding not counted)" % nprod,
            "useful_tflops": tc / nprod, "useful_frac": tc / nprod / bf16}
    else:
        f64 = st["gemm_tc_flops"] / (st["ms_gemm"] * 1e-3) / 1e12 if st["ms_gemm"] > 0 else 0.0
        gemm_obj = {"bound": "alu", "achieved": f64, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                    "frac": f64 / FP64_TFLOPS, "traffic": None, "kernel": "M2L FP64 DGEMM",
                    "peak_source": "FP64 FMA probe (measured)"}
    hbm, peak_kind = _peaks()
    near_ms = st["ms_near"] / max(st["launches_near"], 1)
    near_obj = {"bound": "hbm", "kernel": "k_near_sum (near lists)", "avg_launch_ms": near_ms,
                "bytes_per_launch": st["near_bytes_per_step"],
                "achieved": st["near_bytes_per_step"] / (near_ms * 1e-3) / 1e9, "peak": hbm,
                "unit": "GB/s", "frac": st["near_bytes_per_step"] / (near_ms * 1e-3) / 1e9 / hbm,
                "traffic": _traffic(st), "peak_source": peak_kind + " copy bandwidth"}
    near_share, gemm_share = st["ms_near"] / nsteps, st["ms_gemm"] / nsteps
    dom = dict(near_obj if near_share >= gemm_share else gemm_obj)
    dom["ms_per_step"] = max(near_share, gemm_share)
    return dom, near_obj, gemm_obj


def run_fmm(args):
    """The headline: the space-time FMM (mixed form by default) on the
    benchmark workload, timed over whole cycles of its interval pattern,
    end to end through the C ABI with host buffers, and its error over the
    whole march against the direct path (parity 1e-11 with the FP64 oracle)
    and against the same FMM in FP64."""
    import torch
    from paper_2111_05205_gb300 import abi, build
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
    w = workload(args.workload, nt=args.nt)
    prec = PREC[args.precision]
    stream = torch.cuda.current_stream().cuda_stream
    phi = np.full(w.ns, 1 if w.bc == "neumann" else 0, np.int8)
    fmm = (args.ps, args.pt, 0)
    t0 = time.time()
    s = _solver(w, phi, stream, prec, fmm, args.depth)
    setup_s = time.time() - t0
    ctx = s.ctx
    st0 = s.stats()
    cycle = st0["fmm_lt"] << max(args.depth - 2, 0)  # steps between repeats of the interval pattern
    nsteps = max(cycle, (args.steps + cycle - 1) // cycle * cycle)
    spin = cycle  # every level has finished intervals before the warm-up
    need = spin + args.warmup + nsteps + 2 * args.warmup + nsteps
    if need > w.nt - 1:
        raise SystemExit("workload too short for %d timed steps" % nsteps)
    abi.tdbem_step(ctx, spin + args.warmup)
    abi.tdbem_sync(ctx)
    abi.tdbem_reset_stats(ctx)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        ms = _timed(abi, torch, ctx, nsteps)
        torch.cuda.nvtx.range_pop()
    if dist is not None:
        dist.barrier()
    st = s.stats()
    ms = max_over_ranks(ms, dist, "cuda")
    ms_step = ms / nsteps
    e2e = _e2e(abi, torch, ctx, w, args.warmup, nsteps)
    # the same steps once more with every far-field pass in order on one
    # stream, so that each kernel's own rate can be read (the headline's
    # timed region overlaps the deferred far-field work with the history sums)
    st_alone, ms_alone = None, None
    if prec and abi.tdbem_steps_done(ctx) + nsteps <= w.nt - 1:
        abi.tdbem_set_overlap(ctx, 0)
        abi.tdbem_reset_stats(ctx)
        torch.cuda.nvtx.range_push("alone")
        ms_alone = _timed(abi, torch, ctx, nsteps) / nsteps
        torch.cuda.nvtx.range_pop()
        st_alone = s.stats()
        abi.tdbem_set_overlap(ctx, 1)
    out = {
        "metric": METRIC, "value": world * 1000.0 / ms_step, "unit": "time-steps/s", "n_gpus": world,
        "steps": nsteps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": ("f64+f16" if prec == 4 else "f64+bf16") if prec else "f64", "data": "synthetic",
        "e2e": {"value": world * e2e, "unit": "time-steps/s", "h2d_bytes_per_step": w.ns * 8,
                "d2h_bytes_per_step": w.ns * 8},
        "clocks": clk.summary(),
        "config": {"workload": "%s_fmm_L%d_p%dx%d_%s" % (args.workload, args.depth, args.ps, args.pt, args.precision),
                   "ns": w.ns, "nt": w.nt, "d": w.d, "bie": w.bie, "bc": w.bc, "depth": args.depth,
                   "ps": args.ps, "pt": args.pt, "P": args.ps ** 3 * args.pt, "mu": st0["fmm_mu"],
                   "Lt": st0["fmm_lt"], "precision": PREC_TEXT[prec], "setup_s": round(setup_s, 2),
                   "timed_steps": "%d = whole cycles of %d steps (leaf interval x 2^(depth-2))" % (nsteps, cycle),
                   "l2": "the M2L operator terms (GBs per level) and the near coefficients read every cycle "
                         "exceed the 129 MB L2; no flush",
                   "parallelism": "replicas" if world > 1 else "single-gpu"},
    }
    out["roofline"], out["near_roofline"], out["m2l_gemm_roofline"] = _rooflines(st, nsteps, prec)
    if st_alone is not None:
        r = _rooflines(st_alone, nsteps, prec)
        out["kernels_alone"] = {
            "ms_per_step": ms_alone, "near_roofline": r[1], "m2l_gemm_roofline": r[2],
            "note": "the same steps timed again with every far-field pass in order on the context's stream "
                    "(tdbem_set_overlap 0): each kernel's rate without the overlapped far-field work beside it"}
    out["phases_ms_per_step"] = {
        "m2l": st["ms_m2l"] / nsteps, "m2l_gemm": st["ms_gemm"] / nsteps,
        "far_total": st["ms_far"] / nsteps, "near": st["ms_near"] / nsteps, "solve": st["ms_solve"] / nsteps,
        "solve_sweeps": st["solve_iters"], "m2l_useful_tflops": st["m2l_flops"] / max(st["ms_m2l"], 1e-12) / 1e9,
        "note": "phase times on their own streams: the deferred far-field work (M2L blocks 2..mu, exact rows, "
                "recurrence) runs beside the history sums, so the phases overlap"}
    out["m2l_tile_n_by_level"] = st["m2l_tile_n"][:args.depth + 1]
    out["gpu_launches"] = int(st["launches_near"] + st["launches_solve"] + st["launches_far_kernels"])
    if rank == 0 and args.accuracy:
        # the whole march: this FMM, the direct path, and the FMM's FP64 form
        rest = w.nt - 1 - abi.tdbem_steps_done(ctx)
        abi.tdbem_step(ctx, rest)
        X = _unknown(s, w, w.nt - 1)
        s.close()
        t1 = time.time()
        d = _solver(w, phi, stream, 1)
        dsetup = time.time() - t1
        abi.tdbem_step(d.ctx, 260)
        abi.tdbem_reset_stats(d.ctx)
        msd = _timed(abi, torch, d.ctx, args.warmup + 20)
        abi.tdbem_step(d.ctx, w.nt - 1 - abi.tdbem_steps_done(d.ctx))
        Xd = _unknown(d, w, w.nt - 1)
        d.close()
        marks = [n for n in (60, 120, 240, 480, 720, w.nt - 1) if n <= w.nt - 1]
        acc = {"rel_l2_vs_direct_after_steps": {str(n): _rel(X[:n], Xd[:n]) for n in marks},
               "reference": "direct history sum over all element pairs (split precision, parity 1e-11 with "
                            "the FP64 oracle), the same workload and steps", "target": 1e-3}
        acc["whole_march"] = acc["rel_l2_vs_direct_after_steps"][str(w.nt - 1)]
        acc["meets_1e-3"] = bool(acc["whole_march"] <= 1e-3)
        out["accuracy"] = acc
        out["direct_form"] = {"value": 1000.0 * (args.warmup + 20) / msd, "unit": "time-steps/s",
                              "setup_s": round(dsetup, 1), "note": "exact path (no FMM), all element pairs, "
                              "split precision; timed at steady state (every lag window in use)"}
        if prec and args.fp64_form:
            n64 = min(args.fp64_steps, w.nt - 1)
            f = _solver(w, phi, stream, 0, fmm, args.depth)
            abi.tdbem_step(f.ctx, cycle)
            abi.tdbem_reset_stats(f.ctx)
            ms64 = _timed(abi, torch, f.ctx, cycle)
            abi.tdbem_step(f.ctx, n64 - 2 * cycle)
            X64 = _unknown(f, w, n64)
            f.close()
            out["fp64_form"] = {
                "value": 1000.0 * cycle / ms64, "unit": "time-steps/s", "steps_marched": n64,
                "rel_l2_vs_direct": _rel(X64, Xd[:n64]), "mixed_rel_l2_vs_fp64": _rel(X[:n64], X64),
                "note": "the same FMM with every pass in FP64 (M2L as FP64 DGEMMs, FP64 near field); marched "
                        "%d steps (FP64 GEMMs run at about 1 TFLOP/s on this GPU)" % n64}
        if args.variants:
            # other hierarchies of the same problem: the configuration
            # table's depth 5 with orders 5/5, depth 4 with 6/6, depth 3 with
            # 8/8 and 5/5; the FFT form of the M2L (equispaced nodes) at
            # depth 3 with 5/5 (stable) and 7/8 (the march diverges)
            out["other_forms"] = []
            for depth, ps, pt, pv in ((5, 5, 5, prec), (4, 6, 6, prec), (3, 8, 8, prec), (3, 5, 5, prec), (3, 5, 5, 5),
                                      (3, 7, 8, 5)):
                if (depth, ps, pt, pv) == (args.depth, args.ps, args.pt, prec):
                    continue
                v = _solver(w, phi, stream, pv, (ps, pt, 0), depth)
                try:
                    c2 = v.stats()["fmm_lt"] << max(depth - 2, 0)
                    abi.tdbem_step(v.ctx, c2 + 3)
                    n2 = c2 * max(1, 112 // c2)
                    ms2 = _timed(abi, torch, v.ctx, n2)
                    abi.tdbem_step(v.ctx, w.nt - 1 - abi.tdbem_steps_done(v.ctx))
                    X2 = _unknown(v, w, w.nt - 1)
                finally:
                    v.close()
                e2 = _rel(X2, Xd)
                ok = bool(np.isfinite(e2))  # a diverging march may overflow
                form = {"depth": depth, "ps": ps, "pt": pt, "precision": PREC_NAME[pv], "value": 1000.0 * n2 / ms2,
                        "unit": "time-steps/s", "whole_march_rel_l2_vs_direct": e2 if ok else None,
                        "meets_1e-3": bool(ok and e2 <= 1e-3)}
                if pv == 5:
                    form["note"] = ("FFT form: equispaced nodes, whose interpolation amplifies with the order; on "
                                    "this march it stays bounded up to ps = pt = 5 and grows from 6 on")
                out["other_forms"].append(form)
    else:
        s.close()
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, rows=args.cpu_rows)
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def run_direct(args):
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
    """The FP64 oracle on the host cores on a bounded sample of the workload.

    One sample step is what the oracle's direct march (oracle.mot) does in a
    step, restricted in its history sum: the history sum of Eq. linear for
    `rows` observation rows over every source element and every lag (numpy
    over the oracle's coefficient rows, computed once by its C core with
    OpenMP, untimed), then the whole zero-lag solve A x = b for all Ns
    unknowns by the oracle's dense LU (factorised once, untimed).  A full
    step is estimated as the sampled history sum x Ns / rows plus the solve.
    The coefficient setup of the sampled rows is timed and scaled the same
    way (the oracle's per-row work is the same for every row)."""

    def __init__(self, w, rows):
        import scipy.linalg
        from oracle import coeffs as oc
        cdt = w.c * w.dt
        self.gm = oc.gamma_max(w.xyz, w.tri, w.d, cdt)
        rng = np.random.default_rng(0)
        self.rows = np.sort(rng.choice(w.ns, size=rows, replace=False))
        kind = ("wb" if w.bie == "bmbie" else "cw") if w.bc == "neumann" else ("ub" if w.bie == "bmbie" else "cu")
        t = time.perf_counter()
        self.C = oc.rows(w.xyz, w.tri, w.d, cdt, self.rows, kinds=(kind,), gmax=self.gm)[kind]  # [r, g, j]
        self.coef_s = (time.perf_counter() - t) * w.ns / rows
        t = time.perf_counter()
        A1 = oc.dense(w.xyz, w.tri, w.d, cdt, kinds=(kind,), gmax=1)[kind][1]
        A = -A1 if w.bc == "neumann" else A1  # the oracle's zero-lag matrix (unknown u, resp. q)
        del A1
        self.lu = scipy.linalg.lu_factor(A, overwrite_a=True, check_finite=False)
        self.lu_s = time.perf_counter() - t
        self.hist = np.random.default_rng(1).standard_normal((self.gm + 1, w.ns))
        self.b = np.random.default_rng(2).standard_normal(w.ns)
        self.ns = w.ns
        self.nrows = rows
        self.cores = oc.num_threads()
        self.sample = ("per step: the direct history sum of %d of %d rows over all %d lags (oracle coefficient rows, "
                       "numpy), scaled x%.0f, plus the whole zero-lag solve (oracle dense LU)"
                       % (rows, w.ns, self.gm, w.ns / rows))

    def step(self):
        """(measured seconds of the sample step, estimated seconds of a full step)."""
        import scipy.linalg
        t0 = time.perf_counter()
        b = np.zeros(self.nrows)
        for g in range(1, self.gm + 1):
            b += self.C[:, g, :] @ self.hist[self.gm - g]
        t1 = time.perf_counter()
        x = scipy.linalg.lu_solve(self.lu, self.b, check_finite=False)
        t2 = time.perf_counter()
        assert np.isfinite(b).all() and np.isfinite(x).all()
        return t2 - t0, (t1 - t0) * self.ns / self.nrows + (t2 - t1)

    def info(self, full_s):
        return {"value": 1.0 / full_s, "unit": "time-steps/s", "cores": self.cores, "kind": "oracle",
                "sample": self.sample, "full_step_s": full_s, "coefficient_setup_s": round(self.coef_s, 1),
                "coefficient_setup": "oracle C core (OpenMP) for the sampled rows, scaled to all rows",
                "lu_setup_s": round(self.lu_s, 1)}


def cpu_baseline(w, rows=8, repeats=3):
    o = _OracleSample(w, rows)
    full = min(o.step()[1] for _ in range(repeats))
    return o.info(full)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synth import workload
    w = workload(args.workload)
    o = _OracleSample(w, args.cpu_rows)
    for _ in range(args.warmup):
        o.step()
    meas, full = zip(*[o.step() for _ in range(args.steps)])
    full_s = float(np.mean(full))
    out = {"metric": METRIC, "value": 1.0 / full_s, "unit": "time-steps/s", "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(meas)) * 1e3,
           "ms_per_full_step": full_s * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload + "_direct_oracle", "ns": w.ns,
                      "oracle": "direct FP64 march (history sum + zero-lag solve), bounded row sample"},
           "timing": "ms_per_step is the measured sample step; value is the full-step throughput estimated from it",
           "cpu_baseline": o.info(full_s),
           "e2e": {"value": 1.0 / full_s, "unit": "time-steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_batch(args):
    """Batched driver on a mix shaped like the batched workload: N independent
    instances (seeded ellipsoids; Ns cycling 1280 / 5120 / 20480; Nt drawn
    from U{256..1024}; OBIE d=1 and BMBIE d=2 alternating; sound-hard), every
    one marched with the space-time FMM (ps = pt = 5, octree depth 2 / 3 / 4
    by size, M2L on the tensor cores in the FP32-grade split; the tile width
    of every level's GEMM picked by the setup-time tuner).  From the same
    start (a checkpoint after the warm-up steps) every instance is marched to
    its own last step Nt-1 by (a) plain launches, one instance after another,
    (b) one graph per instance, (c) one batch graph for all instances holding
    16 steps of each (graph launches until the longest is done; shorter ones
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
    sizes = (1280, 5120, 20480)
    depth_of = {1280: 2, 5120: 3, 20480: 4}
    ws = [workload("ellipsoid%d_%s_hard_plane_s%d" % (sizes[i % 3], ("bmbie_d2", "obie_d1")[(i // 3) % 2], i + 1),
                   nt=nts[i]) for i in range(n)]
    t0 = time.time()
    sols, depths = [], []
    for w in ws:
        # the deepest feasible octree up to the size's depth (leaf cells
        # larger than c dt and the element size)
        for depth in range(depth_of[w.ns], 1, -1):
            try:
                sols.append(gpu_solver(w, precision=1, depth=depth, fmm=(5, 5, 0)))
                depths.append(depth)
                break
            except abi.TdbemError as e:
                if e.code != -7 or depth == 2:
                    raise
    setup_s = time.time() - t0
    spl = 16
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
        st = [s.stats() for s in sols]
        reset()
        t = time.perf_counter()
        for s, m in zip(sols, todo):
            abi.tdbem_step_graph(s.ctx, m)
        torch.cuda.synchronize()
        t_graph = time.perf_counter() - t
        same_graph = all(np.array_equal(s.solution(0, nt - 1)[0], x) for s, nt, x in zip(sols, nts, X_plain))
        reset()
        B = abi.tdbem_batch_create_steps([s.ctx for s in sols], spl)
        try:
            t = time.perf_counter()
            abi.tdbem_batch_step(B, max(todo))
            abi.tdbem_batch_sync(B)
            t_batch = time.perf_counter() - t
        finally:
            abi.tdbem_batch_destroy(B)
        same = all(np.array_equal(s.solution(0, nt - 1)[0], x) for s, nt, x in zip(sols, nts, X_plain))
        launches = int(sum(x["launches_near"] + x["launches_solve"] + x["launches_far_kernels"] for x in st))
    finally:
        for s in sols:
            s.close()
    print(json.dumps({"metric": "instance-steps/sec, batched driver", "value": tot / t_batch,
                      "unit": "instance-steps/s", "n_gpus": 1, "steps": max(todo), "warmup": args.warmup,
                      "higher_is_better": True, "dtype": "f64+bf16", "data": "synthetic",
                      "config": {"workload": "batch%d_ellipsoids_ns1280-5120-20480_nt256-1024_obie-d1_bmbie-d2_fmm_p5x5"
                                             % n, "instances": n, "ns": [w.ns for w in ws], "nt": nts,
                                 "depth": depths, "ps": 5, "pt": 5, "precision": PREC_TEXT[1],
                                 "steps_per_graph_launch": spl, "instance_steps": tot,
                                 "setup_s": round(setup_s, 1),
                                 "m2l_tile_n": [x["m2l_tile_n"][:d + 1] for x, d in zip(st, depths)]},
                      "plain_launches": tot / t_plain, "graph_per_instance": tot / t_graph,
                      "batch_equals_plain": bool(same), "graph_equals_plain": bool(same_graph),
                      "gpu_launches_plain": launches,
                      "timing": "host clock around each mode, device synchronised"}))


def run_stability(args):
    """The sphere example of Section 5.1 (Tables 2-3) on the paper-shaped
    geodesic spheres with the raised-cosine pulse, direct path (the paper's
    CONV): for every BIE, order d and boundary condition, whether the march
    stays bounded.  A run counts as diverged when the largest |unknown| over
    the last quarter of the analysis time exceeds ten times its largest value
    over the first half (the pulse has passed the sphere by t ~ 1.5 of 9.6),
    or when the library's guard stops it (non-finite value)."""
    import torch
    from paper_2111_05205_gb300 import abi, build
    from synth import workload
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    rows = []
    for ns in [int(v) for v in args.study_sizes.split(",")]:
        for bie in ("obie", "bmbie"):
            for d in (1, 2, 3):
                for bc in ("soft", "hard"):
                    w = workload("paper_sphere%d_%s_d%d_%s" % (ns, bie, d, bc))
                    phi = np.full(w.ns, 1 if w.bc == "neumann" else 0, np.int8)
                    t0 = time.time()
                    s = _solver(w, phi, stream, 1)
                    status = "bounded"
                    try:
                        s.step()
                        X = _unknown(s, w, w.nt - 1)
                    except abi.TdbemError as e:
                        status, X = "diverged (guard: %s)" % e, None
                    finally:
                        s.close()
                    if X is not None:
                        peak = np.abs(X).max(axis=1)
                        early = peak[: len(peak) // 2].max()
                        late = peak[3 * len(peak) // 4:].max()
                        growth = float(late / max(early, 1e-300))
                        if not np.isfinite(growth) or growth > 10.0:
                            status = "diverged"
                    else:
                        growth = float("inf")
                    rows.append({"ns": ns, "bie": bie, "d": d, "bc": w.bc, "status": status,
                                 "late_over_early_peak": growth, "seconds": round(time.time() - t0, 1)})
                    print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"study": "stability of the sphere example (Section 5.1, Tables 2-3), direct path",
                      "rows": rows}))


def run_sai_study(args):
    """The learned SAI of the zero-lag solve at scale: the network (12 slots,
    32 hidden units, FP16 weights) is trained on the GPU, by the library's
    own forward, backward and Adam kernels, on the zero-lag matrices the
    library assembles for 200 seeded random ellipsoids (Ns cycling 1280 /
    5120 / 20480; Burton-Miller, d = 2, sound-hard); then, on held-out
    problems -- the 81920-element icosphere (subdivision 6, BMBIE d = 2
    sound-hard under the plane pulse, Nt = 2048, FMM) and the 20480-element
    benchmark ellipsoid -- the same march runs once with Jacobi and once
    with the learned SAI installed (tdbem_set_precond), each timed over the
    same steps with CUDA events; reported: sweeps and contraction of each
    solver, the zero-lag solve's ms per step (phase time of the library) and
    the whole step's, and the difference of the two histories (both solve
    to 1e-16)."""
    import torch
    from paper_2111_05205_gb300 import abi, build
    from synth import workload
    from tests.gpu_cases import gpu_solver
    build.build()
    t0 = time.time()
    sizes = (1280, 5120, 20480)
    train = [gpu_solver(workload("ellipsoid%d_bmbie_d2_hard_plane_s%d" % (sizes[i % 3], 1000 + i), nt=2))
             for i in range(args.sai_meshes)]
    setup_s = time.time() - t0
    sai = abi.tdbem_sai_create(12, 32, 3)
    out = {"study": "learned SAI of the zero-lag solve against Jacobi (held-out meshes)",
           "training": {"meshes": len(train), "ns": "cycling 1280/5120/20480", "epochs": args.sai_epochs,
                        "setup_s": round(setup_s, 1)}}
    try:
        t0 = time.time()
        L0 = abi.tdbem_sai_train(sai, [t.ctx for t in train], 1, 0.0)
        L1 = abi.tdbem_sai_train(sai, [t.ctx for t in train], args.sai_epochs, 2e-3)
        out["training"].update({"loss_before": L0, "loss_after": L1, "train_s": round(time.time() - t0, 1)})
        for t in train:
            t.close()
        train = []
        cases = [("sphere81920_bmbie_d2_hard_plane", 5, (4, 4, 0), 2048),
                 ("ellipsoid20480_bmbie_d2_hard_plane", 3, (7, 8, 0), 1024)]
        out["held_out"] = []
        for name, depth, fmm, nt in cases:
            w = workload(name, nt=nt)
            row = {"workload": name, "ns": w.ns, "nt": nt, "depth": depth, "ps": fmm[0], "pt": fmm[1]}
            res = {}
            X = {}
            for label, precond in (("jacobi", 0), ("learned_sai", 1)):
                s = gpu_solver(w, precision=4, depth=depth, fmm=fmm, precond=precond)
                try:
                    if precond:
                        use, sweeps, q = abi.tdbem_set_precond(s.ctx, sai)
                        res["sai_installed"] = bool(use)
                    st = s.stats()
                    cyc = st["fmm_lt"] << max(depth - 2, 0)
                    spin = cyc + 3
                    n = max(cyc, (200 // cyc) * cyc)
                    abi.tdbem_step(s.ctx, spin)
                    abi.tdbem_sync(s.ctx)
                    abi.tdbem_reset_stats(s.ctx)
                    ms = _timed(abi, torch, s.ctx, n)
                    st = s.stats()
                    res[label] = {"sweeps": st["solve_iters"], "contraction": st["solve_contraction"],
                                  "solve_ms_per_step": st["ms_solve"] / n, "step_ms": ms / n,
                                  "solve_launches_per_step": st["launches_solve"] / n}
                    s.step()
                    X[label] = s.solution(0, nt - 1)[0]
                finally:
                    s.close()
            res["rel_l2_sai_vs_jacobi"] = _rel(X["learned_sai"], X["jacobi"])
            res["solve_speedup"] = res["jacobi"]["solve_ms_per_step"] / res["learned_sai"]["solve_ms_per_step"]
            row.update(res)
            out["held_out"].append(row)
    finally:
        for t in train:
            t.close()
        abi.tdbem_sai_destroy(sai)
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=112)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--nt", type=int, default=None, help="override the workload's number of steps")
    ap.add_argument("--cpu-rows", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="f16x2", choices=["split", "fp64", "bf16x3", "bf16", "f16x2", "fft"])
    ap.add_argument("--fp64-steps", type=int, default=240,
                    help="--algo fmm: steps the FP64 form is marched for its comparison")
    ap.add_argument("--no-fp64-form", dest="fp64_form", action="store_false")
    ap.add_argument("--algo", default="fmm", choices=["direct", "fmm"])
    ap.add_argument("--depth", type=int, default=3)
    ap.add_argument("--ps", type=int, default=7)
    ap.add_argument("--pt", type=int, default=8)
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="--algo fmm: skip the other (depth, orders) forms measured beside the headline")
    ap.add_argument("--direct-form", action="store_true")
    ap.add_argument("--no-fmm-form", dest="fmm_form", action="store_false")
    ap.add_argument("--no-accuracy", dest="accuracy", action="store_false",
                    help="--algo fmm: skip the comparison runs against the direct path and the FP64 form")
    ap.add_argument("--batch", type=int, default=0, help="measure the batched driver with N instances")
    ap.add_argument("--study", default="", choices=["", "stability", "sai"],
                    help="stability: the sphere example of Section 5.1 for every BIE, d and boundary condition; "
                         "sai: the learned zero-lag preconditioner trained on 200 meshes, against Jacobi")
    ap.add_argument("--sai-meshes", type=int, default=200)
    ap.add_argument("--sai-epochs", type=int, default=60)
    ap.add_argument("--study-sizes", default="2880,5120,11520")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.study == "stability":
        run_stability(args)
    elif args.study == "sai":
        run_sai_study(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.batch:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
