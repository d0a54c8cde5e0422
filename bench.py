#!/usr/bin/env python
"""Benchmark of the Triad-ATRG RG step (4D Ising) on GB300.

Workload: chi = 48, r = 3, q = 2, beta = 0.1497, h = 1e-4, seed 2 (the chi = 48
configuration), split precision (3xTF32, FP64 small linear algebra).  One benchmark step is
one steady-state RG step (all legs at chi): bond-swap RSVD, triad isometries and tensors,
squeezers, contraction, re-split and the ln Z accumulation, plus the on-device Philox
sketches.  The first steps that grow the bond dimensions to chi are setup, untimed.

Prints one JSON line.  value = whole-job RG steps/s (N GPUs run independent replicas with
their own sketch keys: the path has no data exchange, so scaling is weak).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the
same workload (products of the chi = 48 bond-swap operator with 8 sketch columns), scaled
to RG steps/s by the step's algorithmic flop count.

Whole-run measurements of the other configurations (each writes a file under profiles/
that the benchmark line then reports, marked as stored):
  --c3-run       the 40-step chi = 48 run in FP64 and in split-precision schedules
  --c4-run       the 64-temperature sweep at chi = 32 with the order parameter X^(m)
  --c5-run       the derivatives at chi = 32 against central differences
  --methods-run  Triad-ATRG against plain ATRG (r = 7): step time and ln Z per chi
  --d3-run       3D Ising runs at the critical coupling
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CHI, R, Q, BETA, H, SEED = 48, 3, 2, 0.1497, 1e-4, 2
WORKLOAD = ("4D Ising Triad-ATRG, chi=48 r=3 q=2, beta=0.1497 h=1e-4, seed 2; one "
            "steady-state RG step (legs 48^4, bond 48)")
METRIC = "RG steps/s at chi=48 (split precision); TFLOP/s; df vs FP64 oracle"


def step_flops(chi, r, q):
    """Algorithmic flops of one steady-state step (swap, contraction, triad, squeezers)."""
    return ((2 * q + 2) * 4 * r * chi ** 7 + 8 * r * r * chi ** 7 + 8 * chi ** 7
            + 12 * r ** 4 * chi ** 6)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier_max(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------------------
_ORACLE = {}  # the chi = 48 swap operator, built once per process
SAMPLE_COLS = 8  # sketch columns of the timed oracle sample (the same in every leg)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max((d.get("num_threads", 0) for d in threadpool_info()), default=os.cpu_count())
    except Exception:
        return int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count()))


def workload_name(chi, r):
    if (chi, r) == (CHI, R):
        return WORKLOAD
    return WORKLOAD.replace("chi=48 r=3", "chi=%d r=%d" % (chi, r)).replace(
        "legs 48^4, bond 48", "legs %d^4, bond %d" % (chi, chi))


def oracle_sample(min_seconds=10.0, chi=CHI, r=R):
    """Time the FP64 oracle's bond-swap operator on a steady-state state of bond dimension
    chi (48 for the benchmark): products Mid @ Omega (the first product of the Eq. 1
    randomized SVD) with SAMPLE_COLS sketch columns, repeated until min_seconds have
    passed.  Returns (seconds per RG step scaled by the step's algorithmic flops,
    description, BLAS threads).  Building the state and the sketch is not timed."""
    from oracle import trg
    from paper_2412_14104_gb300 import synth
    if _ORACLE.get("chi") != chi:
        A, s, B = synth.split_state(7, (chi,) * 4, chi)
        Dk, I, Da = chi, chi ** 3, chi
        As = A.reshape(Dk, I, Da) * s[None, None, :]
        Bs = B.reshape(Da, Dk, I) * s[:, None, None]
        _ORACLE["op"] = trg.SwapOp(As, Bs, None)
        _ORACLE["om"] = synth.gaussian_matrix(3, _ORACLE["op"].shape[1], SAMPLE_COLS)
        _ORACLE["chi"] = chi
    op, om = _ORACLE["op"], _ORACLE["om"]
    reps, dt = 0, 0.0
    while dt < min_seconds or reps == 0:
        t = time.perf_counter()
        op.matmul(om)
        dt += time.perf_counter() - t
        reps += 1
    sample_flops = 4.0 * chi ** 6 * SAMPLE_COLS * reps
    per_step = dt * step_flops(chi, r, Q) / sample_flops
    desc = ("oracle SwapOp.matmul (Mid @ Omega of the chi=%d bond swap, %d sketch columns) x %d: "
            "%.3g flop in %.2f s, scaled to one RG step by its %.3g algorithmic flop" %
            (chi, SAMPLE_COLS, reps, sample_flops, dt, step_flops(chi, r, Q)))
    return per_step, desc, blas_threads()


def one_thread_sample(chi=CHI, r=R):
    """The same sample with one BLAS thread, in a child process (the thread count is fixed
    when NumPy loads).  Returns RG steps/s or None."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "print(bench.oracle_sample(min_seconds=1.0, chi=%d, r=%d)[0])" % (ROOT, chi, r))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=300)
        return 1.0 / float(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def cpu_baseline_record(min_seconds, chi=CHI, r=R):
    per, desc, threads = oracle_sample(min_seconds=min_seconds, chi=chi, r=r)
    return {"value": 1.0 / per, "unit": "RG steps/s", "cores": threads, "kind": "oracle",
            "sample": desc, "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "value_1_thread": one_thread_sample(chi, r)}


def run_reference(args, world, rank):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(min_seconds=0.0, chi=args.chi, r=args.r)
    times = []
    desc, threads = "", os.cpu_count()
    for _ in range(args.steps):
        per_step, desc, threads = oracle_sample(min_seconds=args.sample_seconds / max(args.steps, 1),
                                                chi=args.chi, r=args.r)
        times.append(per_step)
    per = sum(times) / len(times)
    value = 1.0 / per
    line = {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "RG steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.chi, args.r), "chi": args.chi, "r": args.r, "q": Q},
        "cpu_baseline": {"value": value, "unit": "RG steps/s", "cores": threads, "kind": "oracle",
                         "sample": desc + "; each timed step is one such sample, ms_per_step is "
                         "the extrapolated step time", "cpu_model": cpu_model(),
                         "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": "RG steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
def delta_f_check(tg):
    """Split-precision free energy against the stored FP64 oracle value of the chi = 24,
    r = 2, q = 2, 40-step run (h = 0, seed 1): relative differences of ln Z / V."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_c2_chi24.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        gold = json.load(f)
    c = gold["config"]
    out = {"config": "chi=24 r=2 q=2 beta=0.1497 h=0 seed 1, 40 steps", "oracle_lnz": gold["lnz"]}
    fp = tg.Context(c["chi"], c["r"], c["q"], seed=c["seed"]).init_ising(c["beta"], c["h"], c["d"])
    out["fp64_gpu_rel"] = abs(fp.rg_step(c["steps"]).lnZ() - gold["lnz"]) / abs(gold["lnz"])
    # 3xTF32 in every step, and the schedule FP64 steps 1-4, Ozaki slices 5-12, 3xTF32 after
    for tag, s0, early, late in (("tf32x3_from_step_1_rel", 1, 0, 0),
                                 ("tf32x3@5/ozaki:13_rel", 5, tg.OZAKI, 13)):
        ctx = tg.Context(c["chi"], c["r"], c["q"], seed=c["seed"], precision=tg.TF32X3, split_from_step=s0,
                         early_precision=early, late_from_step=late).init_ising(c["beta"], c["h"], c["d"])
        out[tag] = abs(ctx.rg_step(c["steps"]).lnZ() - gold["lnz"]) / abs(gold["lnz"])
    return out


C3_STEPS = 40
C3_FILE = os.path.join(ROOT, "profiles", "c3_chi48_runs.json")


def parse_form(text):
    """'fp64', 'tf32x3@13' (split precision from step 13), 'bf16x3' (from step 1),
    'tf32x3@5/bf16x6:13' (FP64 steps 1-4, bf16x6 steps 5-12, tf32x3 from step 13).
    Returns (name, start, early, late_from)."""
    head, _, sched = text.partition("/")
    name, _, start = head.partition("@")
    early, late = None, 0
    if sched:
        early, _, late = sched.partition(":")
        late = int(late)
    return name, int(start) if start else 1, early, late


def run_c3(args):
    """The chi = 48, r = 3, q = 2, h = 1e-4, 40-step configuration in whole runs, one per form
    in --c3-forms.  The FP64 run goes first; a form 'prec@k' (split precision from step k)
    continues from the FP64 run's state after step k - 1 (its first k - 1 steps are FP64
    steps, whose results repeat bit for bit), and its whole-run time is the FP64 run's time
    for those steps plus its own.  Each run's ln c_k per step and ln Z / V are written to
    profiles/c3_chi48_runs.json.  Prints one summary JSON line."""
    import torch
    import paper_2412_14104_gb300 as tg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    prec_of = {"tf32x3": tg.TF32X3, "bf16x3": tg.BF16X3, "bf16x6": tg.BF16X6, "ozaki": tg.OZAKI, "fp64": tg.FP64}
    forms = [(f, parse_form(f)) for f in args.c3_forms.split(",")]
    branch_at = sorted({k for _, (name, k, _, _) in forms if name != "fp64" and k > 1})
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def run(name, start, state=None, early=None, late=0, until=C3_STEPS):
        ctx = tg.Context(CHI, R, Q, seed=SEED, precision=prec_of[name], split_from_step=start,
                         stream=stream, early_precision=prec_of[early] if early else 0,
                         late_from_step=late)
        e0, e1 = ev(), ev()
        torch.cuda.synchronize()
        e0.record(stream)
        if state is None:
            ctx.init_ising(BETA, H, 4)
            k0 = 0
        else:
            A, s, B, k0, part = state
            ctx.set_state(A, s, B, k0, part)
        lnc, step_s, saved = [], [], {}

        def keep(k):  # the FP64 state after step k - 1, where split forms branch off
            torch.cuda.synchronize()
            A, s, B = ctx.get_state()
            saved[k] = (A, s, B, k - 1, ctx.step_info().partial_lnz if k > 1 else None)

        for k in range(k0 + 1, until + 1):
            if state is None and k in branch_at:
                keep(k)
            s0, s1 = ev(), ev()
            s0.record(stream)
            ctx.rg_step()
            s1.record(stream)
            torch.cuda.synchronize()
            lnc.append(ctx.step_info().lnc)
            step_s.append(s0.elapsed_time(s1) / 1e3)
        if state is None and until + 1 in branch_at:
            keep(until + 1)
        lnz = ctx.lnZ() if until == C3_STEPS else None
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.close()
        return {"lnz": lnz, "lnc": lnc, "step_s": step_s}, saved

    out = {}
    full_fp64 = any(name == "fp64" for _, (name, _, _, _) in forms)
    if not full_fp64:
        # reuse the stored whole FP64 run; recompute its trajectory only up to the last
        # branch point (FP64 steps repeat bit for bit)
        with open(C3_FILE) as f:
            out = json.load(f)["runs"]
        stop = max(branch_at) - 1 if branch_at else 0
        fp, saved = run("fp64", 1, until=stop)
        drift = max([abs(a - b) / max(1.0, abs(b)) for a, b in zip(fp["lnc"], out["fp64"]["lnc"][:stop])] + [0.0])
        assert drift < 1e-11, "the FP64 trajectory did not repeat (%.2e)" % drift
        fp = out["fp64"]
    else:
        fp, saved = run("fp64", 1)
        fp["run_s"] = sum(fp["step_s"])
        out["fp64"] = dict(fp, precision="fp64", split_from_step=None)
        print("fp64: lnZ/V = %.16f, %.1f s of steps" % (fp["lnz"], fp["run_s"]), flush=True)
    for tag, (name, k, early, late) in forms:
        if name == "fp64":
            continue
        res, _ = run(name, k, saved[k] if k > 1 else None, early, late)
        res["lnc"] = fp["lnc"][:k - 1] + res["lnc"]
        res["step_s"] = fp["step_s"][:k - 1] + res["step_s"]
        res["run_s"] = sum(res["step_s"])
        res["rel_to_fp64"] = abs(res["lnz"] - fp["lnz"]) / abs(fp["lnz"])
        out[tag] = dict(res, precision=name, split_from_step=k, early_precision=early, late_from_step=late)
        print("%s: lnZ/V = %.16f, rel %.3e, %.1f s of steps" % (tag, res["lnz"], res["rel_to_fp64"],
                                                                 res["run_s"]), flush=True)
    out["fp64"]["rel_to_fp64"] = 0.0
    doc = {"config": "chi=48 r=3 q=2 beta=0.1497 h=1e-4 seed 2, 40 steps, d=4",
           "command": "python bench.py --c3-run --c3-forms " + args.c3_forms,
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "timing": "sum of per-step CUDA-event times (init and state copies excluded)",
           "runs": out}
    os.makedirs(os.path.dirname(C3_FILE), exist_ok=True)
    with open(C3_FILE, "w") as f:
        json.dump(doc, f, indent=1)
    print(json.dumps(c3_summary(doc)), flush=True)


def c3_summary(out):
    """ln Z / V differences and whole-run times of the stored 40-step chi = 48 runs."""
    runs = out["runs"]
    return {"config": out["config"], "measured": out["when"], "command": out["command"],
            "lnz_fp64_gpu": runs["fp64"]["lnz"] if "fp64" in runs else None,
            "forms": {k: {"rel_to_fp64_gpu": v.get("rel_to_fp64"), "run_s": v["run_s"]}
                      for k, v in runs.items()}}


METHODS_FILE = os.path.join(ROOT, "profiles", "methods_scaling.json")


def run_methods(args):
    """Triad-ATRG against plain ATRG (the triad with identity isometries, the O(chi^9)
    contraction) in the paper's comparison setting r = 7 (Table 2, Figs. 5 and 6): for each
    chi of --methods-chis, the steady-state step time (CUDA events over --steps steps after
    the legs reach chi) and ln Z / V after --methods-steps steps, at beta = 0.1497, h = 0,
    d = 4, in the precision of --precision.  Writes profiles/methods_scaling.json with a
    least-squares exponent of step time against chi per method; prints one JSON line."""
    import numpy as np
    import torch
    import paper_2412_14104_gb300 as tg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    prec = {"tf32x3": tg.TF32X3, "bf16x3": tg.BF16X3, "bf16x6": tg.BF16X6, "ozaki": tg.OZAKI, "fp64": tg.FP64}[args.precision]
    chis = [int(c) for c in args.methods_chis.split(",")]
    r = 7
    rows = {}
    skipped = {}
    for method, mname in ((tg.TRIAD, "triad"), (tg.ATRG, "atrg")):
        for chi in chis:
            # ATRG (the triad with identity isometries, k = chi^2): the largest buffer is the
            # contraction's intermediate q of chi^7 doubles, twice over in a split precision
            # (q and its packed tensor-core operand); runs above 160 GB of it are skipped
            if method == tg.ATRG and 16.0 * chi ** 7 > 160e9:
                skipped["atrg_%d" % chi] = "contraction intermediate of 16 chi^7 = %.0f GB" % (16.0 * chi ** 7 / 1e9)
                continue
            ctx = tg.Context(chi, r, Q, method=method, seed=SEED, precision=prec, stream=stream)
            ctx.init_ising(BETA, 0.0, 4)
            k = 0
            while not all(x == chi for x in list(ctx.step_info().dims)[:5]) or k == 0:
                ctx.rg_step()
                k += 1
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.rg_step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            k += args.steps
            ms = e0.elapsed_time(e1) / args.steps
            if args.methods_steps > k:
                ctx.rg_step(args.methods_steps - k)
            lnz = ctx.lnZ()
            ctx.close()
            rows["%s_%d" % (mname, chi)] = {"method": mname, "chi": chi, "r": r, "ms_per_step": ms,
                                             "lnz": lnz, "steps": max(k, args.methods_steps)}
            print("%s chi=%d: %.1f ms/step, lnZ/V %.12f" % (mname, chi, ms, lnz), flush=True)
    fits = {}
    for mname in ("triad", "atrg"):
        pts = [(math.log(v["chi"]), math.log(v["ms_per_step"])) for v in rows.values() if v["method"] == mname]
        if len(pts) >= 2:
            x, y = np.array(pts).T
            fits[mname] = float(np.polyfit(x, y, 1)[0])
    dev = {str(c): abs(rows["triad_%d" % c]["lnz"] - rows["atrg_%d" % c]["lnz"]) / abs(rows["atrg_%d" % c]["lnz"])
           for c in chis if "triad_%d" % c in rows and "atrg_%d" % c in rows}
    doc = {"config": "4D Ising, beta=0.1497 h=0, r=7, q=2, seed 2, precision %s" % args.precision,
           "command": "python bench.py --methods-run --methods-chis %s --steps %d --methods-steps %d --precision %s"
                      % (args.methods_chis, args.steps, args.methods_steps, args.precision),
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "time_exponent": fits, "triad_vs_atrg_rel_lnz": dev, "runs": rows, "skipped": skipped}
    os.makedirs(os.path.dirname(METHODS_FILE), exist_ok=True)
    with open(METHODS_FILE, "w") as f:
        json.dump(doc, f, indent=1)
    print(json.dumps({"time_exponent": fits, "triad_vs_atrg_rel_lnz": dev}), flush=True)


C5_FILE = os.path.join(ROOT, "profiles", "c5_grad_chi32.json")


def run_c5(args):
    """The derivative configuration: chi = 32, r = 2, q = 2, 32 steps, beta = 0.1497,
    h in --c5-h (comma separated; default 1e-3), seed 4.  The forward-mode derivatives of
    tatrg_grad (dlnZ/dbeta, dlnZ/dh, d2lnZ/dbeta2 per site; its tangent passes run
    concurrently) against central differences of the GPU's own FP64 ln Z / V for each step
    of --c5-eps (first derivatives) and --c5-eps2 (second derivative, whose centre value is
    the run the derivatives are taken of).  The computed ln Z / V is only piecewise smooth
    (a truncation that changes with beta moves it by up to the truncation error), so a
    difference is a derivative only while its stencil stays inside one smooth piece: pairs
    of steps (e, 2e) that agree show it.  The difference runs are independent and run on
    concurrent threads and streams.  With --c5-reuse, the tangents and differences already
    stored for the same h are kept and only the missing steps run.  Writes
    profiles/c5_grad_chi32.json after each h; prints one JSON line per h."""
    import concurrent.futures as cf
    import torch
    import paper_2412_14104_gb300 as tg
    torch.cuda.set_device(0)
    chi, r, steps, seed, beta = 32, 2, 32, 4, 0.1497
    eps1 = [float(x) for x in args.c5_eps.split(",") if x]
    eps2 = [float(x) for x in args.c5_eps2.split(",") if x]

    def lnz(b, h):
        st = torch.cuda.Stream()
        t0 = time.perf_counter()
        with torch.cuda.stream(st):
            z = tg.Context(chi, r, Q, seed=seed, stream=st).init_ising(b, h, 4).rg_step(steps).lnZ()
        print("  run beta=%.9f h=%.9g: lnZ/V %.16f (%.0f s)" % (b, h, z, time.perf_counter() - t0), flush=True)
        return z

    stored = {}
    if args.c5_reuse and os.path.exists(C5_FILE):
        with open(C5_FILE) as f:
            stored = json.load(f).get("results", {})
    out = dict(stored)
    for h in [float(x) for x in args.c5_h.split(",")]:
        key = "h=%g" % h
        row = dict(stored.get(key, {}))
        if "dlnz_dbeta" not in row:
            t0 = time.perf_counter()
            ctx = tg.Context(chi, r, Q, seed=seed).init_ising(beta, h, 4).rg_step(steps)
            row["lnz"] = ctx.lnZ()
            row["run_s"] = time.perf_counter() - t0
            t0 = time.perf_counter()
            row["dlnz_dbeta"], row["dlnz_dh"], row["d2lnz_dbeta2"] = ctx.grad(second=True)
            row["grad_s"] = time.perf_counter() - t0
            ctx.close()
        print("  tangents: %.12g %.12g %.12g" % (row["dlnz_dbeta"], row["dlnz_dh"], row["d2lnz_dbeta2"]), flush=True)
        fd = row.setdefault("differences", {})
        need = []
        for e in eps1:
            if "dbeta %g" % e not in fd:
                need += [(beta + e, h), (beta - e, h)]
            if h != 0.0 and "dh %g" % e not in fd:
                need += [(beta, h + e), (beta, h - e)]
        for e in eps2:
            if "d2beta %g" % e not in fd:
                need += [(beta + e, h), (beta - e, h)]
        need = sorted(set(need))
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=3) as ex:
            zs = dict(zip(need, ex.map(lambda bh: lnz(*bh), need)))
        row["fd_runs_s"] = row.get("fd_runs_s", 0.0) + time.perf_counter() - t0
        z0 = row["lnz"]
        for e in eps1:
            if "dbeta %g" % e not in fd:
                v = (zs[(beta + e, h)] - zs[(beta - e, h)]) / (2 * e)
                fd["dbeta %g" % e] = {"fd": v, "rel_to_tangent": abs(row["dlnz_dbeta"] - v) / abs(v)}
            if h != 0.0 and "dh %g" % e not in fd:
                v = (zs[(beta, h + e)] - zs[(beta, h - e)]) / (2 * e)
                fd["dh %g" % e] = {"fd": v, "rel_to_tangent": abs(row["dlnz_dh"] - v) / abs(v)}
        for e in eps2:
            if "d2beta %g" % e not in fd:
                v = (zs[(beta + e, h)] - 2 * z0 + zs[(beta - e, h)]) / (e * e)
                fd["d2beta %g" % e] = {"fd": v, "rel_to_tangent": abs(row["d2lnz_dbeta2"] - v) / abs(v)}
        out[key] = row
        print(json.dumps({"h": h, **row}), flush=True)
        doc = {"config": "chi=32 r=2 q=2, 32 steps, beta=0.1497, seed 4, d=4, FP64",
               "command": "python bench.py --c5-run --c5-h %s --c5-eps %s --c5-eps2 %s%s"
                          % (args.c5_h, args.c5_eps, args.c5_eps2, " --c5-reuse" if args.c5_reuse else ""),
               "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "results": out}
        os.makedirs(os.path.dirname(C5_FILE), exist_ok=True)
        with open(C5_FILE, "w") as f:
            json.dump(doc, f, indent=1)


C4_FILE = os.path.join(ROOT, "profiles", "c4_sweep_chi32.json")


def run_c4(args):
    """The temperature-sweep configuration: 64 temperatures uniformly spaced in
    beta in [0.145, 0.155], h = 0, chi = 32, r = 2, q = 2, 32 steps each, split precision
    (3xTF32), seed 3.  Times tatrg_sweep_observables with --sweep-workers concurrent runs
    against the same call with one worker (the first --c4-serial temperatures, scaled to 64),
    and reads the order parameter X^(m) of every run after every step: for each m, the
    transition estimate is where X^(m) first crosses 1.5 between the disordered value 1 and
    the ordered value 2.  Writes profiles/c4_sweep_chi32.json; prints one JSON line."""
    import numpy as np
    import torch
    import paper_2412_14104_gb300 as tg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    betas = 0.145 + np.arange(64) * (0.01 / 63)
    chi, r, steps, seed = 32, 2, 32, 3
    prec = {"tf32x3": tg.TF32X3, "bf16x3": tg.BF16X3, "bf16x6": tg.BF16X6, "ozaki": tg.OZAKI, "fp64": tg.FP64}[args.precision]
    ctx = tg.Context(chi, r, Q, seed=seed, precision=prec, sweep_workers=args.sweep_workers, stream=stream)
    ctx.sweep_observables(betas[:2], 0.0, 4, steps)  # first-use setup (tuning of the shapes)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    z, x = ctx.sweep_observables(betas, 0.0, 4, steps)
    torch.cuda.synchronize()
    t_sweep = time.perf_counter() - t0
    one = tg.Context(chi, r, Q, seed=seed, precision=prec, sweep_workers=1, stream=stream)
    ns = max(1, min(len(betas), args.c4_serial))
    t0 = time.perf_counter()
    z1, x1 = one.sweep_observables(betas[:ns], 0.0, 4, steps)
    torch.cuda.synchronize()
    t_serial = (time.perf_counter() - t0) * len(betas) / ns

    def crossing(col):
        for i in range(len(betas) - 1):
            if col[i] < 1.5 <= col[i + 1]:
                return float(betas[i] + (1.5 - col[i]) * (betas[i + 1] - betas[i]) / (col[i + 1] - col[i]))
        return None

    beta_c = [crossing(x[:, m]) for m in range(steps)]
    doc = {"config": "64 beta in [0.145, 0.155], h=0, chi=32 r=2 q=2, 32 steps, %s, seed 3, %d workers"
                     % (args.precision, args.sweep_workers),
           "command": "python bench.py --c4-run --sweep-workers %d --c4-serial %d --precision %s"
                      % (args.sweep_workers, args.c4_serial, args.precision),
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "sweep_s": t_sweep, "serial_s_for_64": t_serial,
           "serial_note": "the first %d temperatures through the same call with one worker, scaled to 64" % ns,
           "runs_per_s_sweep": len(betas) / t_sweep, "runs_per_s_serial": len(betas) / t_serial,
           "rg_steps_per_s_sweep": len(betas) * steps / t_sweep,
           "serial_vs_sweep_rel_lnz": [abs(a - b) / abs(b) for a, b in zip(z1, z[:ns])],
           "beta_c_by_step": beta_c,
           "x_max_by_step": [float(x[:, m].max()) for m in range(steps)],
           "x_min_by_step": [float(x[:, m].min()) for m in range(steps)],
           "betas": betas.tolist(), "lnz": z.tolist(), "X_by_step": x.tolist()}
    os.makedirs(os.path.dirname(C4_FILE), exist_ok=True)
    with open(C4_FILE, "w") as f:
        json.dump(doc, f, indent=1)
    print(json.dumps({k: doc[k] for k in ("config", "sweep_s", "serial_s_for_64", "runs_per_s_sweep",
                                          "runs_per_s_serial", "beta_c_by_step", "x_max_by_step")}), flush=True)


D3_FILE = os.path.join(ROOT, "profiles", "d3_runs.json")


def run_d3(args):
    """3D Ising production runs (the MDTRG comparison system of Sec. 1): Triad-ATRG at the 3D
    critical coupling beta = 0.2216544, h = 0, r = 2, q = 2, 30 steps, chi in --d3-chis,
    split precision from step 13; ln Z / V and the steady-state step time per chi.  Writes
    profiles/d3_runs.json."""
    import torch
    import paper_2412_14104_gb300 as tg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    prec = {"tf32x3": tg.TF32X3, "bf16x3": tg.BF16X3, "bf16x6": tg.BF16X6, "ozaki": tg.OZAKI, "fp64": tg.FP64}[args.precision]
    rows = {}
    for chi in [int(c) for c in args.d3_chis.split(",")]:
        ctx = tg.Context(chi, 2, Q, seed=6, precision=prec, split_from_step=13, stream=stream)
        ctx.init_ising(0.2216544, 0.0, 3)
        ms = []
        for k in range(30):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.rg_step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        rows[str(chi)] = {"lnz": ctx.lnZ(), "ms_last_steps": sum(ms[-5:]) / 5, "run_s": sum(ms) / 1e3}
        ctx.close()
        print("d3 chi=%d: %s" % (chi, rows[str(chi)]), flush=True)
    doc = {"config": "3D Ising beta=0.2216544 h=0, r=2 q=2, 30 steps, %s from step 13, seed 6" % args.precision,
           "command": "python bench.py --d3-run --d3-chis %s --precision %s" % (args.d3_chis, args.precision),
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "runs": rows}
    os.makedirs(os.path.dirname(D3_FILE), exist_ok=True)
    with open(D3_FILE, "w") as f:
        json.dump(doc, f, indent=1)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2412_14104_gb300 as tg

    torch.cuda.set_device(local)
    if world > 1:
        # several GPUs in one job: single-CTA tiles only, so no kernel of this process uses
        # the cluster-multicast TMA form (that form is kept for single-GPU runs)
        tg.set_cta_pairs(-1)
    stream = torch.cuda.current_stream()
    prec = {"tf32x3": tg.TF32X3, "bf16x3": tg.BF16X3, "bf16x6": tg.BF16X6, "ozaki": tg.OZAKI, "fp64": tg.FP64}[args.precision]
    seed = SEED + 1000 * rank
    chi, r = args.chi, args.r
    ctx = tg.Context(chi, r, Q, seed=seed, precision=prec, profile=1, stream=stream)
    ctx.init_ising(BETA, H, 4)
    while True:  # setup: grow every leg to chi
        ctx.rg_step()
        if all(x == chi for x in list(ctx.step_info().dims)[:5]):
            break
    for _ in range(args.warmup):
        ctx.rg_step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()  # lets `ncu --profile-from-start off` see the timed steps only
    start.record(stream)
    infos = []
    for _ in range(args.steps):
        ctx.rg_step()
        i = ctx.step_info()
        infos.append((list(i.flops), i.tc_ms, i.tc_flops, i.tc_launches, i.kernel_launches, list(i.ms)))
    end.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    ms_max = barrier_max(world, ms)
    value = args.steps * world / (ms_max / 1e3)
    alg_flops = sum(sum(f) for f, *_ in infos)
    tc_ms = sum(x[1] for x in infos)
    tc_flops = sum(x[2] for x in infos)
    tc_launches = sum(x[3] for x in infos)
    launches = sum(x[4] for x in infos)
    stage_ms = [sum(x[5][k] for x in infos) / len(infos) for k in range(5)]

    # end to end through the C ABI with host buffers: state in from pinned host memory,
    # one step, state out to pinned host memory
    A, s, B = ctx.get_state()
    pins = [torch.empty(a.shape, dtype=torch.float64).pin_memory() for a in (A, s, B)]
    for p_, a in zip(pins, (A, s, B)):
        p_.numpy()[...] = a
    hA, hs, hB = (p_.numpy() for p_ in pins)
    e2e_steps = max(1, min(5, args.steps))
    k0 = ctx.step_info().step
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(e2e_steps):
        ctx.set_state(hA, hs, hB, k0 + j, 0.0)
        ctx.rg_step()
        hA, hs, hB = ctx.get_state()
    torch.cuda.synchronize()
    e2e_s = barrier_max(world, time.perf_counter() - t0)
    io_bytes = 8 * (A.size + s.size + B.size)

    peaks, src = measured_peaks()
    bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    if prec == tg.TF32X3:
        peak = bf16 * (1.1 / 2.25)
        note = ("tf32 peak derived, not measured: %s bf16 sustained %.0f TFLOP/s x the nominal "
                "dense tf32/bf16 ratio 1.1/2.25" % (src, bf16))
    else:
        peak, note = bf16, "%s bf16 sustained" % src
    # achieved: algorithmic flops (2 M N K per contraction) over the kernel's device time;
    # the split forms issue 3 (6 for bf16x6) tensor-core products per algorithmic one
    achieved = tc_flops / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None
    nprod = {tg.BF16X6: 6.0, tg.OZAKI: 15.0}.get(prec, 3.0)
    # DRAM traffic: no capture of this workload's launches (tens of GB resident); the
    # committed one-launch capture of the chi = 32 C2 contraction stands beside it
    traffic_sample = None
    prof = os.path.join(ROOT, "profiles", "tc_gemm_c2_chi32_traffic.json")
    if os.path.exists(prof):
        with open(prof) as f:
            traffic_sample = json.load(f)

    fp64_ms = None
    if args.fp64_steps > 0 and prec != tg.FP64:
        f64 = tg.Context(chi, r, Q, seed=seed, stream=stream)
        f64.set_state(A, s, B, k0, 0.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f64.rg_step(args.fp64_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = e0.elapsed_time(e1) / args.fp64_steps
    df = delta_f_check(tg) if (rank == 0 and not args.no_delta_f) else None

    if rank != 0:
        return
    workload = workload_name(chi, r)
    line = {
        "metric": METRIC,
        "value": value, "unit": "RG steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": workload, "chi": chi, "r": r, "q": Q, "precision": args.precision,
                   "l2": "inputs larger than L2 (each step streams > 10 GB of tensors)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "tile_forms": "single CTAs only" if world > 1 else "autotuned"},
        "tflops_algorithmic": alg_flops / (ms / 1e3) / 1e12,
        "tflops_algorithmic_note": "flops the library counts for the executed contractions; "
                                   "tflops_cost_formula uses the steady-state cost formula",
        "tflops_cost_formula": step_flops(chi, r, Q) / (ms / (1e3 * args.steps)) / 1e12,
        "stage_ms": dict(zip(["swap", "triad", "squeeze", "contract", "resplit"], stage_ms)),
        "roofline": {"bound": "tensor", "kernel": "tc_gemm_kernel (tcgen05 3-product split GEMM)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "frac_algorithmic": (achieved / peak) if achieved else None,
                     "traffic": None,
                     "traffic_note": "not captured on this workload; traffic_sample is one ncu "
                                     "capture of the chi = 32 C2 launch (same kernel, 3xTF32)",
                     "traffic_sample": traffic_sample, "peak_source": note,
                     "launches": tc_launches, "launches_note": "tensor-core launches on the "
                     "context's stream; the small GEMMs of the factorisations that run concurrently "
                     "on worker streams are not timed here",
                     "avg_launch_ms": tc_ms / max(tc_launches, 1),
                     "flops_per_launch": tc_flops / max(tc_launches, 1),
                     "hardware_products": {
                         "achieved": nprod * achieved if achieved else None,
                         "frac": (nprod * achieved / peak) if achieved else None,
                         "note": "%d tensor-core products per algorithmic product" % nprod}},
        "e2e": {"value": e2e_steps * world / e2e_s, "unit": "RG steps/s",
                "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes},
        "gpu_launches": launches,
        "clocks": clk,
        "fp64_gpu_ms_per_step": fp64_ms,
        "split_vs_fp64_speedup": (fp64_ms / (ms_max / args.steps)) if fp64_ms else None,
        "delta_f": df,
    }
    if os.path.exists(C3_FILE) and (chi, r) == (CHI, R):
        with open(C3_FILE) as f:
            line["delta_f_chi48"] = dict(c3_summary(json.load(f)),
                                         note="stored whole-run measurement (not re-run by this "
                                              "command); the FP64 GPU step is checked against the "
                                              "oracle by the chi = 48 teacher-forced step test")
    stored = {}
    for name, path, keys in (
            ("c4_sweep", C4_FILE, ("config", "when", "command", "runs_per_s_sweep", "runs_per_s_serial",
                                   "rg_steps_per_s_sweep", "beta_c_by_step")),
            ("c5_grad", C5_FILE, ("config", "when", "command", "results")),
            ("methods", METHODS_FILE, ("config", "when", "command", "time_exponent", "triad_vs_atrg_rel_lnz")),
            ("d3", D3_FILE, ("config", "when", "command", "runs"))):
        if os.path.exists(path):
            with open(path) as f:
                doc = json.load(f)
            stored[name] = {k: doc.get(k) for k in keys}
    if stored:
        line["stored_runs"] = dict(stored, note="whole-run measurements of the other configurations, "
                                                "written by the commands named in each (not re-run here)")
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_record(10.0, chi, r)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["tf32x3", "bf16x3", "bf16x6", "ozaki", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-delta-f", action="store_true")
    ap.add_argument("--chi", type=int, default=CHI,
                    help="bond dimension (48 is the benchmark; smaller values size ncu captures)")
    ap.add_argument("--r", type=int, default=R)
    ap.add_argument("--sample-seconds", type=float, default=20.0,
                    help="host seconds of oracle work the reference arm times (over all steps)")
    ap.add_argument("--c3-run", action="store_true",
                    help="run the 40-step chi = 48 configuration in the forms of --c3-forms")
    ap.add_argument("--c3-forms", default="fp64,tf32x3@1,bf16x3@1,tf32x3@5,bf16x3@5,tf32x3@9,bf16x3@9,tf32x3@13,bf16x3@13")
    ap.add_argument("--methods-run", action="store_true",
                    help="Triad-ATRG against ATRG (r = 7): step time and ln Z / V per chi")
    ap.add_argument("--methods-chis", default="8,12,16,18,20,24")
    ap.add_argument("--methods-steps", type=int, default=24)
    ap.add_argument("--c5-run", action="store_true",
                    help="derivatives at chi = 32, 32 steps against central differences")
    ap.add_argument("--c5-h", default="1e-3")
    ap.add_argument("--c5-eps", default="1e-5,1e-7,2e-7", help="difference steps of the first derivatives")
    ap.add_argument("--c5-eps2", default="1e-4,1e-6,2e-6", help="difference steps of the second derivative")
    ap.add_argument("--c5-reuse", action="store_true", help="keep stored tangents and differences")
    ap.add_argument("--c4-run", action="store_true", help="the 64-temperature sweep at chi = 32")
    ap.add_argument("--sweep-workers", type=int, default=8)
    ap.add_argument("--c4-serial", type=int, default=16,
                    help="runs timed one after another for the serial comparison (scaled to 64)")
    ap.add_argument("--d3-run", action="store_true", help="3D Ising runs over --d3-chis")
    ap.add_argument("--d3-chis", default="16,24,32,48,64")
    args = ap.parse_args()
    if args.c4_run:
        run_c4(args)
        return
    if args.d3_run:
        run_d3(args)
        return
    if args.c5_run:
        run_c5(args)
        return
    if args.methods_run:
        run_methods(args)
        return
    if args.c3_run:
        run_c3(args)
        return
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
