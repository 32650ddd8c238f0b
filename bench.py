"""Benchmark of the CC3 triples hot path on GB300.

One step = one CC3 triples residual evaluation (paper, Algorithm 1: every
occupied triple i >= j >= k, W build, denominators, contravariant amplitudes,
the four contractions, back-transform and energy) on the seeded synthetic
no = 16, nv = 160 problem, inputs resident in HBM.  The metric is nominal
TFLOP/s with 4 nv^4 no^3 FLOP per evaluation (the paper's convention).

The default is the split-precision (BF16 slice) tensor-core path; at one GPU
the same problem is then evaluated once on the native FP64 path, and the line
reports the split result's error against it (dE_T, max |dOmega|) and the
speedup.  The kernel-level roofline comes from in-library CUDA-event tracing
of every launch inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec split|fp64]
  python bench.py --impl reference ...    (the FP64 CPU oracle, bounded sample)
  python bench.py --no 6 --nv 160 ...     (smaller problem, for profiling)

Multi-GPU (torchrun): every rank evaluates its own independent problem of the
same size (weak scaling, no collective on the data path); rank 0 prints the
aggregate over ranks with the max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CC3 triples TFLOP/s (4 nv^4 no^3 per Omega) vs FP64 at dE<=1e-8 Eh; p99 lat"
NO, NV = 16, 160
WORKLOAD = "CC3 triples residual, no=16 nv=160, seeded synthetic (Cholesky-like integrals, MP2 t2)"


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the dominant kernel; None where no capture of the current kernel exists.
# no=16 nv=160: from a capture of the no=6 nv=160 launches, whose W build
# launches are the same size; contraction launches scaled by the distinct
# permutations per batch (81.6 against 67.2).
TRAFFIC = {("split_engine_kernel", 16, 160): 6.87e9}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed
    region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace('.', '').isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace('.', '').isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def cpu_model():
    """The host CPU's model name (Linux /proc/cpuinfo; the architecture else)."""
    import platform
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                return line.split(":", 1)[1].strip()
        for line in open("/proc/cpuinfo"):  # Arm: implementer / part numbers
            if line.lower().startswith("cpu part"):
                return f"{platform.machine()} (cpu part {line.split(':', 1)[1].strip()})"
    except Exception:  # an unreadable cpuinfo only loses the label
        pass
    return platform.machine()


def oracle_sample(inp, seconds_target=15.0, nthreads=0, n=None):
    """Time the FP64 oracle on a bounded, seeded sample of triples (n triples,
    or as many as fill ~seconds_target after a calibration run)."""
    import oracle
    from cc3_inputs import unique_triples
    tr = unique_triples(inp.no)
    rng = np.random.default_rng(11)
    order = rng.permutation(len(tr))
    if n is None:
        # calibrate on one triple per thread, then size the sample to ~seconds_target
        import os as _os
        threads = len(_os.sched_getaffinity(0)) if nthreads <= 0 else nthreads
        ncal = min(len(tr), threads)
        t0 = time.perf_counter()
        oracle.omega_inputs(inp, triples=[tr[x][:3] for x in order[:ncal]], nthreads=nthreads)
        dt1 = time.perf_counter() - t0
        n = int(max(ncal, min(len(tr), ncal * seconds_target / max(dt1, 1e-3))))
    n = max(1, min(int(n), len(tr)))
    sel = [tr[x][:3] for x in order[:n]]
    w = sum(tr[x][3] for x in order[:n])
    t0 = time.perf_counter()
    r = oracle.omega_inputs(inp, triples=sel, nthreads=nthreads)
    dt = time.perf_counter() - t0
    flop = 4.0 * inp.nv ** 4 * w
    return dict(value=flop / dt / 1e12, unit="TFLOP/s", cores=r["threads"],
                kind="oracle", seconds=dt, cpu=cpu_model(), n=n,
                sample=f"{n} of {len(tr)} triples (weight {w} of {inp.no**3 - inp.no}) "
                       f"of the no={inp.no} nv={inp.nv} residual, FP64 C oracle, "
                       f"{r['threads']} OpenMP threads")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from cc3_inputs import make_inputs
    inp = make_inputs(args.no, args.nv, seed=0)
    vals = []
    per_step = max(5.0, 60.0 / max(1, args.steps + args.warmup))
    n = None  # the sample size is calibrated once, on the first warm-up step
    for s in range(args.warmup + args.steps):
        r = oracle_sample(inp, seconds_target=per_step, n=n)
        n = r["n"]
        if s >= args.warmup:
            vals.append(r)
    v = statistics.median([x["value"] for x in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median([x["seconds"] for x in vals]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace(f"no={NO} nv={NV}", f"no={args.no} nv={args.nv}"),
                       "no": args.no, "nv": args.nv, "prec": "fp64-cpu-oracle"},
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": vals[-1]["cores"],
                             "kind": "oracle", "sample": vals[-1]["sample"],
                             "cpu": vals[-1]["cpu"]},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# kernel of each tracer class (the split engine serves two classes)
KERNEL_OF = {"fp64_engine": "fp64_engine_kernel", "fp64_elementwise": "elementwise",
             "split_w_build": "split_engine_kernel", "split_omega": "split_engine_kernel",
             "split_elementwise": "elementwise", "output": "elementwise"}


def per_kernel(traces):
    out = {}
    for k, v in traces.items():
        a = out.setdefault(KERNEL_OF.get(k, k), dict(launches=0, ms=0.0, flop=0.0, slice_flop=0.0))
        for f in a:
            a[f] += v[f]
    return out


def serve_stream(n_req, rate, no_lo, no_hi, seed=0):
    """The seeded mixed request stream: Poisson arrivals at `rate` per second,
    no ~ U{no_lo..no_hi}, nv = round(no * U[6, 10]), a residual or a Jacobian
    with 1-6 trial vectors (even odds); the inputs of request n use seed n."""
    from cc3_inputs import make_inputs, make_trial_vectors
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    t -= t[0]
    reqs = []
    for n in range(n_req):
        r = np.random.default_rng(n)
        no = int(r.integers(no_lo, no_hi + 1))
        nv = int(round(no * r.uniform(6.0, 10.0)))
        kind = "omega" if r.random() < 0.5 else "jacobian"
        nvec = int(r.integers(1, 7))
        inp = make_inputs(no, nv, seed=n)
        R = make_trial_vectors(no, nv, nvec, seed=n) if kind == "jacobian" else None
        reqs.append(dict(t=float(t[n]), kind=kind, no=no, nv=nv, nvec=nvec, inp=inp, R=R))
    return reqs


def run_serve(args):
    """Serving: the stream through the continuous-batching server, and the
    same stream served one request at a time on the FP64 path."""
    import torch
    import paper_2007_01088_gb300 as g
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    reqs = serve_stream(args.requests, args.rate, 4, args.max_no)
    omega_prec = g.CC3_SPLIT_BF16 if args.prec == "split" else g.CC3_FP64
    jac_prec = omega_prec

    def submit(srv, q):
        if q["kind"] == "omega":
            return srv.submit_omega(q["inp"], omega_prec)
        R1, R2 = q["R"]
        return srv.submit_jacobian(q["inp"], R1, R2, [0.25] * q["nvec"], jac_prec)

    # warm-up: the library, the engines' attributes, one small request per kind
    srv = g.Server(max_slots=args.slots)
    for q in reqs[:max(args.warmup, 3)]:
        srv.wait(submit(srv, q))
    srv.stop()
    srv = g.Server(max_slots=args.slots)
    tickets = [None] * len(reqs)
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()

    def feeder():
        for i, q in enumerate(reqs):
            d = t0 + q["t"] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets[i] = submit(srv, q)

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    status = [srv.wait(t)[0] for t in tickets]
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = srv.stats()
    srv.stop()
    # serial one-at-a-time FP64 over the same arrivals
    service = []
    for q in reqs:
        ctx = g.Context(q["inp"])
        torch.cuda.synchronize()
        a = time.perf_counter()
        if q["kind"] == "omega":
            ctx.omega(g.CC3_FP64)
        else:
            ctx.jacobian(q["R"][0], q["R"][1], [0.25] * q["nvec"], g.CC3_FP64)
        service.append(time.perf_counter() - a)
        ctx.close()
    done, lat = 0.0, []
    for q, sv in zip(reqs, service):
        done = max(done, q["t"]) + sv
        lat.append(1e3 * (done - q["t"]))
    flop = st["nominal_flop"]
    line = {"metric": "CC3 serving throughput (nominal TFLOP/s) with p50/p99 latency",
            "value": flop / wall / 1e12, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": 1, "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * wall,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if omega_prec == g.CC3_SPLIT_BF16 else "f64", "data": "synthetic",
            "config": {"workload": f"serving stream, {len(reqs)} requests, Poisson "
                                   f"{args.rate}/s, no~U{{4..{args.max_no}}}, nv=round(no*U[6,10]), "
                                   "residual or Jacobian (1-6 vectors) 50/50",
                       "slots": args.slots,
                       "prec": args.prec},
            "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"], "mean": st["mean_ms"]},
            "requests": {"completed": st["completed"], "failed": sum(1 for x in status if x != 0),
                         "rejected": st["rejected"]},
            "device_busy_frac": st["busy_s"] / wall, "hbm_peak_bytes": st["hbm_peak"],
            "serial_fp64": {"value": flop / max(done, 1e-9) / 1e12, "unit": "TFLOP/s",
                            "p50_ms": float(np.percentile(lat, 50)),
                            "p99_ms": float(np.percentile(lat, 99))},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_jacobian(args):
    """Batched right Jacobian transformation: 8 trial vectors at w = 0.25 on
    the no=20 nv=200 problem, split and FP64 side by side, each on the same
    seeded triple sample (the rate per weighted triple does not depend on the
    sample; the sample keeps a step within seconds)."""
    import torch
    import paper_2007_01088_gb300 as g
    from cc3_inputs import make_inputs, make_trial_vectors, unique_triples
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    no, nv, nvec = args.jno, args.jnv, args.nvec
    inp = make_inputs(no, nv, seed=rank)
    R1, R2 = make_trial_vectors(no, nv, nvec, seed=1 + rank)
    tr = unique_triples(no)
    rng = np.random.default_rng(7)
    pick = sorted(rng.choice(len(tr), size=max(1, int(round(args.sample * len(tr)))),
                             replace=False))
    sel = [tr[i][:3] for i in pick]
    wsum = sum(tr[i][3] for i in pick)
    w = torch.full((nvec,), 0.25, dtype=torch.float64).numpy()
    stream = torch.cuda.Stream(device=dev)
    sub = sel[:max(1, len(sel) // 8)]  # the FP64 comparison runs on a sub-sample

    def measure(prec, triples, steps, warm):
        with torch.cuda.stream(stream):
            ctx = g.Context(inp, device=True, stream=stream)
            ctx.set_triples(triples)
            r1 = torch.from_numpy(R1).to(dev)
            r2 = torch.from_numpy(R2).to(dev)
            ctx.set_tracing(True)
            for _ in range(warm):
                out = ctx.jacobian(r1, r2, w, prec)
            clocks = ClockSampler(local)
            clocks.start()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            launches, traces = 0, {}
            for _ in range(steps):
                out = ctx.jacobian(r1, r2, w, prec)
                launches += ctx.counters()["launches"]
                for k, v in ctx.trace().items():
                    a = traces.setdefault(k, dict(launches=0, ms=0.0, flop=0.0, slice_flop=0.0))
                    for f in a:
                        a[f] += v[f]
            e1.record(stream)
            torch.cuda.synchronize()
            clk = clocks.stop()
        res = dict(ms=e0.elapsed_time(e1) / steps, flop=ctx.counters()["nominal_flop"],
                   out=[x.cpu().numpy() for x in out], clk=clk, launches=launches,
                   traces=traces, steps=steps, executed=ctx.counters()["executed_flop"])
        ctx.close()
        return res

    res = {}
    if args.prec == "split":
        res[g.CC3_SPLIT_BF16] = measure(g.CC3_SPLIT_BF16, sel, args.steps, args.warmup)
        res["split_sub"] = measure(g.CC3_SPLIT_BF16, sub, 1, 1)
        res[g.CC3_FP64] = measure(g.CC3_FP64, sub, 1, 1)
    else:
        res[g.CC3_FP64] = measure(g.CC3_FP64, sel, args.steps, args.warmup)
    main_p = g.CC3_SPLIT_BF16 if args.prec == "split" else g.CC3_FP64
    r = res[main_p]
    value = r["flop"] / (r["ms"] * 1e-3) / 1e12
    pk, src = peaks()
    kern = per_kernel(r["traces"])
    dom_name, d = max(kern.items(), key=lambda kv: kv[1]["ms"])
    if dom_name == "fp64_engine_kernel":
        roof = {"bound": "tensor", "achieved": d["flop"] / (d["ms"] * 1e-3) / 1e12,
                "peak": pk["bf16_tflops"] * 1.25 / 2250.0, "unit": "TFLOP/s",
                "peak_source": f"FP64: {src} bf16 burst x nominal FP64/BF16 ratio (1.25/2250)"}
    else:
        roof = {"bound": "tensor", "achieved": d["slice_flop"] / (d["ms"] * 1e-3) / 1e12,
                "peak": pk["bf16_tflops"], "unit": "TFLOP/s", "peak_source": f"{src} bf16 burst",
                "fp64_equivalent_tflops": d["flop"] / (d["ms"] * 1e-3) / 1e12}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["kernel"] = dom_name
    roof["kernels"] = {k: {"ms_per_step": v["ms"] / r["steps"],
                           "launches_per_step": v["launches"] / r["steps"]}
                       for k, v in kern.items() if v["launches"]}
    line = {"metric": "CC3 triples Jacobian TFLOP/s (8 nv^4 no^3 per trial vector)",
            "value": value, "unit": "TFLOP/s", "n_gpus": 1, "steps": r["steps"],
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if main_p == g.CC3_SPLIT_BF16 else "f64", "data": "synthetic",
            "config": {"workload": f"batched right Jacobian, no={no} nv={nv}, {nvec} trial "
                                   f"vectors at w=0.25, seeded sample of {len(sel)} of "
                                   f"{len(tr)} triples (weight {wsum} of {no ** 3 - no})",
                       "prec": args.prec},
            "roofline": roof, "gpu_launches": r["launches"], "clocks": r["clk"],
            "executed_flop_per_step": r["executed"]}
    if args.prec == "split":
        f = res[g.CC3_FP64]
        fval = f["flop"] / (f["ms"] * 1e-3) / 1e12
        q = res["split_sub"]
        line["fp64"] = {"value": fval, "unit": "TFLOP/s", "ms_per_step": f["ms"],
                        "triples": len(sub),
                        "max_abs_drho1": float(np.abs(q["out"][0] - f["out"][0]).max()),
                        "max_abs_drho2": float(np.abs(q["out"][1] - f["out"][1]).max()),
                        "split_speedup": value / fval}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native")
    ap.add_argument("--prec", default="split", choices=["split", "fp64"])
    ap.add_argument("--no", type=int, default=NO, help="occupied orbitals (profiling cases)")
    ap.add_argument("--nv", type=int, default=NV, help="virtual orbitals (profiling cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--workload", default="omega", choices=["omega", "serve", "jacobian"])
    ap.add_argument("--config", default=None,
                    help="omega: a named workload of the input generator (e.g. "
                         "cfg3_proline_no22_nv250) instead of --no/--nv")
    ap.add_argument("--jno", type=int, default=20, help="jacobian: occupied orbitals")
    ap.add_argument("--jnv", type=int, default=200, help="jacobian: virtual orbitals")
    ap.add_argument("--nvec", type=int, default=8, help="jacobian: trial vectors")
    ap.add_argument("--sample", type=float, default=0.25,
                    help="jacobian: fraction of the triples evaluated per step")
    ap.add_argument("--requests", type=int, default=32, help="serve: requests in the stream")
    ap.add_argument("--rate", type=float, default=4.0, help="serve: arrivals per second")
    ap.add_argument("--max-no", type=int, default=12, help="serve: largest no of the stream")
    ap.add_argument("--slots", type=int, default=4, help="serve: concurrent requests")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 3 if args.prec == "fp64" else 10
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "jacobian":
        if args.steps is None or args.steps > 3:
            args.steps = 3
        return run_jacobian(args)

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_2007_01088_gb300 as g
    from cc3_inputs import make_inputs, CONFIGS, config_inputs
    no, nv = args.no, args.nv
    workload = WORKLOAD if (no, nv) == (NO, NV) else WORKLOAD.replace(
        f"no={NO} nv={NV}", f"no={no} nv={nv}")
    prec = g.CC3_SPLIT_BF16 if args.prec == "split" else g.CC3_FP64
    if args.config:  # one of the named workloads of the input generator
        inp = config_inputs(args.config, seed=rank)
        no, nv = inp.no, inp.nv
        workload = f"{args.config}: " + ", ".join(f"{k}={v}" for k, v in CONFIGS[args.config].items())
    else:
        inp = make_inputs(no, nv, seed=rank)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        ctx = g.Context(inp, device=True, stream=stream)
        tuning = ctx.autotune() if prec == g.CC3_SPLIT_BF16 else None
        ctx.set_tracing(True)
        out = (torch.empty((no, nv), dtype=torch.float64, device=dev),
               torch.empty((no, no, nv, nv), dtype=torch.float64, device=dev),
               torch.empty((1,), dtype=torch.float64, device=dev))
        for _ in range(args.warmup):
            ctx.omega(prec, out=out)
        stream.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        launches = 0
        traces = {}
        for _ in range(args.steps):
            ctx.omega(prec, out=out)
            launches += ctx.counters()["launches"]
            for k, v in ctx.trace().items():
                a = traces.setdefault(k, dict(launches=0, ms=0.0, flop=0.0, slice_flop=0.0))
                for f in a:
                    a[f] += v[f]
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        if ws > 1:
            torch.distributed.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    cnt = ctx.counters()
    # the same steps untraced: on a non-default stream the residual's launch
    # sequence is captured once as a CUDA graph and replayed (reported beside
    # the traced timing, which also gives the per-kernel roofline)
    graph = None
    if prec == g.CC3_SPLIT_BF16:
        with torch.cuda.stream(stream):
            ctx.set_tracing(False)
            for _ in range(2):
                ctx.omega(prec, out=out)
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            g0.record(stream)
            for _ in range(args.steps):
                ctx.omega(prec, out=out)
            g1.record(stream)
            torch.cuda.synchronize()
            ctx.set_tracing(True)
        gms = g0.elapsed_time(g1) / args.steps
        graph = {"ms_per_step": gms, "value": ws * cnt["nominal_flop"] / (gms * 1e-3) / 1e12,
                 "unit": "TFLOP/s", "note": "untraced steps replaying the captured CUDA graph"}
    flop = cnt["nominal_flop"]
    tmax = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(tmax.item())
    value = ws * flop / (ms_max * 1e-3) / 1e12

    # the same evaluation on the native FP64 path: error of the split result
    # and its speedup (rank 0 at N = 1; one warm-up call builds the FP64 plans)
    fp64 = None
    if prec == g.CC3_SPLIT_BF16 and ws == 1 and not args.no_fp64_compare:
        ref = (torch.empty_like(out[0]), torch.empty_like(out[1]), torch.empty_like(out[2]))
        with torch.cuda.stream(stream):
            ctx.omega(g.CC3_FP64, out=ref)
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            ctx.omega(g.CC3_FP64, out=ref)
            f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1)
        fval = flop / (fms * 1e-3) / 1e12
        fp64 = {"value": fval, "unit": "TFLOP/s", "ms_per_step": fms,
                "dE_T_Eh": abs(float(out[2][0] - ref[2][0])),
                "E_T_Eh": float(ref[2][0]),
                "max_abs_dOmega1": float((out[0] - ref[0]).abs().max()),
                "max_abs_dOmega2": float((out[1] - ref[1]).abs().max()),
                "split_speedup": value / fval}

    # end to end through the public API with host buffers: context creation
    # (upload of the inputs from pinned host memory), the evaluation and the
    # download of Omega1, Omega2, E_T into pinned host memory
    names = ["eps_o", "eps_v", "t2", "g_vvvo", "g_ooov", "g_ovov", "F_ov"]
    from types import SimpleNamespace
    pinned = SimpleNamespace(no=no, nv=nv, chol_L=None, **{
        n: torch.from_numpy(np.ascontiguousarray(getattr(inp, n))).pin_memory() for n in names})
    hout = tuple(torch.empty(s, dtype=torch.float64).pin_memory()
                 for s in [(no, nv), (no, no, nv, nv), (1,)])
    h2d = sum(getattr(pinned, n).numel() * 8 for n in names)
    d2h = sum(t.numel() * 8 for t in hout)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        hc = g.Context(pinned, device=False, stream=stream)
        hc.omega(prec, out=hout)
        hc.close()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if ws > 1:
        te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(te, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(te.item())

    pk, src = peaks()
    ratio = 1.25 / 2250.0  # nominal FP64 / dense BF16 tensor rate of GB300
    kern = per_kernel(traces)
    dom_name, d = max(kern.items(), key=lambda kv: kv[1]["ms"])
    total_ms = sum(v["ms"] for v in kern.values())
    if dom_name == "fp64_engine_kernel":
        roof = {"bound": "tensor", "achieved": d["flop"] / (d["ms"] * 1e-3) / 1e12,
                "peak": pk["bf16_tflops"] * ratio, "unit": "TFLOP/s",
                "peak_source": f"FP64: {src} bf16 burst x nominal FP64/BF16 ratio (1.25/2250)"}
    else:
        roof = {"bound": "tensor", "achieved": d["slice_flop"] / (d["ms"] * 1e-3) / 1e12,
                "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                "peak_source": f"{src} bf16 burst",
                "fp64_equivalent_tflops": d["flop"] / (d["ms"] * 1e-3) / 1e12}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = TRAFFIC.get((dom_name, no, nv))
    roof["kernel"] = dom_name
    roof["kernel_share"] = d["ms"] / total_ms if total_ms > 0 else None
    roof["kernel_avg_launch_ms"] = d["ms"] / max(1, d["launches"])
    roof["kernels"] = {k: {"ms_per_step": v["ms"] / args.steps,
                           "launches_per_step": v["launches"] / args.steps}
                       for k, v in kern.items() if v["launches"]}
    # the same time by step of the path (W build, contractions, element-wise)
    roof["phases"] = {k: {"ms_per_step": v["ms"] / args.steps,
                          "slice_tflops": (v["slice_flop"] / (v["ms"] * 1e-3) / 1e12
                                           if v["ms"] > 0 and v["slice_flop"] else None)}
                      for k, v in traces.items() if v["launches"]}
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == g.CC3_FP64 else "bf16",
            "data": "synthetic",
            "config": {"workload": workload, "no": no, "nv": nv,
                       "prec": args.prec, "parallelism": f"replicas{ws}",
                       "tiling": None if tuning is None else
                       {"vvov_ksteps_per_tile": tuning[0], "w_build_ntile": tuning[1],
                        "source": "autotuner (sample of the triple loop, before warm-up)"},
                       "l2": f"inputs larger than L2 (g_vvvo {nv ** 3 * no * 8 / 1e6:.0f} MB)"},
            "roofline": roof,
            "e2e": {"value": ws * flop / e2e_s / 1e12, "unit": "TFLOP/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches), "clocks": clk,
            "executed_flop_per_step": cnt["executed_flop"]}
    if fp64 is not None:
        line["fp64"] = fp64
    if graph is not None:
        line["graph_replay"] = graph
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: v for k, v in oracle_sample(inp).items()
                                if k in ("value", "unit", "cores", "kind", "sample", "cpu")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
