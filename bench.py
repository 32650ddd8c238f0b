"""Benchmark of the CC3 triples hot path on GB300.

One step = one CC3 triples residual evaluation (paper, Algorithm 1: every
occupied triple i >= j >= k, W build, denominators, contravariant amplitudes,
the four contractions, back-transform and energy) on the seeded synthetic
L-proline-sized problem (22 active occupied orbitals, nv = 250, naux = 700,
a near-degenerate virtual cluster), inputs resident in HBM.  The metric is
nominal TFLOP/s with 4 nv^4 (no^3 - no) FLOP per evaluation (the paper's
convention).  The default path is the split-precision (BF16 slice)
tensor-core path.

At one GPU the line then carries:
  roofline     the engine kernel's algorithmic TFLOP/s (the method's FLOP over
               its summed launch time, from in-library CUDA-event tracing of
               every launch in the timed region) against the measured BF16
               peak, with the slice-product utilisation beside it
  fp64         the FP64 path on a seeded triple sample: its rate, the split
               result's error against it, and both against the oracle on the
               cpu_baseline's triple sample
  e2e          the metric through the public API with pinned host buffers
  cpu_baseline the FP64 C oracle on a bounded seeded triple sample
  jacobian     the batched right Jacobian (8 trial vectors, no=20, nv=200)
  serving      the 256-request mixed serving stream with p50/p99 latency

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec split|fp64]
  python bench.py --impl reference ...    (the FP64 CPU oracle, bounded samples)
  python bench.py --no 6 --nv 160 ...     (smaller problem, for profiling)
  python bench.py --workload jacobian|serve   (one leg alone)

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
DEFAULT_CONFIG = "cfg3_proline_no22_nv250"
WORKLOADS = {
    "cfg1_no5_nv30": "CC3 triples residual (small parity case)",
    "cfg2_no16_nv160": "CC3 triples residual (acetamide-scale)",
    "cfg3_proline_no22_nv250": "L-proline-sized CC3 triples residual (22 active occupied "
                               "after freezing 9 core orbitals, near-degenerate cluster of 10 "
                               "virtual energies), seeded synthetic Cholesky-like integrals, "
                               "MP2 t2",
    "cfg4_jacobian_no20_nv200": "CC3 triples right Jacobian, 8 trial vectors",
}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the dominant kernel, averaged over the 668 engine launches of one residual
# evaluation of the benchmark workload (one-pass capture of the full
# workload); None where no capture of the current kernel exists.
TRAFFIC = {("split_engine_kernel", 22, 250): 15.562e9}
TRAFFIC_NOTE = {("split_engine_kernel", 22, 250):
                "mean of 334 W-build launches (8.00 GB read, 2.23 GB written) and 334 "
                "contraction launches (20.56 GB read, 0.34 GB written), 6 triples per batch"}


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


def oracle_sample(inp, seconds_target=15.0, nthreads=0, n=None, seed=11):
    """Time the FP64 oracle on a bounded, seeded sample of triples (n triples,
    or as many as fill ~seconds_target after a calibration run on one triple).
    Returns the rate, the sample and the oracle's result on it."""
    import oracle
    from cc3_inputs import unique_triples
    tr = unique_triples(inp.no)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(tr))
    if n is None:
        t0 = time.perf_counter()
        oracle.omega_inputs(inp, triples=[tr[order[0]][:3]], nthreads=nthreads)
        dt1 = time.perf_counter() - t0
        n = int(max(1, min(len(tr), seconds_target / max(dt1, 1e-3))))
    n = max(1, min(int(n), len(tr)))
    sel = [tuple(int(x) for x in tr[k][:3]) for k in order[:n]]
    w = sum(tr[k][3] for k in order[:n])
    t0 = time.perf_counter()
    r = oracle.omega_inputs(inp, triples=sel, nthreads=nthreads)
    dt = time.perf_counter() - t0
    flop = 4.0 * inp.nv ** 4 * w
    return dict(value=flop / dt / 1e12, unit="TFLOP/s", cores=r["threads"],
                kind="oracle", seconds=dt, cpu=cpu_model(), n=n, triples=sel, result=r,
                sample=f"{n} of {len(tr)} triples (weight {w} of {inp.no**3 - inp.no}) "
                       f"of the no={inp.no} nv={inp.nv} residual, FP64 C oracle, "
                       f"{r['threads']} OpenMP threads")


def blas_sample(inp, seconds_target=15.0, seed=12):
    """Time the BLAS-backed restatement of Algorithm 1 (the oracle's matrix
    form: one numpy matrix product per contraction, numpy's BLAS threads on
    the host cores) on a bounded, seeded sample of triples, sized from a
    calibration run on one triple.  The reordered integral copies are made
    before the timed region."""
    import oracle
    from oracle import matrix_form as MF
    from cc3_inputs import unique_triples
    tr = unique_triples(inp.no)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(tr))
    blocks = MF.Blocks(oracle.symmetric_blocks(inp))

    def run(sel):
        t0 = time.perf_counter()
        MF.omega(inp.no, inp.nv, inp.eps_o, inp.eps_v, inp.t2, blocks, triples=sel)
        return time.perf_counter() - t0

    dt1 = run([tr[order[0]][:3]])
    n = int(max(1, min(len(tr), seconds_target / max(dt1, 1e-3))))
    sel = [tuple(int(x) for x in tr[k][:3]) for k in order[:n]]
    w = sum(tr[k][3] for k in order[:n])
    dt = run(sel)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return dict(value=4.0 * inp.nv ** 4 * w / dt / 1e12, unit="TFLOP/s", cores=cores,
                kind="blas restatement of Algorithm 1 (numpy matrix products)",
                seconds=dt, cpu=cpu_model(),
                sample=f"{n} of {len(tr)} triples (weight {w} of {inp.no**3 - inp.no}) of "
                       f"the no={inp.no} nv={inp.nv} residual; numpy BLAS threads on "
                       f"{cores} host cores (transposes single-threaded)")


def workload_inputs(args, rank=0):
    """The bench's problem: a named workload of the input generator (default:
    the L-proline-sized residual) or --no/--nv."""
    from cc3_inputs import CONFIGS, config_inputs, make_inputs
    if args.no is not None or args.nv is not None:
        no = args.no if args.no is not None else 16
        nv = args.nv if args.nv is not None else 160
        return make_inputs(no, nv, seed=rank), (
            f"CC3 triples residual, no={no} nv={nv}, seeded synthetic "
            "(Cholesky-like integrals, MP2 t2)")
    name = args.config
    kw = CONFIGS[name]
    desc = WORKLOADS.get(name, "CC3 triples residual") + ", " + ", ".join(
        f"{k}={v}" for k, v in kw.items())
    return config_inputs(name, seed=rank), f"{name}: {desc}"


def run_reference(args):
    """The reference arm: the FP64 C oracle, as it stands, on the host cores,
    each step a bounded seeded triple sample of the same workload (the steps
    take different samples; the value is their median rate)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    inp, workload = workload_inputs(args)
    vals = []
    nsteps = args.warmup + args.steps
    per_step = max(2.0, 150.0 / max(1, nsteps))
    n = None  # the sample size is calibrated once, on the first warm-up step
    for s in range(nsteps):
        r = oracle_sample(inp, seconds_target=per_step, n=n, seed=100 + s)
        n = r["n"]
        if s >= args.warmup:
            vals.append(r)
    v = statistics.median([x["value"] for x in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median([x["seconds"] for x in vals]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "no": inp.no, "nv": inp.nv,
                       "prec": "fp64-cpu-oracle"},
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": vals[-1]["cores"],
                             "kind": "oracle", "sample": vals[-1]["sample"]
                             + f"; per step, {args.steps} steps with different seeded samples",
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


def serve_plan(n_req, rate, no_lo, no_hi, seed=0):
    """The seeded mixed request stream (without inputs): Poisson arrivals at
    `rate` per second, no ~ U{no_lo..no_hi}, nv = round(no * U[6, 10]), a
    residual or a Jacobian with 1-6 trial vectors (even odds).  Request n
    draws its sizes, and later its inputs, from seed n."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    t -= t[0]
    plan = []
    for n in range(n_req):
        r = np.random.default_rng(n)
        no = int(r.integers(no_lo, no_hi + 1))
        nv = int(round(no * r.uniform(6.0, 10.0)))
        kind = "omega" if r.random() < 0.5 else "jacobian"
        nvec = int(r.integers(1, 7))
        mult = 1 if kind == "omega" else 2 * nvec
        plan.append(dict(n=n, t=float(t[n]), kind=kind, no=no, nv=nv, nvec=nvec,
                         flop=4.0 * nv ** 4 * (no ** 3 - no) * mult,
                         bytes=8 * (2 * no * no * nv * nv + nv ** 3 * no + 2 * no ** 3 * nv
                                    + 3 * (no + nv) ** 3 + (nvec * no * no * nv * nv
                                                            if kind == "jacobian" else 0))))
    return plan


def serve_request(q):
    """The inputs of one planned request (seed n)."""
    from cc3_inputs import make_inputs, make_trial_vectors
    inp = make_inputs(q["no"], q["nv"], seed=q["n"])
    R = make_trial_vectors(q["no"], q["nv"], q["nvec"], seed=q["n"]) \
        if q["kind"] == "jacobian" else None
    return inp, R


def serve_stream(n_req, rate, no_lo, no_hi, seed=0):
    """serve_plan with every request's inputs drawn (small streams only)."""
    out = []
    for q in serve_plan(n_req, rate, no_lo, no_hi, seed):
        inp, R = serve_request(q)
        out.append(dict(q, inp=inp, R=R))
    return out


def serving(args, local, prec_name="split"):
    """The serving stream through the continuous-batching server.

    A client thread submits each request at its scheduled arrival time.  Its
    inputs are drawn just in time (the whole stream's inputs, ~190 GB at the
    full size, do not fit host memory at once): the client holds back while the
    requests in the system (submitted, not yet finished) keep more than
    `--serve-host-gb` of inputs, and a request drawn late is submitted late.
    Latency is measured from the scheduled arrival, so any such delay counts
    against the server.  A poller records each completion time.  Beside it, a
    serial one-at-a-time FP64 schedule of the same arrivals, with each
    request's service time extrapolated from its nominal FLOP and the FP64
    rate measured on a seeded subset of the requests."""
    import torch
    import paper_2007_01088_gb300 as g
    plan = serve_plan(args.requests, args.rate, args.min_no, args.max_no, seed=args.serve_seed)
    prec = g.CC3_SPLIT_BF16 if prec_name == "split" else g.CC3_FP64

    def submit(srv, q, inp, R):
        if q["kind"] == "omega":
            return srv.submit_omega(inp, prec)
        return srv.submit_jacobian(inp, R[0], R[1], [0.25] * q["nvec"], prec)

    torch.cuda.empty_cache()
    # warm-up: the library and the engines' attributes, one small request per kind
    srv = g.Server(max_slots=args.slots)
    for kind in ("omega", "jacobian"):
        q = dict(n=10 ** 6, t=0.0, kind=kind, no=4, nv=30, nvec=2)
        inp, R = serve_request(q)
        srv.wait(submit(srv, q, inp, R))
    srv.stop()
    cap = args.serve_host_gb * 1e9
    srv = g.Server(max_slots=args.slots)
    lock = threading.Lock()
    in_sys = {}        # ticket -> planned index, submitted and not finished
    held = [0.0]       # input bytes of those requests
    done_t = {}        # planned index -> completion time (s after t0)
    sub_t = {}         # planned index -> submit time
    status = {}
    backlog = [0]
    finished = threading.Event()
    t0 = time.perf_counter()

    def client():
        for q in plan:
            while True:
                with lock:
                    if held[0] == 0.0 or held[0] + q["bytes"] <= cap:
                        break
                time.sleep(0.02)
            inp, R = serve_request(q)
            d = t0 + q["t"] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tk = submit(srv, q, inp, R)
            with lock:
                sub_t[q["n"]] = time.perf_counter() - t0
                in_sys[tk] = q["n"]
                held[0] += q["bytes"]
            del inp, R

    def poller():
        while not finished.is_set() or in_sys:
            with lock:
                tks = list(in_sys.items())
            now = time.perf_counter() - t0
            arrived = sum(1 for q in plan if q["t"] <= now)
            backlog[0] = max(backlog[0], arrived - len(done_t))
            for tk, n in tks:
                if srv.poll(tk):
                    td = time.perf_counter() - t0
                    st, _ = srv.wait(tk)  # releases the request's outputs
                    with lock:
                        done_t[n] = td
                        status[n] = st
                        held[0] -= plan[n]["bytes"]
                        del in_sys[tk]
            time.sleep(0.02)

    clocks = ClockSampler(local)
    clocks.start()
    th_c = threading.Thread(target=client)
    th_p = threading.Thread(target=poller)
    th_c.start()
    th_p.start()
    th_c.join()
    finished.set()
    th_p.join()
    wall = max(done_t.values())
    clk = clocks.stop()
    st = srv.stats()
    srv.stop()
    lat = [1e3 * (done_t[q["n"]] - q["t"]) for q in plan]
    late = [sub_t[q["n"]] - q["t"] for q in plan]
    flop_ok = sum(q["flop"] for q in plan if status.get(q["n"]) == 0)
    # serial FP64: service rate per kind measured on a seeded subset of the
    # requests (those of at most --serve-fp64-max-flop, to keep it short)
    rng = np.random.default_rng(args.serve_seed + 1)
    small = [q for q in plan if q["flop"] <= args.serve_fp64_max_flop]
    rates, measured = {}, []
    for kind in ("omega", "jacobian"):
        cand = [q for q in small if q["kind"] == kind]
        pick = [cand[i] for i in rng.choice(len(cand), size=min(3, len(cand)), replace=False)]
        fl, sec = 0.0, 0.0
        for q in pick:
            inp, R = serve_request(q)
            ctx = g.Context(inp)
            if kind == "omega":
                ctx.omega(g.CC3_FP64)  # plans and workspace, then the timed call
                a = time.perf_counter()
                ctx.omega(g.CC3_FP64)
            else:
                ctx.jacobian(R[0][:1], R[1][:1], [0.25], g.CC3_FP64)
                a = time.perf_counter()
                ctx.jacobian(R[0], R[1], [0.25] * q["nvec"], g.CC3_FP64)
            torch.cuda.synchronize()
            sec += time.perf_counter() - a
            fl += q["flop"]
            ctx.close()
            measured.append(dict(n=q["n"], kind=kind, no=q["no"], nv=q["nv"], nvec=q["nvec"]))
        rates[kind] = fl / max(sec, 1e-9)
    done, slat = 0.0, []
    for q in plan:
        done = max(done, q["t"]) + q["flop"] / rates[q["kind"]]
        slat.append(1e3 * (done - q["t"]))
    n_fail = sum(1 for q in plan if status.get(q["n"]) != 0)
    return {
        "workload": f"serving stream, {len(plan)} requests, Poisson {args.rate}/s, "
                    f"no~U{{{args.min_no}..{args.max_no}}}, nv=round(no*U[6,10]), residual or "
                    "Jacobian (1-6 vectors at w=0.25) 50/50, request inputs seeded by id",
        "prec": prec_name, "slots": args.slots,
        "value": flop_ok / wall / 1e12, "unit": "TFLOP/s",
        "offered_tflops": sum(q["flop"] for q in plan) / max(plan[-1]["t"], 1e-9) / 1e12,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(np.mean(lat)),
                       "from": "scheduled arrival to completion seen by the client"},
        "server_latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"],
                              "from": "submit to completion inside the server"},
        "requests": {"completed": len(done_t) - n_fail, "failed": n_fail,
                     "rejected": st["rejected"]},
        "makespan_s": wall, "last_arrival_s": plan[-1]["t"],
        "backlog": {"max_requests_waiting": backlog[0],
                    "drain_after_last_arrival_s": wall - plan[-1]["t"]},
        "submit_delay_s": {"p50": float(np.percentile(late, 50)), "max": float(max(late)),
                           "note": f"client draws inputs just in time, <= "
                                   f"{args.serve_host_gb:g} GB of inputs in the system"},
        "device_busy_frac": st["busy_s"] / wall, "hbm_peak_bytes": st["hbm_peak"],
        "clocks": clk,
        "serial_fp64": {"value": sum(q["flop"] for q in plan) / done / 1e12, "unit": "TFLOP/s",
                        "p50_ms": float(np.percentile(slat, 50)),
                        "p99_ms": float(np.percentile(slat, 99)),
                        "kind": "extrapolation",
                        "rates_tflops": {k: v / 1e12 for k, v in rates.items()},
                        "note": "serial one-at-a-time FP64 over the same arrivals; each "
                                "request's service time = its nominal FLOP / the FP64 rate of "
                                "its kind measured on a seeded subset",
                        "measured": measured},
    }


def run_serve(args):
    """--workload serve: the serving stream alone, as its own line."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    r = serving(args, local, args.prec)
    line = {"metric": "CC3 serving throughput (nominal TFLOP/s) with p50/p99 latency",
            "value": r["value"], "unit": "TFLOP/s", "n_gpus": 1, "steps": 1,
            "warmup": 2, "ms_per_step": 1e3 * r["makespan_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if args.prec == "split" else "f64", "data": "synthetic",
            "config": {"workload": r["workload"], "slots": args.slots, "prec": args.prec},
            "serving": r, "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def jacobian_measure(args, local):
    """Batched right Jacobian transformation (eq. "jcc3"): `--nvec` trial
    vectors at w = 0.25 on the no=20 nv=200 workload, split path over a
    seeded fraction `--sample` of the triples (1: the whole loop), and the
    FP64 path on a smaller seeded sample (`--fp64-sample`) with the split
    result on the same triples for the error."""
    import torch
    import paper_2007_01088_gb300 as g
    from cc3_inputs import config_inputs, make_trial_vectors, unique_triples
    dev = torch.device("cuda", local)
    inp = config_inputs("cfg4_jacobian_no20_nv200")
    no, nv, nvec = inp.no, inp.nv, args.nvec
    R1, R2 = make_trial_vectors(no, nv, nvec, seed=1)
    tr = unique_triples(no)
    rng = np.random.default_rng(7)

    def pick(frac):
        if frac >= 1.0:
            return None, sum(t[3] for t in tr), len(tr)
        k = sorted(rng.choice(len(tr), size=max(1, int(round(frac * len(tr)))), replace=False))
        return [tr[i][:3] for i in k], sum(tr[i][3] for i in k), len(k)

    sel, wsel, nsel = pick(args.sample)
    sub, wsub, nsub = pick(args.fp64_sample)
    w = np.full(nvec, 0.25)
    stream = torch.cuda.Stream(device=dev)

    def measure(prec, triples, steps, warm):
        with torch.cuda.stream(stream):
            ctx = g.Context(inp, device=True, stream=stream)
            if triples is not None:
                ctx.set_triples(triples)
            r1 = torch.from_numpy(R1).to(dev)
            r2 = torch.from_numpy(R2).to(dev)
            ctx.set_tracing(True)
            for _ in range(warm):
                out = ctx.jacobian(r1, r2, w, prec)
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
        res = dict(ms=e0.elapsed_time(e1) / steps, flop=ctx.counters()["nominal_flop"],
                   out=[x.cpu().numpy() for x in out], launches=launches / steps,
                   traces=traces, steps=steps, executed=ctx.counters()["executed_flop"])
        ctx.close()
        return res

    r = measure(g.CC3_SPLIT_BF16, sel, args.jsteps, 1)
    value = r["flop"] / (r["ms"] * 1e-3) / 1e12
    pk, src = peaks()
    kern = per_kernel(r["traces"])
    eng = kern.get("split_engine_kernel", dict(ms=0.0, flop=0.0, slice_flop=0.0, launches=0))
    out = {"workload": f"batched right Jacobian, no={no} nv={nv} naux={inp.naux}, {nvec} trial "
                       f"vectors at w=0.25, " + ("the whole triple loop" if sel is None else
                                                f"seeded sample of {nsel} of {len(tr)} triples "
                                                f"(weight {wsel} of {no ** 3 - no})"),
           "value": value, "unit": "TFLOP/s", "ms_per_step": r["ms"], "steps": r["steps"],
           "launches_per_step": r["launches"],
           "executed_flop_per_step": r["executed"],
           "engine": {"ms_per_step": eng["ms"] / r["steps"],
                      "frac_of_bf16_sustained_algorithmic":
                          (r["flop"] / (eng["ms"] * 1e-3) / 1e12) / pk["bf16_tflops_sustained"]
                          if eng["ms"] else None,
                      "slice_utilisation_of_bf16_sustained":
                          (eng["slice_flop"] / (eng["ms"] * 1e-3) / 1e12)
                          / pk["bf16_tflops_sustained"] if eng["ms"] else None},
           "kernels": {k: {"ms_per_step": v["ms"] / r["steps"],
                           "launches_per_step": v["launches"] / r["steps"]}
                       for k, v in kern.items() if v["launches"]}}
    if args.fp64_sample > 0:
        f = measure(g.CC3_FP64, sub, 1, 0)
        q = measure(g.CC3_SPLIT_BF16, sub, 1, 0)
        fval = f["flop"] / (f["ms"] * 1e-3) / 1e12
        qval = q["flop"] / (q["ms"] * 1e-3) / 1e12
        out["fp64"] = {"value": fval, "unit": "TFLOP/s", "ms_per_step": f["ms"],
                       "sample": f"seeded sample of {nsub} triples (weight {wsub})",
                       "split_value_same_sample": qval,
                       "max_abs_drho1": float(np.abs(q["out"][0] - f["out"][0]).max()),
                       "max_abs_drho2": float(np.abs(q["out"][1] - f["out"][1]).max()),
                       "max_abs_rho2": float(np.abs(f["out"][1]).max()),
                       "split_speedup": qval / fval}
    return out


def density_measure(args, local):
    """Triples contributions of Algorithm 3 to the one-electron density of a
    left state: no=12, nv=120, a seeded left vector normalised like the trial
    vectors at w = 0.25, one warm-up call and `--dsteps` timed calls per path
    with inputs and outputs resident on the device.  The split (BF16 slice)
    path gives the figures, with its largest deviation from the FP64
    densities; the FP64 path is reported beside it (`fp64`)."""
    import torch
    import paper_2007_01088_gb300 as g
    from cc3_inputs import make_inputs, make_trial_vectors
    dev = torch.device("cuda", local)
    no, nv = args.density_no, args.density_nv
    inp = make_inputs(no, nv, seed=5)
    L1, L2 = make_trial_vectors(no, nv, 1, seed=6)
    stream = torch.cuda.Stream(device=dev)
    pk, src = peaks()
    fp64_peak = pk["bf16_tflops_sustained"] * 1.25 / 2250.0

    def one(ctx, l1, l2, prec):
        ctx.set_tracing(True)
        ctx.density(l1, l2, 0.25, prec=prec)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        traces, launches = {}, 0
        for _ in range(args.dsteps):
            out = ctx.density(l1, l2, 0.25, prec=prec)
            launches += ctx.counters()["launches"]
            for k, v in ctx.trace().items():
                a = traces.setdefault(k, dict(launches=0, ms=0.0, flop=0.0, slice_flop=0.0))
                for f in a:
                    a[f] += v[f]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.dsteps
        cnt = ctx.counters()
        kern = per_kernel(traces)
        r = {"value": cnt["nominal_flop"] / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
             "ms_per_step": ms, "steps": args.dsteps,
             "nominal_flop_per_step": cnt["nominal_flop"],
             "executed_flop_per_step": cnt["executed_flop"],
             "launches_per_step": launches / args.dsteps,
             "kernels": {k: {"ms_per_step": v["ms"] / args.dsteps,
                             "launches_per_step": v["launches"] / args.dsteps}
                         for k, v in kern.items() if v["launches"]}}
        return r, kern, [x.cpu().numpy() for x in out]

    with torch.cuda.stream(stream):
        ctx = g.Context(inp, device=True, stream=stream)
        l1 = torch.from_numpy(L1[0]).to(dev)
        l2 = torch.from_numpy(L2[0]).to(dev)
        r, kern, (doo, dov, dvv) = one(ctx, l1, l2, g.CC3_FP64)
        eng = kern.get("fp64_engine_kernel", dict(ms=0.0, flop=0.0, launches=0))
        r["fp64_engine"] = {"ms_per_step": eng["ms"] / args.dsteps,
                            "achieved_tflops": eng["flop"] / (eng["ms"] * 1e-3) / 1e12
                            if eng["ms"] else None,
                            "peak_tflops": fp64_peak,
                            "peak_source": f"{src} bf16 sustained x nominal FP64/BF16 (1.25/2250)"}
        split, _, (soo, sov, svv) = one(ctx, l1, l2, g.CC3_SPLIT_BF16)
        ctx.close()
    split["max_abs_dev_from_fp64"] = {
        "D_oo": float(np.abs(soo - doo).max()), "D_ov": float(np.abs(sov - dov).max()),
        "D_vv": float(np.abs(svv - dvv).max())}
    split["max_abs"] = {"D_oo": float(np.abs(doo).max()), "D_ov": float(np.abs(dov).max()),
                        "D_vv": float(np.abs(dvv).max())}
    split["workload"] = (f"triples density of a left state (Algorithm 3), no={no} nv={nv}, "
                         "w=0.25, split (BF16 slice) path, seeded synthetic inputs and a "
                         "normalised left vector")
    r["trace_D_vv_plus_trace_D_oo"] = float(np.trace(dvv) + np.trace(doo))
    r["trace_D_vv"] = float(np.trace(dvv))
    split["fp64"] = r
    return split


def _timed_calls(stream, fn, steps):
    """CUDA-event time of `steps` calls of fn on `stream` (ms per call)."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, out


def widening_measure(args, local):
    """The NEXT rows besides the densities, each on one seeded problem with
    inputs resident on the device, one warm-up and one timed call:
    - the left (transpose) Jacobian: FP64 path at no=12 nv=120 with 2 left
      vectors, split path on the batched-Jacobian workload with 8;
    - the core-valence separation filter: the batched Jacobian workload
      (no=20, nv=200, 8 vectors) restricted to the triples that contain
      occupied orbital 0, split path;
    - general (non-symmetric) five-block integrals: the residual on seeded
      symmetric blocks plus a seeded non-symmetric perturbation of 1e-3 of
      each block's scale, split path, no=16 nv=160."""
    import torch
    import paper_2007_01088_gb300 as g
    from cc3_inputs import config_inputs, make_inputs, make_trial_vectors
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    out = {}
    with torch.cuda.stream(stream):
        # left Jacobian
        no, nv, nvec = 12, 120, 2
        inp = make_inputs(no, nv, seed=21)
        rng = np.random.default_rng(22)
        L2 = rng.normal(size=(nvec, no, no, nv, nv))
        L2 = 0.5 * (L2 + np.transpose(L2, (0, 2, 1, 4, 3)))
        l1 = torch.from_numpy(rng.normal(size=(nvec, no, nv))).to(dev)
        l2 = torch.from_numpy(L2).to(dev)
        w = [0.25, 0.1]
        ctx = g.Context(inp, device=True, stream=stream)
        ctx.left_jacobian(l1, l2, w)
        ms, _ = _timed_calls(stream, lambda: ctx.left_jacobian(l1, l2, w), 1)
        flop = ctx.counters()["nominal_flop"]
        ctx.close()
        out["left_jacobian"] = {
            "workload": f"left (transpose) Jacobian, no={no} nv={nv} naux={inp.naux}, {nvec} "
                        "left vectors at w=0.25, 0.1, FP64 path",
            "value": flop / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
            "nominal_flop_per_step": flop}
        # the split path on the batched-Jacobian workload, 8 left vectors
        inp = config_inputs("cfg4_jacobian_no20_nv200")
        no, nv, nvec = inp.no, inp.nv, 8
        A1, A2 = make_trial_vectors(no, nv, nvec, seed=23)
        a1, a2 = torch.from_numpy(A1).to(dev), torch.from_numpy(A2).to(dev)
        wv = np.full(nvec, 0.25)
        ctx = g.Context(inp, device=True, stream=stream)
        ctx.left_jacobian(a1, a2, wv, g.CC3_SPLIT_BF16)
        ms, _ = _timed_calls(stream, lambda: ctx.left_jacobian(a1, a2, wv, g.CC3_SPLIT_BF16), 1)
        flop = ctx.counters()["nominal_flop"]
        # one traced call: device time per kernel class (the timed call above is untraced)
        ctx.set_tracing(True)
        ctx.left_jacobian(a1, a2, wv, g.CC3_SPLIT_BF16)
        phases = {k: {"ms": v["ms"], "launches": v["launches"]} for k, v in ctx.trace().items()
                  if v["launches"]}
        ctx.close()
        out["left_jacobian"]["split"] = {
            "workload": f"left (transpose) Jacobian, no={no} nv={nv} naux={inp.naux}, {nvec} "
                        "left vectors at w=0.25, the whole triple loop, split path",
            "value": flop / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
            "nominal_flop_per_step": flop, "phases_traced_call": phases}
        torch.cuda.empty_cache()
        # CVS filter
        inp = config_inputs("cfg4_jacobian_no20_nv200")
        no, nv, nvec = inp.no, inp.nv, 8
        R1, R2 = make_trial_vectors(no, nv, nvec, seed=1)
        r1, r2 = torch.from_numpy(R1).to(dev), torch.from_numpy(R2).to(dev)
        wv = np.full(nvec, 0.25)
        ctx = g.Context(inp, device=True, stream=stream)
        tr = ctx.set_cvs([0])
        ctx.jacobian(r1, r2, wv, g.CC3_SPLIT_BF16)
        ms, _ = _timed_calls(stream, lambda: ctx.jacobian(r1, r2, wv, g.CC3_SPLIT_BF16), 1)
        flop = ctx.counters()["nominal_flop"]
        ctx.close()
        out["cvs"] = {
            "workload": f"core-valence separation: the batched Jacobian (no={no}, nv={nv}, "
                        f"{nvec} vectors at w=0.25) on the {len(tr)} triples that contain "
                        "occupied orbital 0, split path",
            "value": flop / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
            "nominal_flop_per_step": flop, "triples": len(tr)}
        torch.cuda.empty_cache()
        # general integrals
        no, nv = 16, 160
        inp = make_inputs(no, nv, seed=31)
        rng = np.random.default_rng(32)
        # the five blocks of the symmetric problem (oovo = (lj|kc) reordered,
        # vvov = (bd|ck) reordered), then perturbed out of symmetry
        blocks = {"vvvo": inp.g_vvvo, "oovo": np.transpose(inp.g_ooov, (0, 1, 3, 2)),
                  "ooov": inp.g_ooov, "ovov": inp.g_ovov,
                  "vvov": np.transpose(inp.g_vvvo, (1, 0, 3, 2)), "F_ov": inp.F_ov}
        for k in ("vvvo", "oovo", "ooov", "ovov", "vvov"):
            x = blocks[k]
            blocks[k] = np.ascontiguousarray(x + 1e-3 * np.abs(x).max() * rng.normal(size=x.shape))
        ctx = g.Context(inp, device=True, stream=stream, blocks=blocks)
        ctx.omega(g.CC3_SPLIT_BF16)
        ms, _ = _timed_calls(stream, lambda: ctx.omega(g.CC3_SPLIT_BF16), 3)
        flop = ctx.counters()["nominal_flop"]
        ctx.close()
        out["general_integrals"] = {
            "workload": f"residual on general (non-symmetric) five-block integrals, no={no} "
                        f"nv={nv}, split path",
            "value": flop / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
            "nominal_flop_per_step": flop}
    torch.cuda.empty_cache()
    return out


def run_density(args):
    """--workload density: the Algorithm 3 densities alone, as their own line."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    clocks = ClockSampler(local)
    clocks.start()
    r = density_measure(args, local)
    clk = clocks.stop()
    line = {"metric": "CC3 triples density TFLOP/s (Algorithm 3 FLOP per left state)",
            "value": r["value"], "unit": "TFLOP/s", "n_gpus": 1, "steps": r["steps"],
            "warmup": 1, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": r["workload"]}, "density": r, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_jacobian(args):
    """--workload jacobian: the batched Jacobian alone, as its own line."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    clocks = ClockSampler(local)
    clocks.start()
    r = jacobian_measure(args, local)
    clk = clocks.stop()
    line = {"metric": "CC3 triples Jacobian TFLOP/s (8 nv^4 no^3 per trial vector)",
            "value": r["value"], "unit": "TFLOP/s", "n_gpus": 1, "steps": r["steps"],
            "warmup": 1, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": r["workload"]}, "jacobian": r, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native")
    ap.add_argument("--prec", default="split", choices=["split", "fp64"])
    ap.add_argument("--config", default=DEFAULT_CONFIG,
                    help="the residual's workload, a named workload of the input generator")
    ap.add_argument("--no", type=int, default=None, help="occupied orbitals (profiling cases; "
                                                         "replaces --config)")
    ap.add_argument("--nv", type=int, default=None, help="virtual orbitals (profiling cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-jacobian", action="store_true", help="skip the batched-Jacobian leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-density", action="store_true", help="skip the density leg")
    ap.add_argument("--no-widening", action="store_true",
                    help="skip the left-Jacobian, CVS and general-integral legs")
    ap.add_argument("--density-no", type=int, default=12, help="density: occupied orbitals")
    ap.add_argument("--density-nv", type=int, default=120, help="density: virtual orbitals")
    ap.add_argument("--dsteps", type=int, default=1, help="density: timed calls")
    ap.add_argument("--compare-triples", type=int, default=24,
                    help="seeded triple sample of the split-vs-FP64 comparison")
    ap.add_argument("--workload", default="omega",
                    choices=["omega", "serve", "jacobian", "density"])
    ap.add_argument("--nvec", type=int, default=8, help="jacobian: trial vectors")
    ap.add_argument("--sample", type=float, default=1.0,
                    help="jacobian: fraction of the triples of the split measurement")
    ap.add_argument("--fp64-sample", type=float, default=1.0 / 64,
                    help="jacobian: fraction of the triples of the FP64 comparison (0: none)")
    ap.add_argument("--jsteps", type=int, default=2, help="jacobian: timed steps")
    ap.add_argument("--requests", type=int, default=256, help="serve: requests in the stream")
    ap.add_argument("--rate", type=float, default=4.0, help="serve: arrivals per second")
    ap.add_argument("--min-no", type=int, default=4, help="serve: smallest no of the stream")
    ap.add_argument("--max-no", type=int, default=24, help="serve: largest no of the stream")
    ap.add_argument("--slots", type=int, default=4, help="serve: concurrent requests")
    ap.add_argument("--serve-seed", type=int, default=0, help="serve: arrival-time seed")
    ap.add_argument("--serve-host-gb", type=float, default=48.0,
                    help="serve: cap on the inputs held by requests in the system")
    ap.add_argument("--serve-fp64-max-flop", type=float, default=3e12,
                    help="serve: largest request of the FP64 rate sample")
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
        return run_jacobian(args)
    if args.workload == "density":
        return run_density(args)
    return run_omega(args)


def run_omega(args):
    """The headline: the triples residual (Algorithm 1) on the workload, each
    step one whole evaluation, inputs resident in HBM; at N = 1 (rank 0) the
    comparison legs, the batched Jacobian and the serving stream follow."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_2007_01088_gb300 as g
    prec = g.CC3_SPLIT_BF16 if args.prec == "split" else g.CC3_FP64
    inp, workload = workload_inputs(args, rank)
    no, nv = inp.no, inp.nv
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
    flop = cnt["nominal_flop"]
    tmax = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(tmax.item())
    value = ws * flop / (ms_max * 1e-3) / 1e12
    # untraced steps: on a non-default stream the residual's launch sequence is
    # captured once as a CUDA graph and replayed
    graph = None
    if prec == g.CC3_SPLIT_BF16:
        with torch.cuda.stream(stream):
            ctx.set_tracing(False)
            for _ in range(2):
                ctx.omega(prec, out=out)
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            gsteps = min(args.steps, 3)
            torch.cuda.synchronize()
            g0.record(stream)
            for _ in range(gsteps):
                ctx.omega(prec, out=out)
            g1.record(stream)
            torch.cuda.synchronize()
            ctx.set_tracing(True)
        gms = g0.elapsed_time(g1) / gsteps
        graph = {"ms_per_step": gms, "value": ws * flop / (gms * 1e-3) / 1e12,
                 "unit": "TFLOP/s", "steps": gsteps,
                 "note": "untraced steps replaying the captured CUDA graph"}
    pk, src = peaks()
    kern = per_kernel(traces)
    dom_name, d = max(kern.items(), key=lambda kv: kv[1]["ms"])
    total_ms = sum(v["ms"] for v in kern.values())
    if dom_name == "fp64_engine_kernel":
        ratio = 1.25 / 2250.0  # nominal FP64 / dense BF16 tensor rate of GB300
        roof = {"bound": "tensor", "achieved": d["flop"] / (d["ms"] * 1e-3) / 1e12,
                "peak": pk["bf16_tflops_sustained"] * ratio, "unit": "TFLOP/s",
                "peak_source": f"FP64: {src} bf16 sustained x nominal FP64/BF16 ratio "
                               "(1.25/2250)"}
    else:
        # algorithmic FLOP: the nominal 4 nv^4 (no^3 - no) of the step, all of
        # it in the engine's launches, over the engine's summed launch time
        roof = {"bound": "tensor", "achieved": flop * args.steps / (d["ms"] * 1e-3) / 1e12,
                "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                "peak_source": f"{src} bf16 sustained (the engine runs inside a long step)",
                "slice_tflops": d["slice_flop"] / (d["ms"] * 1e-3) / 1e12,
                "slice_utilisation": d["slice_flop"] / (d["ms"] * 1e-3) / 1e12
                / pk["bf16_tflops_sustained"],
                "slice_products_per_useful_flop": d["slice_flop"] / max(d["flop"], 1.0),
                "note": "frac counts the method's 4 nv^4 (no^3-no) FLOP; slice_utilisation "
                        "counts the BF16 slice products the engine executes"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = TRAFFIC.get((dom_name, no, nv))
    roof["traffic_note"] = TRAFFIC_NOTE.get((dom_name, no, nv))
    roof["kernel"] = dom_name
    roof["kernel_share"] = d["ms"] / total_ms if total_ms > 0 else None
    roof["kernel_avg_launch_ms"] = d["ms"] / max(1, d["launches"])
    roof["kernels"] = {k: {"ms_per_step": v["ms"] / args.steps,
                           "launches_per_step": v["launches"] / args.steps}
                       for k, v in kern.items() if v["launches"]}
    roof["phases"] = {k: {"ms_per_step": v["ms"] / args.steps,
                          "slice_tflops": (v["slice_flop"] / (v["ms"] * 1e-3) / 1e12
                                           if v["ms"] > 0 and v["slice_flop"] else None)}
                      for k, v in traces.items() if v["launches"]}
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == g.CC3_FP64 else "bf16",
            "data": "synthetic",
            "config": {"workload": workload, "no": no, "nv": nv, "naux": inp.naux,
                       "prec": args.prec, "parallelism": f"replicas{ws}",
                       "tiling": None if tuning is None else
                       {"vvov_ksteps_per_tile": tuning[0], "w_build_ntile": tuning[1],
                        "source": "autotuner (sample of the triple loop, before warm-up)"},
                       "l2": f"inputs larger than L2 (g_vvvo {nv ** 3 * no * 8 / 1e6:.0f} MB)"},
            "roofline": roof, "gpu_launches": int(launches), "clocks": clk,
            "executed_flop_per_step": cnt["executed_flop"]}
    if graph is not None:
        line["graph_replay"] = graph
    one = rank == 0 and ws == 1
    # cpu_baseline: the oracle on a bounded seeded triple sample; the split and
    # FP64 paths on the same triples give the error against the oracle
    sample = None
    if one and not args.no_cpu_baseline:
        sample = oracle_sample(inp)
        line["cpu_baseline"] = {k: v for k, v in sample.items()
                                if k in ("value", "unit", "cores", "kind", "sample", "cpu")}
        blas = blas_sample(inp)
        line["cpu_baseline"]["blas"] = {k: v for k, v in blas.items()
                                        if k in ("value", "unit", "cores", "kind", "sample")}
    # the split path against the FP64 path (seeded triple sample) and both
    # against the oracle (the cpu_baseline sample)
    if one and prec == g.CC3_SPLIT_BF16 and not args.no_fp64_compare:
        line["fp64"] = compare_paths(g, ctx, stream, inp, out, args.compare_triples, sample)
    ctx.close()
    del ctx
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if not args.no_e2e:
        line["e2e"] = end_to_end(g, inp, prec, stream, args.steps, ws, dev)
    if one and not args.no_jacobian:
        line["jacobian"] = jacobian_measure(args, local)
        torch.cuda.empty_cache()
    if one and not args.no_density:
        line["density"] = density_measure(args, local)
        torch.cuda.empty_cache()
    if one and not args.no_widening:
        line.update(widening_measure(args, local))
    if one and not args.no_serve:
        line["serving"] = serving(args, local, args.prec)
        s = line["serving"]
        line["latency_ms"] = {"p50": s["latency_ms"]["p50"], "p99": s["latency_ms"]["p99"],
                              "source": "serving stream (see serving)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def compare_paths(g, ctx, stream, inp, out, ntri, sample):
    """Split vs FP64 on a seeded triple sample of the same context (with the
    FP64 rate on it), and both against the oracle's result on its sample."""
    import torch
    from cc3_inputs import unique_triples
    tr = unique_triples(inp.no)
    rng = np.random.default_rng(23)
    pick = sorted(rng.choice(len(tr), size=min(ntri, len(tr)), replace=False))
    sel = [tr[i][:3] for i in pick]
    wsel = sum(tr[i][3] for i in pick)
    res = {}
    ref = tuple(torch.empty_like(x) for x in out)
    with torch.cuda.stream(stream):
        ctx.set_tracing(False)
        ctx.set_triples(sel)
        ctx.omega(g.CC3_SPLIT_BF16, out=out)
        ctx.omega(g.CC3_FP64, out=ref)  # plans and workspace of the FP64 path
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        ctx.omega(g.CC3_FP64, out=ref)
        f1.record(stream)
        torch.cuda.synchronize()
    fms = f0.elapsed_time(f1)
    fflop = 4.0 * inp.nv ** 4 * wsel
    res = {"value": fflop / (fms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms": fms,
           "sample": f"seeded sample of {len(sel)} of {len(tr)} triples (weight {wsel})",
           "dE_T_Eh": abs(float(out[2][0] - ref[2][0])), "E_T_Eh_sample": float(ref[2][0]),
           "max_abs_dOmega1": float((out[0] - ref[0]).abs().max()),
           "max_abs_dOmega2": float((out[1] - ref[1]).abs().max()),
           "max_abs_Omega2": float(ref[1].abs().max())}
    if sample is not None:
        r = sample["result"]
        with torch.cuda.stream(stream):
            ctx.set_triples(sample["triples"])
            ctx.omega(g.CC3_SPLIT_BF16, out=out)
            ctx.omega(g.CC3_FP64, out=ref)
            torch.cuda.synchronize()
        vs = {}
        for name, o in (("split", out), ("fp64", ref)):
            vs[name] = {"dE_T_Eh": abs(float(o[2][0]) - r["E_T"]),
                        "max_abs_dOmega1": float(np.abs(o[0].cpu().numpy() - r["omega1"]).max()),
                        "max_abs_dOmega2": float(np.abs(o[1].cpu().numpy() - r["omega2"]).max())}
        vs["sample"] = sample["sample"]
        vs["E_T_Eh_sample"] = r["E_T"]
        vs["max_abs_Omega2"] = float(np.abs(r["omega2"]).max())
        res["vs_oracle"] = vs
    ctx.set_triples(None)
    return res


def end_to_end(g, inp, prec, stream, steps, ws, dev):
    """The same metric through the public API with pinned host buffers: each
    step creates a context (upload of the inputs), evaluates and downloads
    Omega1, Omega2 and E_T."""
    import torch
    from types import SimpleNamespace
    no, nv = inp.no, inp.nv
    names = ["eps_o", "eps_v", "t2", "g_vvvo", "g_ooov", "g_ovov", "F_ov"]
    pinned = SimpleNamespace(no=no, nv=nv, chol_L=None, **{
        n: torch.from_numpy(np.ascontiguousarray(getattr(inp, n))).pin_memory() for n in names})
    hout = tuple(torch.empty(s, dtype=torch.float64).pin_memory()
                 for s in [(no, nv), (no, no, nv, nv), (1,)])
    h2d = sum(getattr(pinned, n).numel() * 8 for n in names)
    d2h = sum(t.numel() * 8 for t in hout)
    e2e_steps = max(1, min(steps, 3))
    flop = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        hc = g.Context(pinned, device=False, stream=stream)
        hc.omega(prec, out=hout)
        flop = hc.counters()["nominal_flop"]
        hc.close()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if ws > 1:
        te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(te, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(te.item())
    return {"value": ws * flop / e2e_s / 1e12, "unit": "TFLOP/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": e2e_steps, "ms_per_step": 1e3 * e2e_s}


if __name__ == "__main__":
    sys.exit(main())
