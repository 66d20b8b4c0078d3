#!/usr/bin/env python
"""Benchmark: ensembles of adaptive tau-leaping trajectories on one GPU per rank.

Workload (default): the batched particle-filter workload -- two-state gene expression,
3 species, 6 reactions, per-trajectory rate constants theta_j ~ Gamma(2, 2/theta_true_j)
and horizons T ~ U[50, 200], x0 = 0, eps = 0.03, n_c = 10, 1,000,000 trajectories per GPU
(weak scaling: rank k simulates trajectory ids [k B, (k+1) B)).  --config selects another
workload (0 immigration-death, 1 stiff dimerisation, 3 random 50 x 100 network).

A step is one simulate call over the whole batch.  Two forms are timed:
  batched  fast precision (FP32 propensities, step sizes, Poisson means and G
           increments; FP64 time, G totals and implicit Newton solve), persistent refill
           kernel compiled for the model at run time, launched from a CUDA graph, shape
           autotuned on the whole batch  -> the headline `value`;
  plain    reference precision (FP64 everywhere), one launch, one thread per trajectory
           (`plain_fp64`, timed for at most --plain-budget-s seconds, at least 2 steps).
Inputs are resident in HBM when timing starts; a 256 MB buffer is written between steps to
flush L2.  `e2e` times the host-buffer entry point (pinned host memory, copies inside).
`cpu_baseline` times the CPU oracle on one host core on a bounded sample and
`cpu_baseline_all_cores` as one process per core; `parity` compares the last timed step
with the oracle on the same ids; `roofline` reports the algorithmic and the issue-rate
view; `other_workloads` repeats the fast form with FP64 and FP32 Newton solves and the
plain form on the stiff dimerisation; `pipe_peaks` the measured pipe throughputs,
`bayes_step` the posterior draw and resampling, `accuracy` the paper's KL study (Section 3,
Table 1), `serving` the continuous-batching mix.
`--impl reference` times only the oracle (the reference arm for this method).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "trajectories/s & leap-steps/s, batched vs plain launch, at oracle-matched stats"
MAX_STEPS = 1_000_000
_T0 = time.perf_counter()


def stage(msg):
    """Progress of the run on stderr (the JSON line is the only stdout output)."""
    sys.stderr.write(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}\n")
    sys.stderr.flush()


def guarded(line, key, fn):
    """Runs one optional leg; its failure is recorded in the line instead of losing the
    headline measurement."""
    stage(f"{key} ...")
    try:
        v = fn()
        if v is not None:
            line[key] = v
    except Exception as e:  # noqa: BLE001 - recorded, the headline still prints
        line[key] = {"error": f"{type(e).__name__}: {e}"[:300]}
        stage(f"{key} failed: {e}")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--n-traj", type=int, default=None)
    ap.add_argument("--horizon", type=float, default=None,
                    help="override the workload's horizon T (one value for every trajectory)")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0,
                    help="target CPU seconds for the oracle baseline sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--jacobian", choices=["fd", "analytic"], default="fd",
                    help="Jacobian of the implicit solve, same for both forms")
    ap.add_argument("--newton", choices=["fp64", "fp32"], default="fp64",
                    help="arithmetic of the fast precision's implicit Newton solve")
    ap.add_argument("--plain-budget-s", type=float, default=60.0,
                    help="the plain FP64 form stops timing after this many seconds (>= 2 steps)")
    ap.add_argument("--e2e-budget-s", type=float, default=20.0,
                    help="the end-to-end leg stops timing after this many seconds (>= 2 steps)")
    ap.add_argument("--extra-configs", default="1",
                    help="comma-separated workloads measured beside the headline")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-order", action="store_true",
                    help="hand trajectories out in index order (no longest-first queue order)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--plain-n-traj", type=int, default=None,
                    help="time the plain FP64 form on this prefix of the batch (slow workloads)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--generic", action="store_true",
                    help="batched form on the precompiled kernels (no model-specialized kernels)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default launch shape (for very long workloads)")
    ap.add_argument("--shape", type=int, default=0,
                    help="force a launch shape (ML_SHAPE_*; skips the autotuner)")
    ap.add_argument("--block", type=int, default=0, help="force threads per CTA")
    ap.add_argument("--serving-seconds", type=float, default=60.0,
                    help="arrival window of the serving mix (0 = skip it)")
    ap.add_argument("--ncu", action="store_true",
                    help="skip the CPU leg, autotune, e2e and clocks (for profiler runs)")
    return ap.parse_args()


def workload_name(w):
    return (f"{w.name}: {w.crn.n_species} species x {w.crn.n_reactions} reactions, "
            f"{w.n_traj} trajectories per GPU, T={'per-trajectory' if w.T.size > 1 else float(w.T[0])}, "
            f"eps={w.eps}, n_c={w.n_c}")


# ---------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------
# algorithmic work model: the arithmetic the method needs per event (explicit leap,
# implicit leap with its Newton iterations, SSA firing, rejected leap)
# ---------------------------------------------------------------------------------
PHILOX_OPS = 70      # 10 rounds x (2 wide multiplies, 3 xors, 2 key adds)
UNIFORM_OPS = 3
LOG_OPS = 15
POISSON_INV_OPS = 40  # exp, ~3 search steps of 3 ops, uniform
POISSON_PTRS_OPS = 110
NEWTON_ITERATIONS = 4.3  # mean iterations per implicit leap on dimerisation states (oracle)

# Per-launch figures measured by ncu for the headline kernel, keyed by (config, shape,
# threads per CTA, specialized) of the launch the bench times: DRAM bytes read + written,
# warp instructions issued and FP64-pipe instruction rate (of peak), with the capture they
# come from (a profiles/ summary).  A launch shape without a capture of the current kernel
# reports null.  Captures: the full 1,000,000-trajectory batch, one launch each, CTAs per
# SM by occupancy.
_SRC = ("ncu --metrics gpu__time_duration.sum,smsp__inst_executed.sum,dram__bytes_read.sum,"
        "dram__bytes_write.sum,sm__inst_executed_pipe_fp64... -k regex:ml_jit -s 1 -c 1 "
        "python bench.py --config 2 --steps 1 --warmup 1 --no-plain --no-cpu "
        "--serving-seconds 0 --ncu --shape S --block B "
        "(profiles/k_jit_pool_fast_gene_expression_1M.md)")
PROFILED = {
    (2, 6, 128, 1): {"dram_bytes": 262120960 + 209241088, "warp_inst": 123710711486,
                     "fp64_pipe_pct": 31.60, "source": _SRC},
    (2, 6, 256, 1): {"dram_bytes": 263632640 + 209561856, "warp_inst": 123667242930,
                     "fp64_pipe_pct": 31.62, "source": _SRC},
    (2, 6, 64, 1): {"dram_bytes": 265054208 + 209970688, "warp_inst": 123713090021,
                    "fp64_pipe_pct": 31.53, "source": _SRC},
    (2, 1, 256, 1): {"dram_bytes": 271331584 + 210071040, "warp_inst": 188576129640,
                     "fp64_pipe_pct": 41.24, "source": _SRC},
    (2, 7, 64, 1): {"dram_bytes": 280494336 + 1490402048, "warp_inst": 135008423302,
                    "fp64_pipe_pct": 35.65, "source": _SRC},
}


def work_model(crn):
    import numpy as np
    o, nu = crn.orders, crn.stoich
    N, M = crn.n_species, crn.n_reactions
    fac = {1: 1, 2: 4, 3: 6}
    props = int(sum(sum(fac[int(m)] for m in row if m > 0) + 1 for row in o))
    nnz = int((nu != 0).sum())
    nreact = int((o.sum(0) > 0).sum())
    ssa = props + (M - 1) + PHILOX_OPS + 2 * UNIFORM_OPS + LOG_OPS + 1 + 2 * M + 2 * (nnz / M) + 2 * M + 1
    leap = (2 * props + (M - 1) + 2 * int((nu < 0).sum()) + 4 * nnz + 7 * nreact
            + M * (PHILOX_OPS + POISSON_INV_OPS) + nnz + 3 * M + M)
    # one Newton iteration with the exact Jacobian: propensities at y, residual, Jacobian
    # entries and assembly, elimination and back substitution, update and stopping test
    newton_it = props + 2 * nnz + 3 * N + 4 * int((o > 0).sum()) + 2 * nnz + (2 * N ** 3) // 3 + 2 * N * N + 4 * N
    implicit = leap + NEWTON_ITERATIONS * newton_it + 6 * M + 3 * 2
    reject = leap - props - nnz
    return {"explicit_leap": leap, "implicit_leap": round(implicit, 1), "ssa_firing": ssa,
            "rejected_leap": reject, "newton_iterations": NEWTON_ITERATIONS}


def ops_from_counts(model_ops, counts):
    return (counts[0] * model_ops["explicit_leap"] + counts[1] * model_ops["implicit_leap"]
            + counts[2] * model_ops["ssa_firing"] + counts[3] * model_ops["rejected_leap"])


# ---------------------------------------------------------------------------------
# reference arm and CPU baseline: the oracle on the host
# ---------------------------------------------------------------------------------
def oracle_rate(w, budget_s, seed=0, first_id=0, jacobian=1):
    """Time the oracle on a prefix sample of the workload sized to ~budget_s.
    Returns (trajectories/s, n_sample, seconds, outputs)."""
    from oracle import oracle as O
    params = O.Params(max_steps=MAX_STEPS, jacobian=jacobian)
    n = min(w.n_traj, 200)
    t0 = time.perf_counter()
    O.simulate(w.crn, n, w.x0[:n] if w.x0.ndim == 2 else w.x0, w.T[:n] if w.T.size > 1 else w.T,
               None if w.theta is None else w.theta[:n], params=params, seed=seed, traj_id_base=first_id)
    dt = max(time.perf_counter() - t0, 1e-6)
    n = int(min(w.n_traj, max(n, n * budget_s / dt)))
    xs = w.x0[:n] if w.x0.ndim == 2 else w.x0
    Ts = w.T[:n] if w.T.size > 1 else w.T
    th = None if w.theta is None else w.theta[:n]
    t0 = time.perf_counter()
    out = O.simulate(w.crn, n, xs, Ts, th, params=params, seed=seed, traj_id_base=first_id)
    dt = time.perf_counter() - t0
    return n / dt, n, dt, out


def _oracle_worker(task):
    """One process of the parallel oracle run: trajectory ids [lo, hi) of the workload."""
    cfg, n_total, lo, hi, seed, jac = task
    from oracle import oracle as O
    from paper_1608_07058_gb300 import workloads as W
    w = W.config(cfg, n_traj=n_total)
    if hi <= lo:
        return 0, 0.0
    xs = w.x0[lo:hi] if w.x0.ndim == 2 else w.x0
    Ts = w.T[lo:hi] if w.T.size > 1 else w.T
    th = None if w.theta is None else w.theta[lo:hi]
    t0 = time.perf_counter()
    O.simulate(w.crn, hi - lo, xs, Ts, th, params=O.Params(max_steps=MAX_STEPS, jacobian=jac),
               seed=seed, traj_id_base=lo)
    return hi - lo, time.perf_counter() - t0


def oracle_rate_parallel(cfg, n_total, rate1, budget_s, seed=0, jacobian=1, procs=None):
    """The unmodified oracle as `procs` independent processes (spawn) over disjoint id
    ranges, each sized for ~budget_s from the single-core rate; returns (trajectories/s over
    the wall clock of the timed map, processes, trajectories)."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    per = max(1, int(rate1 * budget_s))
    per = min(per, max(1, n_total // procs))
    tasks = [(cfg, n_total, k * per, (k + 1) * per, seed, jacobian) for k in range(procs)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_worker, [(cfg, n_total, 0, 0, seed, jacobian)] * procs)  # start-up
        t0 = time.perf_counter()
        done = pool.map(_oracle_worker, tasks)
        wall = time.perf_counter() - t0
    n = sum(d[0] for d in done)
    return n / wall, procs, n


def run_reference(args):
    from paper_1608_07058_gb300 import workloads as W
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = W.config(args.config, n_traj=args.n_traj)
    per_step_budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    rates, n_used = [], 0
    for s in range(args.warmup + args.steps):
        rate, n, dt, _ = oracle_rate(w, per_step_budget, seed=s,
                                     jacobian=1 if args.jacobian == "analytic" else 0)
        if s >= args.warmup:
            rates.append(rate)
            n_used = n
    value1 = statistics.mean(rates)
    # the same oracle on every host core (independent processes over disjoint id ranges)
    value, procs, n_par = oracle_rate_parallel(args.config, w.n_traj, value1,
                                               per_step_budget,
                                               jacobian=1 if args.jacobian == "analytic" else 0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "trajectories/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * w.n_traj / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(w)},
            "cpu_baseline": {"value": value, "unit": "trajectories/s", "cores": procs,
                             "kind": "oracle",
                             "sample": f"{n_par} trajectories as {procs} independent processes "
                                       f"over disjoint id ranges of the workload (C oracle, FP64 "
                                       f"reference algorithm); single-threaded: {value1:.4g} "
                                       f"trajectories/s on the first {n_used} ids per step"},
            "cpu_single_core": {"value": value1, "unit": "trajectories/s", "cores": 1},
            "e2e": {"value": value, "unit": "trajectories/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------
# serving mix: continuous batching against one request per launch
# ---------------------------------------------------------------------------------
def run_serving(ml, seconds, rate_hz=200.0, seed=11, max_inflight=8, budget=8 << 30,
                n_drain=200):
    import threading
    import numpy as np
    from paper_1608_07058_gb300 import workloads as W
    n_req = max(1, int(round(seconds * rate_hz)))
    reqs = W.serving_requests(n_req, seed=seed, rate_hz=rate_hz)
    models = {m: ml.model_from_crn(W.config(m, n_traj=1).crn) for m in (0, 1, 2, 3)}
    params = ml.ml_default_params(precision=ml.ML_PREC_FAST_FP32, form=ml.ML_FORM_PERSISTENT,
                                  max_steps=MAX_STEPS, jacobian=ml.ML_JAC_ANALYTIC,
                                  specialize=1)
    total_traj = sum(q["workload"].n_traj for q in reqs)

    # one request per launch, in arrival order: measured service times, queueing by the
    # arrival process (f_i = max(a_i, f_{i-1}) + s_i)
    for m in models:  # warm the per-model tables and kernels
        w1 = W.config(m, n_traj=64)
        ml.ml_simulate_host(models[m], 64, w1.x0, w1.T[:64] if w1.T.size > 1 else w1.T,
                            None if w1.theta is None else w1.theta[:64], params=params)
    service = []
    per_model = {m: {"requests": 0, "trajectories": 0, "busy_s": 0.0} for m in models}
    for q in reqs:
        wl = q["workload"]
        t0 = time.perf_counter()
        ml.ml_simulate_host(models[q["model_index"]], wl.n_traj, wl.x0, wl.T, wl.theta,
                            params=params, seed=wl.seed, traj_id_base=wl.traj_id_base)
        service.append(time.perf_counter() - t0)
        pm = per_model[q["model_index"]]
        pm["requests"] += 1
        pm["trajectories"] += wl.n_traj
        pm["busy_s"] += service[-1]
    arr = np.array([q["arrival_s"] for q in reqs])
    fin = np.zeros(len(reqs))
    prev = 0.0
    for i, (a, sv) in enumerate(zip(arr, service)):
        prev = max(a, prev) + sv
        fin[i] = prev
    lat_seq = fin - arr
    seq = {"p50_latency_ms": 1e3 * float(np.percentile(lat_seq, 50)),
           "p99_latency_ms": 1e3 * float(np.percentile(lat_seq, 99)),
           "sustained_traj_per_s": total_traj / (fin[-1] - arr[0]),
           "saturated_traj_per_s": total_traj / float(sum(service)),
           "busy_s": float(sum(service)),
           "per_model": {W.config(m, n_traj=1).name: {**v, "traj_per_s": v["trajectories"] / max(v["busy_s"], 1e-9)}
                         for m, v in per_model.items()}}

    # continuous batching: open-loop arrivals submitted by a thread at their times; the
    # main thread takes the requests in arrival order, records each latency and frees the
    # request's pinned buffers at once, so host memory holds only the requests in flight
    srv = ml.ml_server(budget, max_inflight, params)
    handles = [None] * len(reqs)
    submitted = threading.Semaphore(0)

    def submitter(t_start):
        for i, q in enumerate(reqs):
            dt = t_start + q["arrival_s"] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            wl = q["workload"]
            handles[i] = srv.submit(models[q["model_index"]], wl.n_traj, wl.x0, wl.T, wl.theta,
                                    seed=wl.seed, traj_id_base=wl.traj_id_base)
            submitted.release()

    t_start = time.perf_counter()
    th = threading.Thread(target=submitter, args=(t_start,))
    th.start()
    lat = []
    for i in range(len(reqs)):
        submitted.acquire()
        h = handles[i]
        h.wait(-1)
        lat.append(h.latency()[0])
        h.free()
        handles[i] = None
    th.join()
    t_end = time.perf_counter()
    st = srv.stats()
    # the completion of the last request, measured from the first arrival
    makespan = max(t_end - t_start - reqs[0]["arrival_s"], 1e-9)
    # capacity: the first n_drain requests submitted at once, time to drain (bounded so
    # that their pinned inputs and results fit in host memory)
    drain_set = reqs[:n_drain]
    drain_traj = sum(q["workload"].n_traj for q in drain_set)
    t0 = time.perf_counter()
    hs = [srv.submit(models[q["model_index"]], q["workload"].n_traj, q["workload"].x0,
                     q["workload"].T, q["workload"].theta, seed=q["workload"].seed,
                     traj_id_base=q["workload"].traj_id_base) for q in drain_set]
    for h in hs:
        h.wait(-1)
    drain = time.perf_counter() - t0
    for h in hs:
        h.free()
    srv.close()
    drain_busy = float(sum(service[:n_drain]))
    lat = np.array(lat)
    span = reqs[-1]["arrival_s"] - reqs[0]["arrival_s"]
    return {"requests": len(reqs), "arrival_rate_hz": rate_hz, "window_s": seconds,
            "trajectories": int(total_traj),
            "offered_traj_per_s": total_traj / max(span, 1e-9),
            "models": "immigration-death, dimerisation, gene expression, random 50x100",
            "horizon_scale": {W.config(m, n_traj=1).name: W.SERVING_HORIZON_SCALE[m] for m in models},
            "theta_gamma_shape": {W.config(m, n_traj=1).name: W.SERVING_THETA_SHAPE[m] for m in models},
            "why_scaled": "at 200 requests/s of 1e3-1e5 trajectories each model is offered "
                          "about 1.07e6 trajectories/s; at its benchmark horizon gene "
                          "expression would need 2.3 GPUs and the 50 x 100 network about "
                          "5,000, so each model's horizon is scaled to a fraction of one GPU",
            "p50_latency_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_latency_ms": 1e3 * float(np.percentile(lat, 99)),
            "sustained_traj_per_s": total_traj / makespan,
            "sustained_vs_one_request_per_launch": (total_traj / makespan) / seq["sustained_traj_per_s"],
            "p99_latency_vs_one_request_per_launch": float(np.percentile(lat, 99)) * 1e3 / seq["p99_latency_ms"],
            "saturated_traj_per_s": drain_traj / drain,
            "saturated_vs_one_request_per_launch": (drain_traj / drain) / (drain_traj / drain_busy),
            "saturated_requests": len(drain_set),
            "peak_inflight": st["peak_inflight"], "max_inflight": max_inflight,
            "peak_device_bytes": st["peak_bytes"], "budget_bytes": budget,
            "one_request_per_launch": seq,
            "note": "sustained = all trajectories / (last completion - first arrival) at the "
                    "offered load; one request per launch is timed request by request and "
                    "queued by the same arrival times; saturated = the first "
                    f"{n_drain} requests submitted at once (and served one per launch)",
            "inputs": "per-trajectory rate constants and horizons: B consecutive rows at a "
                      "random offset of a per-model pool of 100,000 draws"}


# ---------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------
def run_bayes(ml, out, reps=20):
    """Times the Bayesian step on the bench's own simulation output: posterior draws
    theta ~ Gamma(1 + r, 1 + G) for every (trajectory, reaction), then systematic
    resampling of the trajectories as particles (log-weights N(0, 9), seeded)."""
    import torch
    r, G = out["r"], out["G"]
    B, M = r.shape
    dev = r.device
    stream = torch.cuda.current_stream()
    one = torch.ones(M, dtype=torch.float64, device=dev)
    theta = torch.empty((B, M), dtype=torch.float64, device=dev)
    st = torch.empty((B,), dtype=torch.int32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    logw = torch.randn(B, dtype=torch.float64, device=dev, generator=g) * 3.0
    anc = torch.empty((B,), dtype=torch.int64, device=dev)
    ws = torch.empty(max(ml.ml_resample_workspace_bytes(B), 1), dtype=torch.uint8, device=dev)

    def time_it(fn):
        for k in range(3):
            fn(k)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(reps):
            fn(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    post_ms = time_it(lambda k: ml.ml_posterior_sample(one, one, r, G, seed=k, theta_out=theta,
                                                       status_out=st))
    res_ms = time_it(lambda k: ml.ml_resample_systematic(logw, seed=k, ancestors=anc,
                                                         workspace=ws))
    return {"posterior_draws_per_s": B * M / (post_ms / 1e3), "posterior_ms": post_ms,
            "resample_particles_per_s": B / (res_ms / 1e3), "resample_ms": res_ms,
            "particles": B, "reactions": M, "dtype": "f64",
            "note": "Gamma(1 + r, 1 + G) draws of the bench's last simulation output, then "
                    "systematic resampling of the trajectories; L2-resident inputs"}


def run_accuracy(ml, n=10_000, K=20, replicates=5, seed=500):
    """The accuracy study of Section 3 (Table 1) on the stiff dimerisation: per method, the
    KL divergence of its marginals from exact SSA averaged over K time points and all
    species (mean and std over replicates of n trajectories, each against a fresh SSA
    reference sample), and the device time of one n-trajectory run."""
    import numpy as np
    import torch
    from paper_1608_07058_gb300 import workloads as W
    w = W.config(1, n_traj=n)
    model = ml.model_from_crn(w.crn)
    dev = torch.device("cuda")
    x0 = torch.as_tensor(w.x0, device=dev)
    T = torch.as_tensor(w.T, device=dev)
    t_obs = torch.linspace(float(w.T[0]) / K, float(w.T[0]), K, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    methods = {"ssa": dict(mode=ml.ML_MODE_SSA_ONLY),
               "adaptive": dict(mode=ml.ML_MODE_ADAPTIVE, jacobian=ml.ML_JAC_FD),
               "adaptive_symbolic_jacobian": dict(mode=ml.ML_MODE_ADAPTIVE,
                                                  jacobian=ml.ML_JAC_ANALYTIC),
               "explicit": dict(mode=ml.ML_MODE_EXPLICIT_ONLY)}

    def run(kw, sd):
        p = ml.ml_default_params(precision=ml.ML_PREC_FAST_FP32, form=ml.ML_FORM_PERSISTENT,
                                 max_steps=MAX_STEPS, **kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = ml.ml_simulate_grid(model, n, x0, T, t_obs, params=p, seed=sd, counters=False)
        e1.record(stream)
        torch.cuda.synchronize()
        return out["X_obs"], e0.elapsed_time(e1)

    run(methods["ssa"], seed - 1)  # warm-up (tables, graph-free first launch)
    kl = {m: [] for m in methods}
    ms = {m: [] for m in methods}
    for rep in range(replicates):
        ref, _ = run(methods["ssa"], seed + 1000 * rep)
        for i, (m, kw) in enumerate(methods.items()):
            X, t = run(kw, seed + 1000 * rep + 1 + i)
            _, mean = ml.ml_kl_divergence(ref, X)
            kl[m].append(mean.item())
            ms[m].append(t)
    # Every grid point also ends a leap, so a denser grid shortens the implicit leaps that
    # damp the fast pair's fluctuations: the adaptive method's divergence against grid size
    by_k = {}
    for Kd in (K, 10 * K, 100 * K):
        td = torch.linspace(float(w.T[0]) / Kd, float(w.T[0]), Kd, dtype=torch.float64,
                            device=dev)
        outs = []
        for kw, sd in ((methods["ssa"], seed + 7), (methods["adaptive"], seed + 8)):
            p = ml.ml_default_params(precision=ml.ML_PREC_FAST_FP32,
                                     form=ml.ML_FORM_PERSISTENT, max_steps=MAX_STEPS, **kw)
            outs.append(ml.ml_simulate_grid(model, n, x0, T, td, params=p, seed=sd + Kd))
        kls, mean = ml.ml_kl_divergence(outs[0]["X_obs"], outs[1]["X_obs"])
        torch.cuda.synchronize()
        sd_ratio = (outs[1]["X_obs"][:, -1].double().std(0) /
                    outs[0]["X_obs"][:, -1].double().std(0)).cpu().numpy()
        by_k[str(Kd)] = {"kl_mean": mean.item(),
                         "kl_per_species": kls.mean(0).cpu().numpy().tolist(),
                         "std_ratio_at_T_per_species": sd_ratio.tolist(),
                         "implicit_leaps_per_traj": float(outs[1]["counters"][:, 1].double().mean())}
    return {m: {"kl_mean": float(np.mean(kl[m])), "kl_std": float(np.std(kl[m])),
                "ms_per_run": float(np.median(ms[m]))} for m in methods} | {
        "adaptive_vs_grid_points": by_k,
        "setup": (
        f"dimerisation x0 = (400, 798, 0), T = 0.2, eps = 0.03, {n} trajectories per "
        f"run, {K} time points, {replicates} replicates, each against a fresh exact-SSA "
        "sample; fast precision; KL of binned, half-count-smoothed marginals from SSA, "
        "averaged over time points and species (Section 3, Table 1)")}


SHAPE_NAMES = {1: "thread, round-based", 2: "warp", 3: "thread, round-based, occupancy build",
               4: "thread, sequential per lane", 5: "thread, sequential per lane, occupancy build",
               6: "thread, phase pool", 7: "thread, phase pool, occupancy build"}


def precision_label(ml, p):
    """What the fast kernels compute in which arithmetic, from the parameters used."""
    jac = "forward-difference" if p.jacobian == ml.ML_JAC_FD else "exact"
    if p.newton_precision == ml.ML_NEWTON_FP32:
        newton = ("FP32 Newton solve for the increment z = y - x (exact Jacobian) in the "
                  "thread kernel, FP32 factorization under an FP64 residual in the warp kernel")
    else:
        newton = f"FP64 Newton solve ({jac} Jacobian, pivoted elimination, rounding)"
    return ("FP32 propensities, step sizes, Poisson means and G increments; FP64 time and G "
            f"totals; {newton}; int64 counts")


class Bench:
    """Timing helpers shared by the headline workload and the extra workloads."""

    def __init__(self, ml, dev, stream, args, world, barrier):
        import torch
        self.ml, self.dev, self.stream, self.args = ml, dev, stream, args
        self.world, self.barrier = world, barrier
        self.flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2

    def outputs(self, model, B):
        import torch
        d = self.dev
        return {"X": torch.empty((B, model.N), dtype=torch.int64, device=d),
                "r": torch.empty((B, model.M), dtype=torch.int64, device=d),
                "G": torch.empty((B, model.M), dtype=torch.float64, device=d),
                "status": torch.empty((B,), dtype=torch.int32, device=d),
                "counters": torch.empty((B, 4), dtype=torch.int64, device=d)}

    def timed(self, model, B, x0, T, theta, params, seed0, id_base, steps, warmup,
                      budget_s=None, min_steps=2, order_from_warmup=False):
        """`warmup` full untimed steps (or, with warmup = 0, one launch on a 4,096-trajectory
        prefix), then timed steps: `steps` of them, or fewer once budget_s seconds of timed
        work have passed (never fewer than min_steps).  L2 is flushed before every step;
        each step is bracketed by CUDA events on the launching stream.  With
        order_from_warmup the timed steps hand trajectories out longest first, by the last
        warm-up step's per-trajectory event counts (an implicit or explicit leap counted as 8
        SSA firings); the order is computed once, before timing."""
        import torch
        ml, stream = self.ml, self.stream
        out = self.outputs(model, B)
        for s in range(warmup):
            ml.ml_simulate(model, B, x0, T, theta, params=params, seed=seed0 + s,
                           traj_id_base=id_base, out=out)
        if order_from_warmup and warmup > 0:
            c = out["counters"]
            cost = 8 * (c[:, 0] + c[:, 1]) + c[:, 2] + c[:, 3]
            self.order = torch.argsort(cost, descending=True, stable=True).to(torch.int64).contiguous()
            self.order_host = self.order.cpu().pin_memory()
            params.queue_order = self.order.data_ptr()
        if warmup == 0:
            n0 = min(B, 4096)
            ml.ml_simulate(model, n0, x0 if x0.dim() == 1 else x0[:n0],
                           T if T.numel() == 1 else T[:n0], None if theta is None else theta[:n0],
                           params=params, seed=seed0, traj_id_base=id_base)
        torch.cuda.synchronize()
        acc = torch.zeros(4, dtype=torch.int64, device=self.dev)
        evs, launches = [], 0
        self.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
        t0 = time.perf_counter()
        k = 0
        while k < steps:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            self.flush.zero_()
            e0.record(stream)
            ml.ml_simulate(model, B, x0, T, theta, params=params, seed=seed0 + warmup + k,
                           traj_id_base=id_base, out=out)
            e1.record(stream)
            evs.append((e0, e1))
            launches += ml.ml_model_last_launch_count(model)
            acc += out["counters"].sum(0)
            k += 1
            if budget_s is not None and k >= min_steps:
                e1.synchronize()
                if time.perf_counter() - t0 > budget_s:
                    break
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        self.barrier()
        wall = time.perf_counter() - t0
        ms = [a.elapsed_time(b) for a, b in evs]
        bad = int((out["status"] & ~(ml.ML_ST_NEWTON_FAIL | ml.ML_ST_PTRS_CAP)).ne(0).sum().item())
        return {"ms": ms, "mean_ms": statistics.mean(ms), "counts": acc.cpu().numpy(),
                "wall_s": wall, "steps": k, "launches": launches, "last_out": out,
                "last_seed": seed0 + warmup + k - 1, "bad_status": bad}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1608_07058_gb300 import matleap as ml
    from paper_1608_07058_gb300 import workloads as W

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor(v, dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.cpu().numpy()

    stream = torch.cuda.current_stream()
    bench = Bench(ml, dev, stream, args, world, barrier)
    jac = ml.ML_JAC_ANALYTIC if args.jacobian == "analytic" else ml.ML_JAC_FD
    newton = ml.ML_NEWTON_FP32 if args.newton == "fp32" else ml.ML_NEWTON_FP64

    def fast_params(newton_precision=newton):
        return ml.ml_default_params(precision=ml.ML_PREC_FAST_FP32, form=ml.ML_FORM_PERSISTENT,
                                    use_graph=1, max_steps=MAX_STEPS, jacobian=jac,
                                    newton_precision=newton_precision,
                                    specialize=0 if args.generic else 1)

    def plain_params(crn):
        return ml.ml_default_params(precision=ml.ML_PREC_REF_FP64, form=ml.ML_FORM_PLAIN,
                                    max_steps=MAX_STEPS, block_size=128, jacobian=jac,
                                    shape=ml.ML_SHAPE_THREAD_SEQ if crn.n_reactions <= 16
                                    else ml.ML_SHAPE_WARP)

    def load(cfg, n_traj=None, horizon=None):
        w = W.config(cfg, n_traj=n_traj)
        if horizon is not None:
            w.T = np.array([horizon])
        model = ml.model_from_crn(w.crn)
        x0 = torch.as_tensor(w.x0, device=dev)
        T = torch.as_tensor(w.T, device=dev)
        theta = None if w.theta is None else torch.as_tensor(w.theta, device=dev)
        return w, model, x0, T, theta

    def tune(model, B, x0, T, theta, p, n_sample=100_000):
        if args.shape:
            p.shape, p.block_size, p.ctas_per_sm = args.shape, args.block, 0
        elif not args.ncu and not args.no_autotune:
            best = ml.ml_autotune(model, B, x0, T, theta, params=p, n_sample=min(B, n_sample))
            p.shape, p.block_size, p.ctas_per_sm = best.shape, best.block_size, best.ctas_per_sm
        return p

    def shape_of(p):
        return {"shape": SHAPE_NAMES.get(p.shape, "auto"), "shape_id": int(p.shape),
                "block_size": int(p.block_size), "ctas_per_sm": int(p.ctas_per_sm),
                "kernels": "compiled at run time for this model (tables as constants)"
                if p.specialize else "precompiled (tables read at run time)"}

    # ---------------- the headline workload
    w, model, x0, T, theta = load(args.config, args.n_traj, args.horizon)
    B = w.n_traj
    # weak scaling: rank k simulates ids [k B, (k+1) B) of a world x B batch
    id_base, _ = ml.shard_bounds(world * B, rank, world)
    stage(f"headline workload {workload_name(w)}: autotune ...")
    # the headline batch is tuned as a whole, in the longest-first order of a pilot run
    # with another seed: a prefix under-fills the GPU differently (the pool driver keeps 64
    # trajectories per warp) and its tail is not the batch's
    p0 = fast_params()
    if not args.no_order and not args.shape and not args.ncu and not args.no_autotune:
        pilot = ml.ml_simulate(model, B, x0, T, theta, params=p0, seed=999,
                               traj_id_base=id_base)
        c = pilot["counters"]
        pilot_order = torch.argsort(8 * (c[:, 0] + c[:, 1]) + c[:, 2] + c[:, 3], descending=True,
                                    stable=True).to(torch.int64).contiguous()
        p0.queue_order = pilot_order.data_ptr()
    fast = tune(model, B, x0, T, theta, p0, n_sample=B)
    fast.queue_order = None
    stage(f"headline: shape {int(fast.shape)}, block {int(fast.block_size)}; timing ...")
    clocks = ClockSampler(local)
    if not args.ncu:
        clocks.start()
    res_fast = bench.timed(model, B, x0, T, theta, fast, 1000, id_base, args.steps,
                           args.warmup, order_from_warmup=not args.no_order)
    clk = clocks.stop() if not args.ncu else None
    ms_fast = max_over_ranks(res_fast["mean_ms"])
    counts_fast = sum_over_ranks(res_fast["counts"].astype(np.float64)) / res_fast["steps"]
    value = world * B / (ms_fast / 1e3)
    leap_steps = float(counts_fast[0] + counts_fast[1] + counts_fast[2])
    line = {"metric": METRIC, "value": value, "unit": "trajectories/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_fast,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": workload_name(w),
                       "form": "persistent refill kernel, CUDA graph, autotuned",
                       "precision": precision_label(ml, fast),
                       "jacobian": args.jacobian, "shape": shape_of(fast),
                       "queue_order": "longest first by the last warm-up step's per-trajectory "
                                      "event counts (computed once, before timing)"
                                      if fast.queue_order else "trajectory index",
                       "l2": "flushed between steps (256 MB write)"},
            "leap_steps_per_s": leap_steps / (ms_fast / 1e3),
            "accepted_leaps_per_s": float(counts_fast[0] + counts_fast[1]) / (ms_fast / 1e3),
            "ssa_steps_per_s": float(counts_fast[2]) / (ms_fast / 1e3),
            "mode_mix_per_step": {"explicit_leaps": float(counts_fast[0]),
                                  "implicit_leaps": float(counts_fast[1]),
                                  "ssa_firings": float(counts_fast[2]),
                                  "rejected_leaps": float(counts_fast[3])},
            "gpu_launches": int(res_fast["launches"])}

    def plain_leg(model, B, x0, T, theta, crn, seed0, budget_s, n_sub=None):
        # n_sub: time the plain form on a prefix of the batch (its rate is per trajectory)
        if n_sub is not None and n_sub < B:
            x0 = x0 if x0.dim() == 1 else x0[:n_sub]
            T = T if T.numel() == 1 else T[:n_sub]
            theta = None if theta is None else theta[:n_sub]
            B = n_sub
        res = bench.timed(model, B, x0, T, theta, plain_params(crn), seed0, id_base,
                                  args.steps, 0, budget_s=budget_s)
        msp = max_over_ranks(res["mean_ms"])
        cnt = sum_over_ranks(res["counts"].astype(np.float64)) / res["steps"]
        return {"value": world * B / (msp / 1e3), "unit": "trajectories/s", "ms_per_step": msp,
                "steps": res["steps"], "trajectories_per_step": B,
                "warmup": "one untimed launch on a 4,096-trajectory prefix",
                "leap_steps_per_s": float(cnt[:3].sum()) / (msp / 1e3),
                "gpu_launches": int(res["launches"]),
                "form": "one launch, one thread (warp for the 50 x 100 network) per trajectory "
                        "run to its end, FP64 reference precision"}

    if not args.no_plain:
        guarded(line, "plain_fp64",
                lambda: plain_leg(model, B, x0, T, theta, w.crn, 5000, args.plain_budget_s,
                                  args.plain_n_traj))
        if "value" in line["plain_fp64"]:
            line["batched_vs_plain"] = line["value"] / line["plain_fp64"]["value"]

    # roofline of the headline kernel: algorithmic operations against the issue rate
    ops_model = work_model(w.crn)
    ops_per_launch = ops_from_counts(ops_model, counts_fast / world)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peak_clock = 2070.0
    peak = sms * 128 * peak_clock * 1e6 / 1e12   # Tops/s: SMs x 4 schedulers x 32 lanes x clock
    achieved = ops_per_launch / (ms_fast / 1e3) / 1e12
    prof = PROFILED.get((args.config, int(fast.shape), int(fast.block_size),
                         int(fast.specialize)), {}) \
        if (args.n_traj is None and args.horizon is None) else {}
    line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                        "frac": achieved / peak, "traffic": prof.get("dram_bytes"),
                        "traffic_source": prof.get("source"),
                        "algorithmic_bytes_per_launch": int(B * (8 * model.N + 16 * model.M + 36)
                                                            + (0 if theta is None else B * 8 * model.M)
                                                            + (0 if w.T.size == 1 else B * 8)),
                        "peak_basis": f"{sms} SMs x 128 lanes x {peak_clock:.0f} MHz (one operation per lane per clock; measured FP32 FMA rate in pipe_peaks)",
                        "work_model_ops_per_event": ops_model}
    inst = prof.get("warp_inst")
    issue_peak = sms * 4 * peak_clock * 1e6
    line["roofline"]["issue"] = {
        "achieved": None if inst is None else inst / (ms_fast / 1e3), "peak": issue_peak,
        "unit": "warp-inst/s", "frac": None if inst is None else inst / (ms_fast / 1e3) / issue_peak,
        "warp_inst_per_launch": inst, "fp64_pipe_busy_pct": prof.get("fp64_pipe_pct"),
        "peak_basis": f"{sms} SMs x 4 warp instructions per clock x {peak_clock:.0f} MHz"}
    if clk:
        line["clocks"] = clk
        line["roofline"]["frac_at_measured_clock"] = achieved / (sms * 128 * clk["sm_mhz"] * 1e6 / 1e12)

    # end to end through the host-buffer entry point (pinned host memory)
    def e2e_leg():
        pin = lambda a: torch.as_tensor(a).pin_memory()
        hx0, hT = pin(w.x0), pin(w.T)
        hth = None if w.theta is None else pin(w.theta)
        hout = {"X": torch.empty((B, model.N), dtype=torch.int64).pin_memory(),
                "r": torch.empty((B, model.M), dtype=torch.int64).pin_memory(),
                "G": torch.empty((B, model.M), dtype=torch.float64).pin_memory(),
                "status": torch.empty((B,), dtype=torch.int32).pin_memory(),
                "counters": torch.empty((B, 4), dtype=torch.int64).pin_memory()}
        if fast.queue_order:  # the host entry point takes the order in host memory
            fast.queue_order = bench.order_host.data_ptr()
        ml.ml_simulate_host(model, B, hx0, hT, hth, params=fast, seed=99, traj_id_base=id_base,
                            out=hout, stream=stream)
        barrier()
        t0 = time.perf_counter()
        k = 0
        while k < args.steps:
            ml.ml_simulate_host(model, B, hx0, hT, hth, params=fast, seed=100 + k,
                                traj_id_base=id_base, out=hout, stream=stream)
            k += 1
            if k >= 2 and time.perf_counter() - t0 > args.e2e_budget_s:
                break
        barrier()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / k)
        h2d = hx0.numel() * 8 + hT.numel() * 8 + (0 if hth is None else hth.numel() * 8)
        d2h = sum(v.numel() * v.element_size() for v in hout.values())
        e2e = {"value": world * B / e2e_s, "unit": "trajectories/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": k, "warmup": 1,
               "path": "ml_simulate_host: pinned host inputs (and the queue order) -> "
                       "device -> simulate -> host"}
        if fast.queue_order:
            e2e["h2d_bytes_per_step"] += B * 8
        return e2e

    if not args.ncu and not args.no_e2e:
        dev_order = fast.queue_order
        try:
            guarded(line, "e2e", e2e_leg)
        finally:
            fast.queue_order = dev_order

    # CPU oracle baseline and oracle-matched statistics (rank 0, N = 1 only for the baseline)
    def cpu_leg():
        rate, n, dt, oout = oracle_rate(w, args.cpu_budget_s, seed=res_fast["last_seed"],
                                        first_id=id_base, jacobian=jac)
        if world == 1:
            line["cpu_baseline"] = {"value": rate, "unit": "trajectories/s", "cores": 1, "kind": "oracle",
                                    "sample": f"first {n} trajectory ids of the workload ({dt:.1f} s), "
                                              f"single-threaded C oracle, FP64 reference algorithm"}
            prate, procs, pn = oracle_rate_parallel(args.config, w.n_traj, rate,
                                                    args.cpu_budget_s, seed=res_fast["last_seed"],
                                                    jacobian=jac)
            line["cpu_baseline_all_cores"] = {
                "value": prate, "unit": "trajectories/s", "cores": procs, "kind": "oracle",
                "sample": f"{pn} trajectories as {procs} independent processes over disjoint id "
                          f"ranges (spawned pool, start-up excluded)"}
        from tests import stats_util
        g = {k: v[:n].cpu().numpy() for k, v in res_fast["last_out"].items()}
        rows = stats_util.compare(g, oout, g_res=stats_util.G_RESOLUTION_FAST)
        line["parity"] = {"fast_vs_oracle": stats_util.summary(rows), "n_compared": n,
                          "ids": f"first {n} trajectory ids of the last timed step, same seed",
                          "bad_status": res_fast["bad_status"]}
        line["parity"]["holm_pass_0.01"] = line["parity"]["fast_vs_oracle"]["holm_pass_0.01"]

    if rank == 0 and not args.no_cpu and not args.ncu:
        guarded(line, "cpu_baseline_and_parity", cpu_leg)  # sets its keys; an error stays here

    # the other workloads, each as a whole: fast (FP64 and FP32 Newton) and plain FP64
    def other_workload(cfg):
        we, me, x0e, Te, the = load(cfg)
        Be = we.n_traj
        entry = {"workload": workload_name(we)}
        for key, nw in (("fast_fp64_newton", ml.ML_NEWTON_FP64), ("fast_fp32_newton", ml.ML_NEWTON_FP32)):
            pe = tune(me, Be, x0e, Te, the, fast_params(nw))
            r = bench.timed(me, Be, x0e, Te, the, pe, 2000, id_base, args.steps,
                            args.warmup, budget_s=30.0)
            mse = max_over_ranks(r["mean_ms"])
            ce = sum_over_ranks(r["counts"].astype(np.float64)) / r["steps"]
            opse = ops_from_counts(work_model(we.crn), ce / world)
            entry[key] = {"value": world * Be / (mse / 1e3), "unit": "trajectories/s",
                          "ms_per_step": mse, "steps": r["steps"], "warmup": args.warmup,
                          "leap_steps_per_s": float(ce[:3].sum()) / (mse / 1e3),
                          "mode_mix_per_step": [float(v) for v in ce],
                          "precision": precision_label(ml, pe), "shape": shape_of(pe),
                          "roofline_frac": opse / (mse / 1e3) / 1e12 / peak,
                          "bad_status": r["bad_status"]}
        if not args.no_plain:
            entry["plain_fp64"] = plain_leg(me, Be, x0e, Te, the, we.crn, 6000, 30.0)
            entry["batched_vs_plain"] = entry["fast_fp64_newton"]["value"] / entry["plain_fp64"]["value"]
        return entry

    extras = {}
    for cfg in [int(c) for c in args.extra_configs.split(",") if c.strip()]:
        if cfg == args.config or args.ncu:
            continue
        guarded(extras, W.config(cfg, n_traj=1).name, lambda cfg=cfg: other_workload(cfg))
    if extras:
        line["other_workloads"] = extras

    def pipe_peaks_leg():
        pk = ml.ml_measure_pipe_peaks()
        return {"fp64_fma_tflops": pk["fp64_fma_flops"] / 1e12,
                "fp32_fma_tflops": pk["fp32_fma_flops"] / 1e12,
                "mufu_lg2_tops": pk["mufu_lg2_ops"] / 1e12,
                "note": "project microbenchmarks (8 independent chains per thread, "
                        "8 CTAs of 256 threads per SM, ~20 ms each)"}

    if rank == 0 and world == 1 and not args.ncu:
        guarded(line, "pipe_peaks", pipe_peaks_leg)
        guarded(line, "bayes_step", lambda: run_bayes(ml, res_fast["last_out"]))
        if not args.no_accuracy:
            guarded(line, "accuracy", lambda: run_accuracy(ml))
    if rank == 0 and world == 1 and args.serving_seconds > 0 and not args.ncu:
        guarded(line, "serving", lambda: run_serving(ml, args.serving_seconds))
    stage("done")
    if rank == 0:
        print(json.dumps(line, default=float), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
