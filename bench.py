"""H-FMM matvec benchmark: Mtargets/s of y = G q on one GB300.

Workload (default): three-layer medium k = 40 / 80 / 60, middle layer
0.5 thick, N = 1,048,576 points uniform in [0, 8] x [0.02, 8.02] (top layer),
64 complex right-hand sides with N(0,1) parts, tolerance 1e-6.  A step is one
apply (P2M, M2M, L2L + free-space and reaction M2L, L2P, P2P and the directly
summed reaction) over all right-hand sides; the plan (tree, lists, tables) is
built once before timing, as the paper precomputes its tables.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  value = N * nrhs / time per step / 1e6 over all ranks
(independent replicas, one per GPU).  e2e = the same through the C ABI with
pinned host buffers (copies inside the timed region).  The timed plan is
built without profiling; stage times and the leaf-kernel roofline come from a
second, profiling plan after the timed region.  cpu_baseline / the reference
arm = the CPU oracle (plain NumPy/SciPy H-FMM) on a bounded sample of the
same workload: the points of a 2 x 2 corner of the domain (same density, same
distance to the interface), all 64 right-hand sides split over one
single-threaded worker process per host core.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FP64_PEAK_TFLOPS = 1.25      # nominal GB300 FP64 rate (no measured FP64 figure exists)
# FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz (max SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
CPU_SAMPLE_SIDE = 2.0       # side of the corner of the domain the CPU oracle is timed on
FALLBACK_BF16_TFLOPS = 1900.0  # used only when MEASURED_PEAKS.json is absent
HEADLINE_METRIC = "H-FMM matvec Mtargets/s at N=1M (64 RHS) & rel-l2 err vs FP64; adjoint time"
PROFILE_STEPS = 10           # applies of the profiling plan (stage and leaf-kernel times)


# DRAM bytes of one full-size launch of the leaf-level downward kernel
# (m2l_tc_kernel<48> with the fused L2P), from an ncu capture of the
# 65536-point case of the same workload (dram__bytes_read.sum 110.8 MB,
# dram__bytes_write.sum 12.8 MB on 4096 leaves: p = 10, 16 points per leaf, 64 RHS), scaled
# by the leaf count to the 65536 leaves of the 1M-point workload (same order,
# width and points per leaf: the traffic grows in proportion).  It belongs to
# the kernel as captured; a changed kernel reports null until re-captured.
LEAF48_TRAFFIC_BYTES = (110.769408e6 + 13.832448e6) * 16


def max_over_ranks(x):
    """The largest x over the ranks of the default process group (x itself
    without one): the job's time is its slowest rank's.  The tensor lives on
    the GPU under NCCL and on the host under gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _measured_bf16(key="bf16_tflops"):
    """Dense bf16 TFLOP/s measured on this GPU type (burst, or with
    key="bf16_tflops_sustained" the seconds-long figure), and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_BF16_TFLOPS * (1.7 / 1.9 if key != "bf16_tflops" else 1.0), "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--n", type=int, default=0, help="override the number of points")
    ap.add_argument("--nrhs", type=int, default=0, help="override the number of right-hand sides")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-fp64-check", action="store_true",
                    help="skip the FP64 reference apply (accuracy and one-RHS FP64 time)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--adaptive", action="store_true",
                    help="FP64 uniform vs adaptive tree on config 2's clusters (N = 6400 .. 262144) and exit")
    ap.add_argument("--cases", default="",
                    help="--adaptive: workload:n pairs (e.g. 8:65536); --diag: k:n pairs (e.g. 1500:65536)")
    ap.add_argument("--diag", action="store_true",
                    help="FP64 diagonal vs dense translations at high frequency (k = 400, 1500) and exit")
    ap.add_argument("--sweep", action="store_true",
                    help="the N-sweep of the paper's timing table instead of the benchmark")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the two-layer and uneven-batch workloads measured after the headline")
    ap.add_argument("--cpu-sample-n", type=int, default=0)
    ap.add_argument("--box", type=float, nargs=4, default=None, metavar=("X0", "X1", "Y0", "Y1"),
                    help="draw the points in this box instead of the workload's domain (small profiling cases)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample: a child process runs a spawn pool with one
# single-threaded worker per host core; each worker holds the oracle's plan for
# the sample's points and applies it to its own chunk of right-hand sides.
# ---------------------------------------------------------------------------
_CPU_WORKER = {}


def _cpu_worker_init(job):
    """One worker's share of the CPU oracle: the points of a box of workload
    job["cfg"] (or instance job["salt"] of its own point family) and the
    right-hand sides lo..hi of its strengths."""
    import workloads as W
    from oracle import fmm
    cfg = job["cfg"]
    w = W.WORKLOADS[cfg]
    if job.get("box"):
        box = tuple(tuple(b) for b in job["box"])
        xy = W.points_in_box(cfg, job["n"], box)
        q = W.strengths(cfg, job["n"], job["nrhs"])
    else:
        xy = W.points(cfg, job["n"], salt=job["salt"])
        q = W.strengths(cfg, job["n"], job["nrhs"], salt=job["salt"])
    lo, hi = job["lo"], job["hi"]
    _CPU_WORKER["F"] = fmm.CpuFmm(xy, w.medium, tol=w.tol, leaf_size=16) if hi > lo else None
    _CPU_WORKER["q"] = q[lo:hi]


def _cpu_worker_apply(_):
    F = _CPU_WORKER["F"]
    if F is not None:
        F.apply(_CPU_WORKER["q"])
    return os.getpid()


def _cpu_child(spec):
    """Body of the CPU child process: one single-threaded worker process per
    job, `reps` applies of all jobs at once; returns the wall time of each."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pools = [ctx.Pool(1, initializer=_cpu_worker_init, initargs=(job,)) for job in spec["jobs"]]
    try:
        for pl in pools:                   # wait until every worker holds its plan
            pl.apply(os.getpid)
        times = []
        for _ in range(spec["reps"]):
            t0 = time.perf_counter()
            res = [pl.apply_async(_cpu_worker_apply, (0,)) for pl in pools]
            for r in res:
                r.get()
            times.append(time.perf_counter() - t0)
    finally:
        for pl in pools:
            pl.terminate()
    return {"apply_s": times, "cores": len(spec["jobs"])}


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _run_cpu_child(jobs, reps):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    spec = {"jobs": jobs, "reps": reps}
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child", json.dumps(spec)],
                       capture_output=True, text=True, env=env, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_oracle_sample(cfg, nrhs, reps=1, n=0, side=None):
    """The oracle on the points of a side x side corner of the workload's
    domain at the workload's density (default 2 x 2, i.e. 1/16 of the 8 x 8
    three-layer domain), all right-hand sides split over one worker per host
    core (a single worker for one right-hand side)."""
    import workloads as W
    w = W.WORKLOADS[cfg]
    (X0, X1), (Y0, Y1) = w.box
    density = w.n / ((X1 - X0) * (Y1 - Y0))
    side = side or CPU_SAMPLE_SIDE
    box = ((X0, X0 + side), (Y0, Y0 + side))
    n = n or int(round(density * side * side))
    cores = max(1, min(_host_cores(), nrhs))
    jobs = [{"cfg": cfg, "box": box, "n": n, "nrhs": nrhs, "lo": nrhs * c // cores, "hi": nrhs * (c + 1) // cores}
            for c in range(cores)]
    out = _run_cpu_child(jobs, reps)
    out.update({"n": n, "nrhs": nrhs, "box": box, "share": n / w.n})
    return out


def cpu_oracle_instances(cfg, sizes, nrhs, reps=2, max_points=60000):
    """The oracle on the smallest instances of an uneven batch (their sizes
    summing to at most max_points), one worker per instance, all at once."""
    order = sorted(range(len(sizes)), key=lambda i: sizes[i])
    pick, tot = [], 0
    for i in order:
        if pick and (tot + sizes[i] > max_points or len(pick) >= _host_cores()):
            break
        pick.append(i)
        tot += sizes[i]
    jobs = [{"cfg": cfg, "n": int(sizes[i]), "salt": i, "nrhs": nrhs, "lo": 0, "hi": nrhs} for i in pick]
    out = _run_cpu_child(jobs, reps)
    out.update({"n": tot, "nrhs": nrhs, "instances": pick, "share": tot / float(sum(sizes))})
    return out


def _cpu_sample_text(s, t_apply):
    if "box" in s:
        where = (f"the {s['n']} points of the [{s['box'][0][0]:g}, {s['box'][0][1]:g}] x "
                 f"[{s['box'][1][0]:g}, {s['box'][1][1]:g}] corner of the workload ({100 * s['share']:.2f}% of its "
                 f"points, same density and medium)")
        split = (f"{s['nrhs']} RHS split over {s['cores']} single-threaded worker processes (one per host core)"
                 if s["cores"] > 1 else f"{s['nrhs']} RHS on one single-threaded worker")
    else:
        where = (f"the {len(s['instances'])} smallest instances of the batch ({s['n']} points, "
                 f"{100 * s['share']:.2f}% of the batch's points)")
        split = f"{s['nrhs']} RHS, one single-threaded worker process per instance ({s['cores']} at once)"
    return (f"CPU oracle H-FMM (oracle/fmm.py, FP64) on {where}, {split}; apply {t_apply:.2f} s "
            f"(tables built in an untimed first apply)")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
def _profile_pass(Plan, xy, w, prec, nrhs, q, steps):
    """Per-stage and leaf-kernel times from a plan built with profiling (its
    own events around every stage; each query synchronises), kept out of the
    timed region: returns (avg stage ms, info, leaf ms, leaf flops, near ms,
    near flops)."""
    from paper_1703_09136_gb300 import FP64, PART_NEAR_FREE
    import torch
    plan = Plan(xy, w.medium, tol=w.tol, leaf_size=w.leaf, precision=prec, max_rhs=nrhs, profile=True)
    y = torch.empty_like(q)
    for _ in range(2):
        plan.apply(q, out=y)
    stage_ms, leaf_ms, leaf_flops = {}, 0.0, 0.0
    for _ in range(steps):
        plan.apply(q, out=y)
        for k, v in plan.stage_times().items():
            stage_ms[k] = stage_ms.get(k, 0.0) + v / steps
        if prec != FP64:
            lm, lf = plan.leaf_down_time()
            leaf_ms += lm / steps
            leaf_flops += lf / steps
    info = plan.info
    # the near field alone (no far field, so nothing runs beside it)
    near_ms = near_flops = 0.0
    if prec != FP64:
        for _ in range(3):
            plan.apply(q, out=y, parts=PART_NEAR_FREE)
            near_ms += plan.stage_times()["p2p"] / 3
            near_flops += plan.info["flops_last_apply"]["p2p"] / 3
    plan.close()
    return stage_ms, info, leaf_ms, leaf_flops, near_ms, near_flops


def _events_ms(fn, reps):
    """Mean CUDA-event time (ms) of fn() on the current stream, after two
    untimed calls."""
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _dominant_roofline(Plan, xy, w, prec, nrhs, q):
    """Stage times of a profiling plan and the roofline of its dominant stage
    (the warp-level SIMT kernels of few-RHS applies: FP32 pipe)."""
    avg, info, leaf_ms, leaf_fl, near_ms, near_fl = _profile_pass(Plan, xy, w, prec, nrhs, q, PROFILE_STEPS)
    dom = max(avg, key=avg.get)
    fl = info["flops_last_apply"][dom]
    if prec == 0:
        peak, src = FP64_PEAK_TFLOPS, "nominal GB300 FP64 rate"
    else:
        peak, src = FP32_PEAK_TFLOPS, "derived FP32 SIMT peak: 152 SMs x 128 lanes x 2 x 2.07 GHz"
    roof = {"kernel": f"stage '{dom}'", "bound": "alu", "achieved": fl / (avg[dom] * 1e-3) / 1e12, "peak": peak,
            "unit": "TFLOP/s", "peak_source": src, "traffic": None}
    roof["frac"] = roof["achieved"] / peak
    return avg, roof


def measure_two_layer(dev, steps, cpu=True):
    """Two-layer medium (k = 60 over 90), N = 262,144 uniform in [0, 4] x
    [0.02, 4.02], one right-hand side, tol 1e-6: the mixed-precision apply
    (few-RHS warp-level engine) against the plain FP64 apply on the same GPU."""
    import torch
    import workloads as W
    from paper_1703_09136_gb300 import Plan, FP64, MIXED
    cfg = 3
    w = W.WORKLOADS[cfg]
    xy_h = W.points(cfg)
    q_h = W.strengths(cfg, w.n, 1)
    xy = torch.from_numpy(xy_h).to(dev)
    q64 = torch.from_numpy(q_h).to(dev)
    q32 = q64.to(torch.complex64)
    t0 = time.perf_counter()
    pm = Plan(xy, w.medium, tol=w.tol, leaf_size=w.leaf, precision=MIXED, max_rhs=1)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    ym = torch.empty_like(q32)
    ms_mixed = _events_ms(lambda: pm.apply(q32, out=ym), steps)
    launches = int(pm.info["launches_last_apply"])
    qh = q32.cpu().pin_memory()
    yh = torch.empty_like(qh).pin_memory()
    pm._run(plan_lib_apply(), qh, yh, None)
    e2e_t = []
    for _ in range(5):
        t1 = time.perf_counter()
        pm._run(plan_lib_apply(), qh, yh, None)
        e2e_t.append(time.perf_counter() - t1)
    e2e_s = statistics.median(e2e_t)
    adj_ms = _events_ms(lambda: pm.adjoint(q32, out=ym), 5)
    pm.apply(q32, out=ym)
    y_mixed = ym.to(torch.complex128)
    pm.close()
    p64 = Plan(xy, w.medium, tol=w.tol, leaf_size=w.leaf, precision=FP64, max_rhs=1)
    y64 = torch.empty_like(q64)
    ms_fp64 = _events_ms(lambda: p64.apply(q64, out=y64), 3)
    p64.apply(q64, out=y64)
    err = float(torch.linalg.norm(y_mixed - y64) / torch.linalg.norm(y64))
    diag = {"levels": [l for l in range(32) if p64.info["diag_levels"] >> l & 1],
            "check": p64.info["diag_check"]}
    p64.close()
    # the same FP64 apply with every level's translations dense
    pd = Plan(xy, w.medium, tol=w.tol, leaf_size=w.leaf, precision=FP64, max_rhs=1, dense_m2l=True)
    yd = torch.empty_like(q64)
    ms_dense = _events_ms(lambda: pd.apply(q64, out=yd), 3)
    pd.apply(q64, out=yd)
    diag["fp64_dense_ms_per_apply"] = ms_dense
    diag["rel_l2_vs_dense"] = float(torch.linalg.norm(yd - y64) / torch.linalg.norm(yd))
    pd.close()
    stages, roof = _dominant_roofline(Plan, xy, w, MIXED, 1, q32)
    out = {"workload": w.name, "n": w.n, "nrhs": 1, "tol": w.tol, "medium": "two-layer k=60/90",
           "metric": "Mtargets/s (N x nrhs / apply time)", "value": w.n / (ms_mixed * 1e-3) / 1e6,
           "ms_per_apply": ms_mixed, "fp64_ms_per_apply": ms_fp64, "mixed_speedup_vs_fp64": ms_fp64 / ms_mixed,
           "fp64_diagonal_m2l": diag,
           "rel_l2_mixed_vs_fp64": err, "adjoint_ms": adj_ms, "plan_s": plan_s, "gpu_launches": launches,
           "engine": "few-RHS warp-level kernels (small_rhs default 4)", "stage_ms": stages, "roofline": roof,
           "e2e": {"value": w.n / e2e_s / 1e6, "unit": "Mtargets/s", "h2d_bytes_per_step": 8 * w.n,
                   "d2h_bytes_per_step": 8 * w.n}}
    if cpu:
        s = cpu_oracle_sample(cfg, 1, reps=2, side=1.0)
        t = s["apply_s"][-1]
        out["cpu_baseline"] = {"value": s["n"] / t / 1e6, "unit": "Mtargets/s", "cores": s["cores"],
                               "kind": "oracle", "sample": _cpu_sample_text(s, t)}
    return out


def measure_batch(dev, steps, cpu=True):
    """32 impedance instances (k = 40, alpha = 20) with N log-uniform in
    [4096, 200000], one right-hand side, through the batch API (one CUDA graph
    per apply), mixed precision and FP64."""
    import torch
    import workloads as W
    from paper_1703_09136_gb300 import Batch, FP64, MIXED
    cfg = 5
    w = W.WORKLOADS[cfg]
    sizes = [int(v) for v in W.batch_sizes(cfg)]
    ntot = sum(sizes)
    xys = [W.points(cfg, n, salt=i) for i, n in enumerate(sizes)]
    out = {"workload": w.name, "instances": len(sizes), "total_n": ntot, "n_min": min(sizes), "n_max": max(sizes),
           "nrhs": 1, "tol": w.tol, "medium": "impedance k=40 alpha=20",
           "metric": "Mtargets/s (sum of N x nrhs / batch apply time)"}
    for prec, name, cdt, pers in ((MIXED, "mixed", torch.complex64, False),
                                  (MIXED, "mixed_persistent", torch.complex64, True),
                                  (FP64, "fp64", torch.complex128, False)):
        qs = [torch.from_numpy(W.strengths(cfg, n, 1, salt=i)).to(dev, cdt) for i, n in enumerate(sizes)]
        ys = [torch.empty_like(q) for q in qs]
        t0 = time.perf_counter()
        batch = Batch(xys, w.medium, tol=w.tol, leaf_size=w.leaf, precision=prec, max_rhs=1, persistent=pers)
        torch.cuda.synchronize()
        plan_s = time.perf_counter() - t0
        ms = _events_ms(lambda: batch.apply(qs, ys), steps if prec == MIXED else 3)
        rec = {"ms_per_apply": ms, "value": ntot / (ms * 1e-3) / 1e6, "plan_s": plan_s}
        if not pers:
            # position gradient of every instance (FP64 pass for both precisions) and the
            # strength gradient (the batch adjoint), for a loss gradient g = y
            ys_g = [y.clone() for y in ys]
            rec["position_grad_ms"] = _events_ms(lambda: batch.grad(qs, ys_g), 3)
            rec["strength_grad_ms"] = _events_ms(lambda: batch.apply(ys_g, ys, adjoint=True), 3)
        if pers:
            rec["engine"] = "one persistent kernel over a device work queue (HFMM_FLAG_PERSISTENT)"
            rec["device_error"] = batch.device_error
            batch.close()
            out[name] = rec
            continue
        if prec == MIXED:
            rec["engine"] = "one CUDA graph, a branch of warp-level kernels per instance"
            rec["adjoint_ms"] = _events_ms(lambda: batch.apply(qs, ys, adjoint=True), 5)
            # end to end: pinned host strengths in, results out, around every batch apply
            qh = [q.cpu().pin_memory() for q in qs]
            yh = [torch.empty_like(q).pin_memory() for q in qh]
            e2e_t = []
            for it in range(6):
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                for a, d in zip(qh, qs):
                    d.copy_(a, non_blocking=True)
                batch.apply(qs, ys)
                for a, d in zip(yh, ys):
                    a.copy_(d, non_blocking=True)
                torch.cuda.synchronize()
                if it:
                    e2e_t.append(time.perf_counter() - t1)
            rec["e2e"] = {"value": ntot / statistics.median(e2e_t) / 1e6, "unit": "Mtargets/s",
                          "h2d_bytes_per_step": 8 * ntot, "d2h_bytes_per_step": 8 * ntot}
            batch.apply(qs, ys)
            y_mixed = [y.to(torch.complex128) for y in ys]
        else:
            batch.apply(qs, ys)
            num = sum(float(torch.linalg.norm(a - b) ** 2) for a, b in zip(y_mixed, ys))
            den = sum(float(torch.linalg.norm(b) ** 2) for b in ys)
            out["rel_l2_mixed_vs_fp64"] = (num / den) ** 0.5
        batch.close()
        out[name] = rec
    out["value"] = out["mixed"]["value"]
    out["mixed_speedup_vs_fp64"] = out["fp64"]["ms_per_apply"] / out["mixed"]["ms_per_apply"]
    if cpu:
        s = cpu_oracle_instances(cfg, sizes, 1, reps=2)
        t = s["apply_s"][-1]
        out["cpu_baseline"] = {"value": s["n"] / t / 1e6, "unit": "Mtargets/s", "cores": s["cores"],
                               "kind": "oracle", "sample": _cpu_sample_text(s, t)}
    return out


# Times of the paper's serial CPU code for this sweep (Sec. 4, Table 2: Xeon E5
# 3.7 GHz, k = 0.1, p = 39; the precision is not stated), seconds per apply.
PAPER_TABLE2_S = {100: 0.01, 6400: 0.67, 10000: 1.19, 90000: 10.92, 360000: 46.58, 640000: 100.85,
                  810000: 116.03, 1000000: 135.05}


def run_sweep(args):
    """The N-sweep of the paper's timing table: impedance alpha = 1, k = 0.1
    and 1, points uniform in the unit box centred at (0, 1.5), fixed order
    p = 39 on every level, one right-hand side; FP64 and mixed precision."""
    import torch
    import workloads as W
    from paper_1703_09136_gb300 import Plan, FP64, MIXED
    from paper_1703_09136_gb300 import build as _build
    _build.build()
    w = W.WORKLOADS[6]
    dev = torch.device("cuda", 0)
    rows = []
    for k in w.extra["k"]:
        med = W.Medium(W.IMPEDANCE, (k,), alpha=w.medium.alpha)
        for n in w.extra["n"]:
            xy = torch.from_numpy(W.points_in_box(6, n, w.box)).to(dev)
            q64 = torch.from_numpy(W.strengths(6, n, 1)).to(dev)
            row = {"k": k, "n": n, "paper_cpu_s": PAPER_TABLE2_S.get(n) if k == 0.1 else None}
            for prec, name in ((FP64, "fp64"), (MIXED, "mixed")):
                q = q64 if prec == FP64 else q64.to(torch.complex64)
                # the order rule adds ceil(k R_l) = 1 at these sizes: base 38 gives p = 39 on every level
                t0 = time.perf_counter()
                plan = Plan(xy, med, p=w.extra["p"] - 1, leaf_size=w.leaf, precision=prec, max_rhs=1)
                torch.cuda.synchronize()
                row[name + "_plan_s"] = time.perf_counter() - t0
                y = torch.empty_like(q)
                row[name + "_ms"] = _events_ms(lambda: plan.apply(q, out=y), 5 if prec == FP64 else 20)
                inf = plan.info
                row["levels"], row["p"] = inf["levels"], sorted(set(inf["p"][inf["lmin"]:]))
                if prec == FP64:
                    y64 = y.clone()
                else:
                    row["rel_l2_mixed_vs_fp64"] = float(torch.linalg.norm(y.to(torch.complex128) - y64)
                                                        / torch.linalg.norm(y64))
                plan.close()
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    out = {"metric": "H-FMM apply time vs N (shape of the paper's timing table)", "unit": "ms",
           "workload": w.name, "medium": "impedance alpha=1", "box": w.box, "p": w.extra["p"], "nrhs": 1,
           "rows": rows, "paper_hardware": "serial CPU code, Xeon E5 3.7 GHz, 32 GB, gcc 4.9.3 (k = 0.1)"}
    print(json.dumps(out), flush=True)


def run_diag(args):
    """FP64 apply with the coarse levels' translations in diagonal form against
    the same plan with every level dense (HFMM_FLAG_DENSE_M2L): impedance
    half-space (alpha = k / 2) on the unit box at k = 400 and 1500, where the
    level-2 boxes are ~30 and ~120 wavelengths wide; one right-hand side."""
    import torch
    import workloads as W
    from paper_1703_09136_gb300 import Plan
    from paper_1703_09136_gb300 import build as _build
    _build.build()
    w = W.WORKLOADS[7]
    dev = torch.device("cuda", 0)
    rows = []
    cases = w.extra["cases"]
    if args.cases:
        cases = [(float(c.split(":")[0]), int(c.split(":")[1])) for c in args.cases.split(",")]
    for k, n in cases:
        med = W.Medium(W.IMPEDANCE, (k,), alpha=k / 2)
        xy = torch.from_numpy(W.points_in_box(7, n, w.box)).to(dev)
        q = torch.from_numpy(W.strengths(7, n, 1)).to(dev)
        row = {"k": k, "n": n}
        ys = {}
        for dense in (False, True):
            name = "dense" if dense else "diagonal"
            t0 = time.perf_counter()
            plan = Plan(xy, med, tol=w.tol, leaf_size=w.leaf, max_rhs=1, dense_m2l=dense, profile=True)
            torch.cuda.synchronize()
            row[name + "_plan_s"] = time.perf_counter() - t0
            y = torch.empty_like(q)
            row[name + "_ms"] = _events_ms(lambda: plan.apply(q, out=y), 5)
            plan.apply(q, out=y)
            row[name + "_down_ms"] = plan.stage_times()["down"]
            inf = plan.info
            row["p"] = inf["p"]
            if not dense:
                row["diagonal_levels"] = [l for l in range(32) if inf["diag_levels"] >> l & 1]
                row["diagonal_check"] = inf["diag_check"]
            ys[dense] = y.clone()
            plan.close()
        row["rel_l2_diagonal_vs_dense"] = float(torch.linalg.norm(ys[False] - ys[True]) / torch.linalg.norm(ys[True]))
        row["speedup"] = row["dense_ms"] / row["diagonal_ms"]
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    out = {"metric": "FP64 H-FMM apply time, diagonal vs dense translations", "unit": "ms",
           "workload": w.name, "medium": "impedance alpha = k/2", "box": w.box, "tol": w.tol, "nrhs": 1,
           "rows": rows}
    print(json.dumps(out), flush=True)


def measure_adaptive(dev):
    """Uniform against adaptive tree (FP64, 1 RHS, tol 1e-6) on config 2
    itself (6400 clustered points) and on 65,536 particles of the star curve:
    apply times, tree depths, and the two results' difference; the adaptive
    tree also in mixed precision."""
    import torch
    import workloads as W
    from paper_1703_09136_gb300 import Plan, MIXED
    out = {}
    for cfg, n in ((2, 6400), (8, 65536)):
        w = W.WORKLOADS[cfg]
        xy = torch.from_numpy(W.points(cfg, n)).to(dev)
        q = torch.from_numpy(W.strengths(cfg, n, 1)).to(dev)
        row, ys = {"n": n}, {}
        for ad in (False, True):
            name = "adaptive" if ad else "uniform"
            plan = Plan(xy, w.medium, tol=w.tol, leaf_size=w.leaf, max_rhs=1, adaptive=ad)
            y = torch.empty_like(q)
            row[name + "_ms"] = _events_ms(lambda: plan.apply(q, out=y), 5)
            plan.apply(q, out=y)
            inf = plan.info
            row[name + "_levels"], row[name + "_leaves"] = inf["levels"], inf["nonempty_leaves"]
            ys[ad] = y.clone()
            plan.close()
        # the adaptive tree in mixed precision (FP32 passes)
        q32 = q.to(torch.complex64)
        plan = Plan(xy, w.medium, tol=w.tol, leaf_size=w.leaf, max_rhs=1, adaptive=True, precision=MIXED)
        y32 = torch.empty_like(q32)
        row["adaptive_mixed_ms"] = _events_ms(lambda: plan.apply(q32, out=y32), 5)
        plan.apply(q32, out=y32)
        plan.close()
        row["rel_l2_adaptive_mixed_vs_fp64"] = float(torch.linalg.norm(y32.to(torch.complex128) - ys[True]) /
                                                     torch.linalg.norm(ys[True]))
        row["rel_l2_adaptive_vs_uniform"] = float(torch.linalg.norm(ys[True] - ys[False]) / torch.linalg.norm(ys[False]))
        row["speedup"] = row["uniform_ms"] / row["adaptive_ms"]
        out[w.name] = row
    return out


def run_adaptive(args):
    """FP64 apply on the uniform tree against the adaptive tree (Sec. 3.1):
    config 2's clustered distribution (80% in two Gaussian blobs of sigma 0.1)
    at N = 6400 (config 2 itself), 65,536 and 262,144, and particles on a
    star-shaped curve (workload 8) at N = 65,536 and 262,144; impedance k = 40,
    alpha = 20, tol 1e-6, leaf size 32, one right-hand side; the adaptive tree
    also in mixed precision."""
    import torch
    import workloads as W
    from paper_1703_09136_gb300 import Plan, MIXED
    from paper_1703_09136_gb300 import build as _build
    _build.build()
    dev = torch.device("cuda", 0)
    rows = []
    cases = [(2, n) for n in (6400, 65536, 262144)] + [(8, n) for n in W.WORKLOADS[8].extra["bench_n"]]
    if args.cases:
        cases = [tuple(int(v) for v in c.split(":")) for c in args.cases.split(",")]
    for cfg, n in cases:
        w = W.WORKLOADS[cfg]
        xy = torch.from_numpy(W.points(cfg, n)).to(dev)
        q = torch.from_numpy(W.strengths(cfg, n, 1)).to(dev)
        row = {"workload": w.name, "n": n}
        ys = {}
        for ad in (False, True):
            name = "adaptive" if ad else "uniform"
            t0 = time.perf_counter()
            plan = Plan(xy, w.medium, tol=w.tol, leaf_size=w.leaf, max_rhs=1, adaptive=ad, profile=True)
            torch.cuda.synchronize()
            row[name + "_plan_s"] = time.perf_counter() - t0
            y = torch.empty_like(q)
            row[name + "_ms"] = _events_ms(lambda: plan.apply(q, out=y), 5)
            plan.apply(q, out=y)
            row[name + "_stage_ms"] = {k: round(v, 4) for k, v in plan.stage_times().items()}
            inf = plan.info
            row[name + "_levels"] = inf["levels"]
            row[name + "_leaves"] = inf["nonempty_leaves"]
            row[name + "_u_point_pairs"] = inf["u_pairs"]
            if ad:
                row["adaptive_w_pairs"], row["adaptive_x_pairs"] = inf["w_pairs"], inf["x_pairs"]
            ys[ad] = y.clone()
            plan.close()
        q32 = q.to(torch.complex64)
        plan = Plan(xy, w.medium, tol=w.tol, leaf_size=w.leaf, max_rhs=1, adaptive=True, precision=MIXED, profile=True)
        y32 = torch.empty_like(q32)
        row["adaptive_mixed_ms"] = _events_ms(lambda: plan.apply(q32, out=y32), 5)
        plan.apply(q32, out=y32)
        row["adaptive_mixed_stage_ms"] = {k: round(v, 4) for k, v in plan.stage_times().items()}
        plan.close()
        row["rel_l2_adaptive_mixed_vs_fp64"] = float(torch.linalg.norm(y32.to(torch.complex128) - ys[True]) /
                                                     torch.linalg.norm(ys[True]))
        row["rel_l2_adaptive_vs_uniform"] = float(torch.linalg.norm(ys[True] - ys[False]) / torch.linalg.norm(ys[False]))
        row["speedup"] = row["uniform_ms"] / row["adaptive_ms"]
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    out = {"metric": "FP64 H-FMM apply time, uniform vs adaptive tree", "unit": "ms",
           "workloads": [W.WORKLOADS[2].name, W.WORKLOADS[8].name], "medium": "impedance k=40 alpha=20",
           "tol": 1e-6, "nrhs": 1, "rows": rows}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import workloads as W
    from paper_1703_09136_gb300 import Plan, FP64, MIXED
    from paper_1703_09136_gb300 import build as _build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        torch.distributed.barrier()

    cfg = args.config
    w = W.WORKLOADS[cfg]
    n = args.n or w.n
    nrhs = args.nrhs or w.nrhs
    prec = FP64 if args.precision == "fp64" else MIXED
    cdt = torch.complex128 if prec == FP64 else torch.complex64
    if args.box:
        x0, x1, y0, y1 = args.box
        xy_h = W.points_in_box(cfg, n, ((x0, x1), (y0, y1)))
    else:
        xy_h = W.points(cfg, n)
    q_h = W.strengths(cfg, n, nrhs)
    dev = torch.device("cuda", local)
    xy = torch.from_numpy(xy_h).to(dev)
    q = torch.from_numpy(q_h).to(dev, cdt)
    # the timed plan: no profiling, so the K applies run back to back
    t0 = time.perf_counter()
    plan = Plan(xy, w.medium, tol=w.tol, leaf_size=w.leaf, precision=prec, max_rhs=nrhs)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    y = torch.empty_like(q)
    for _ in range(args.warmup):
        plan.apply(q, out=y)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        plan.apply(q, out=y)
    ev1.record(stream)
    torch.cuda.synchronize()
    total_ms = ev0.elapsed_time(ev1)
    ck = clocks.stop()
    if world > 1:
        total_ms = max_over_ranks(total_ms)
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = world * n * nrhs / (ms_per_step * 1e-3) / 1e6
    info = plan.info
    launches = int(info["launches_last_apply"]) * args.steps
    # end to end through the C ABI with pinned host buffers
    qh = torch.from_numpy(q_h).to(cdt).pin_memory()
    yh = torch.empty_like(qh).pin_memory()
    plan._run(plan_lib_apply(), qh, yh, None)        # untimed: first touch of the pinned pages
    e2e_t = []
    for _ in range(args.e2e_steps):
        t1 = time.perf_counter()
        plan._run(plan_lib_apply(), qh, yh, None)
        e2e_t.append(time.perf_counter() - t1)
    e2e_s = max_over_ranks(statistics.median(e2e_t))
    cbytes = 16 if prec == FP64 else 8
    e2e = {"value": world * n * nrhs / e2e_s / 1e6, "unit": "Mtargets/s",
           "h2d_bytes_per_step": cbytes * n * nrhs, "d2h_bytes_per_step": cbytes * n * nrhs}
    # adjoint time (one warm-up, then the mean of five)
    plan.adjoint(q, out=y)
    ev0.record(stream)
    for _ in range(5):
        plan.adjoint(q, out=y)
    ev1.record(stream)
    torch.cuda.synchronize()
    adjoint_ms = ev0.elapsed_time(ev1) / 5
    # accuracy against the plain FP64 path on the first right-hand sides, and
    # the FP64 path's time for one right-hand side
    accuracy = fp64_ms = None
    if prec != FP64 and not args.no_fp64_check:
        nchk = min(2, nrhs)
        plan.apply(q, out=y)
        y_mixed = y[:nchk].to(torch.complex128)
        p64 = Plan(xy, w.medium, tol=w.tol, leaf_size=w.leaf, precision=FP64, max_rhs=nchk)
        q64 = torch.from_numpy(q_h[:nchk].copy()).to(dev)
        y64 = torch.empty_like(q64)
        p64.apply(q64, out=y64)
        err = float(torch.linalg.norm(y_mixed - y64) / torch.linalg.norm(y64))
        q1 = q64[:1].contiguous()
        y1 = torch.empty_like(q1)
        p64.apply(q1, out=y1)
        ev0.record(stream)
        p64.apply(q1, out=y1)
        ev1.record(stream)
        torch.cuda.synchronize()
        accuracy = {"rel_l2_vs_fp64": err, "rhs_compared": nchk}
        fp64_ms = ev0.elapsed_time(ev1)
        p64.close()
    plan.close()
    del y
    # stage and leaf-kernel times from a profiling plan, outside the timed region
    avg, pinfo, leaf_ms, leaf_flops, near_ms, near_flops = _profile_pass(Plan, xy, w, prec, nrhs, q,
                                                                          PROFILE_STEPS)
    dom = max(avg, key=avg.get)
    flops = pinfo["flops_last_apply"][dom]
    bound = "alu"
    if prec == FP64:
        peak, src = FP64_PEAK_TFLOPS, "nominal GB300 FP64 rate (MEASURED_PEAKS.json has no FP64 figure)"
    elif dom in ("m2m", "down") and pinfo["tensor_levels"] > 0 and nrhs > pinfo["small_rhs"]:
        # FP32-accurate terms as three f16 tensor-core products (hi*hi + hi*lo +
        # lo*hi, kind::f16 with FP32 accumulation): the measured bf16 burst
        # peak (f16 runs at the bf16 rate) / 3
        bf16, how = _measured_bf16()
        peak = bf16 / 3.0
        src = f"derived 3xF16 peak: {how} bf16 {bf16:.1f} TFLOP/s (= f16 rate) / 3"
        bound = "tensor"
    else:
        peak, src = FP32_PEAK_TFLOPS, "derived FP32 SIMT peak: 152 SMs x 128 lanes x 2 x 2.07 GHz"
    roof = {"kernel": dom, "bound": bound, "achieved": flops / (avg[dom] * 1e-3) / 1e12,
            "peak": peak, "unit": "TFLOP/s", "traffic": None, "peak_source": src}
    roof["frac"] = roof["achieved"] / roof["peak"]
    stage_roof = near_roof = None
    if leaf_ms > 0.0 and bound == "tensor":
        # the dominant kernel itself: the leaf-level downward launch, its CUDA-event
        # time on the launching stream (the library's events) and its algorithmic flops
        stage_roof = dict(roof, kernel=f"stage '{dom}' (all levels)")
        roof = {"kernel": f"m2l_tc_kernel<{pinfo['leaf_tc_width']}> (leaf-level downward: L2L + free and reaction "
                          f"M2L{' + L2P' if pinfo['leaf_l2p_fused'] else ''})",
                "bound": "tensor", "achieved": leaf_flops / (leaf_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s",
                "traffic": (LEAF48_TRAFFIC_BYTES if pinfo["leaf_tc_width"] == 48 and pinfo["leaf_l2p_fused"]
                            and n == 1048576 and nrhs == 64 else None),
                "traffic_source": "ncu dram bytes of the 65536-point case (4096 leaves) x 16 leaves",
                "peak_source": src,
                "launch_ms": leaf_ms,
                "timing": f"CUDA events around the launch on its stream, mean of {PROFILE_STEPS} applies "
                          "of a profiling plan after the timed region"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        sus, _ = _measured_bf16("bf16_tflops_sustained")
        roof["frac_vs_sustained"] = roof["achieved"] / (sus / 3.0)
        if near_ms > 0.0:
            near_roof = {"kernel": "p2p_tc_kernel (near-field P2P, precomputed Green's-function tiles)",
                         "bound": "tensor", "achieved": near_flops / (near_ms * 1e-3) / 1e12, "peak": peak,
                         "unit": "TFLOP/s", "launch_ms": near_ms, "peak_source": src}
            near_roof["frac"] = near_roof["achieved"] / near_roof["peak"]
    medium = _medium_text(w.medium)
    out = {
        "metric": _metric_name(cfg, w, n, nrhs),
        "value": value, "unit": "Mtargets/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == FP64 else "f32", "data": "synthetic",
        "config": {"workload": w.name, "n": n, "nrhs": nrhs, "medium": medium,
                   "tol": w.tol, "levels": info["levels"], "p": info["p"], "plan_s": plan_s,
                   "l2": "inputs larger than L2 (q, y and expansions are GBs)",
                   **({"box": args.box} if args.box else {}),
                   "parallelism": f"replicas{world}"},
        "stage_ms": avg, "adjoint_ms": adjoint_ms, "gpu_launches": launches, "e2e": e2e, "roofline": roof,
        **({"roofline_stage": stage_roof} if stage_roof else {}),
        **({"roofline_near": near_roof} if near_roof else {}),
        **({"accuracy": accuracy, "fp64_one_rhs_ms": fp64_ms} if accuracy else {}),
        "clocks": ck,
    }
    if not args.no_extra and cfg == 4 and n == w.n and nrhs == w.nrhs and not args.box:
        # the other full-size workloads, measured in the same run on the same GPU
        out["workloads"] = {"two-layer-262144-1rhs": measure_two_layer(dev, 20, cpu=rank == 0 and not args.no_cpu_baseline),
                            "impedance-batch32-1rhs": measure_batch(dev, 20, cpu=rank == 0 and not args.no_cpu_baseline),
                            "adaptive-tree-fp64": measure_adaptive(dev)}
    if rank == 0 and not args.no_cpu_baseline:
        s = cpu_oracle_sample(cfg, nrhs, reps=2, n=args.cpu_sample_n)
        t_apply = s["apply_s"][-1]
        out["cpu_baseline"] = {"value": s["n"] * s["nrhs"] / t_apply / 1e6, "unit": "Mtargets/s",
                               "cores": s["cores"], "kind": "oracle", "sample": _cpu_sample_text(s, t_apply)}
        out["config"]["cpu_sample"] = {"n": s["n"], "share_of_points": s["share"], "box": s["box"],
                                       "cores": s["cores"]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def plan_lib_apply():
    from paper_1703_09136_gb300 import library
    return library().hfmm_apply


def _medium_text(m):
    if m.kind == 0:
        return f"impedance k={m.k[0]:g} alpha={m.alpha:g}"
    if m.kind == 1:
        return f"two-layer k={m.k[0]:g}/{m.k[1]:g}"
    return f"three-layer k={m.k[0]:g}/{m.k[1]:g}/{m.k[2]:g} d={m.d:g}"


def _metric_name(cfg, w, n, nrhs):
    if cfg == 4 and n == w.n and nrhs == w.nrhs:
        return HEADLINE_METRIC
    kind = {0: "impedance half-space", 1: "two-layer", 2: "three-layer"}[w.medium.kind]
    return f"H-FMM matvec throughput (targets x RHS per second), {kind} medium, N={n}, {nrhs} RHS"


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on every host core, each
    step one apply over all right-hand sides on a corner of the workload
    (2 x 2 when the whole run is at most 12 steps, else 1 x 1 so that it ends
    within a few minutes)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as W
    cfg = args.config
    w = W.WORKLOADS[cfg]
    nrhs = args.nrhs or w.nrhs
    side = CPU_SAMPLE_SIDE if args.warmup + args.steps <= 12 else 1.0
    s = cpu_oracle_sample(cfg, nrhs, reps=max(1, args.warmup) + args.steps, n=args.cpu_sample_n, side=side)
    times = s["apply_s"][max(1, args.warmup):]
    t = sum(times) / len(times)
    value = s["n"] * s["nrhs"] / t / 1e6
    out = {"impl": "reference", "metric": _metric_name(cfg, w, args.n or w.n, nrhs),
           "value": value, "unit": "Mtargets/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "n": w.n, "nrhs": s["nrhs"], "tol": w.tol,
                      "cpu_sample": {"n": s["n"], "share_of_points": s["share"], "box": s["box"],
                                     "cores": s["cores"]},
                      "parallelism": "rank 0 only (CPU)"},
           "cpu_baseline": {"value": value, "unit": "Mtargets/s", "cores": s["cores"], "kind": "oracle",
                            "sample": _cpu_sample_text(s, t)},
           "e2e": {"value": value, "unit": "Mtargets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batch(args):
    """Config 5: uneven independent instances applied together through the
    batch API (one captured CUDA graph, a branch per instance)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_1703_09136_gb300 import Batch, FP64, MIXED
    from paper_1703_09136_gb300 import build as _build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    cfg = 5
    w = W.WORKLOADS[cfg]
    sizes = [int(v) for v in W.batch_sizes(cfg)]
    nrhs = args.nrhs or w.nrhs
    prec = FP64 if args.precision == "fp64" else MIXED
    cdt = torch.complex128 if prec == FP64 else torch.complex64
    dev = torch.device("cuda", local)
    xys = [W.points(cfg, n, salt=i) for i, n in enumerate(sizes)]
    qs_h = [torch.from_numpy(W.strengths(cfg, n, nrhs, salt=i)).to(cdt) for i, n in enumerate(sizes)]
    qs = [q.to(dev) for q in qs_h]
    ys = [torch.empty_like(q) for q in qs]
    t0 = time.perf_counter()
    batch = Batch(xys, w.medium, tol=w.tol, leaf_size=w.leaf, precision=prec, max_rhs=nrhs)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        batch.apply(qs, ys)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        batch.apply(qs, ys)
    e1.record(st)
    torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    ck = clocks.stop()
    if world > 1:
        total_ms = max_over_ranks(total_ms)
    ms_per_step = total_ms / args.steps
    ntot = sum(sizes)
    value = world * ntot * nrhs / (ms_per_step * 1e-3) / 1e6
    # end to end: pinned host strengths in, results out, around every batch apply
    qh = [q.pin_memory() for q in qs_h]
    yh = [torch.empty_like(q).pin_memory() for q in qh]
    e2e_t = []
    for it in range(1 + max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for q, qd in zip(qh, qs):
            qd.copy_(q, non_blocking=True)
        batch.apply(qs, ys)
        for y, yd in zip(yh, ys):
            y.copy_(yd, non_blocking=True)
        torch.cuda.synchronize()
        if it > 0:
            e2e_t.append(time.perf_counter() - t1)
    e2e_s = max_over_ranks(statistics.median(e2e_t))
    cbytes = 16 if prec == FP64 else 8
    out = {
        "metric": "batched H-FMM matvec throughput (targets x RHS per second), 32 uneven impedance instances",
        "value": value, "unit": "Mtargets/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == FP64 else "f32", "data": "synthetic",
        "config": {"workload": w.name, "instances": len(sizes), "total_n": ntot, "n_min": min(sizes),
                   "n_max": max(sizes), "nrhs": nrhs, "medium": "impedance k=40 alpha=20", "tol": w.tol,
                   "plan_s": plan_s, "l2": "inputs and expansions larger than L2",
                   "parallelism": f"replicas{world}"},
        "gpu_launches": None,
        "e2e": {"value": world * ntot * nrhs / e2e_s / 1e6, "unit": "Mtargets/s",
                "h2d_bytes_per_step": cbytes * ntot * nrhs, "d2h_bytes_per_step": cbytes * ntot * nrhs},
        "roofline": None, "clocks": ck, "cpu_baseline": None,
    }
    batch.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    if len(sys.argv) == 3 and sys.argv[1] == "--cpu-child":
        print(json.dumps(_cpu_child(json.loads(sys.argv[2]))), flush=True)
        return
    args = parse()
    if args.adaptive:
        run_adaptive(args)
        return
    if args.diag:
        run_diag(args)
        return
    if args.sweep:
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.config == 5:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
