"""Benchmark: time-to-gap of the GB300 TT interior-point method at n = 2^10,
with contraction throughput, roofline, an end-to-end number through the C ABI
from host buffers, and the oracle timed on the host cores.

Default workload: Max-Cut SDP, n = 2^10 vertices (d = 10 TT cores, 2 x 2
modes), seeded Kronecker graph (ten seeded 2 x 2 0/1 patterns, unit
weights), TT rank cap 64, target gap 1e-4. The headline form is the plain
FP64 solve; the same instance is also solved with TF32 and BF16 tensor-core
contractions (FP32 accumulation, FP64 refinement sweep, rounding and gap
checks), each form reported with its error against the oracle's optimum.

The workload with Erdos-Renyi edges and weights U[0.5, 1.5] at the same size
and cap (`--workload maxcut_d10_kron_er_cap64`) cannot reach the gap at rank
cap 64: its dual residual is bounded below by the truncation error of the
objective's unfoldings (see `dual_residual_lower_bound`). Its line reports
value null with that bound, the residuals reached, per-iteration times and
contraction throughput.

One step is one interior-point iteration (Algorithm 1: residuals, mu, the
Mehrotra predictor and corrector block-AMEn Newton solves, step lengths,
update and rounding). The timed region runs K steps of one solve from its
initial point; the solve's time-to-gap is the device time of the steps up to
and including the first iteration at which the stopping rules hold.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "maxcut_d10_kron_cap64": dict(kind="maxcut", d=10, cap=64),
    "maxcut_d10_kron_er_cap64": dict(kind="maxcut_er", d=10, cap=64),
    "maxcut_d6_kron_cap16": dict(kind="maxcut", d=6, cap=16),
    # Lovasz theta, n = 2^10: hypercube Q_10 OR Kronecker extras (density ~1%), cap 64
    "theta_d10_hypercube_cap64": dict(kind="theta", d=10, cap=64, sub_d=6),
    # correlation clustering, n = 2^12, complete signed graph, cap 128; the oracle checks the
    # principal 2^6 sub-instance
    "cc_d12_signed_cap128": dict(kind="cc", d=12, cap=128, sub_d=6),
    # 64 independent Kronecker Max-Cut instances, d ~ U{6..11}, unit weights
    "maxcut_batch64_d6to11_cap64": dict(kind="batch", count=64, d_lo=6, d_hi=11, cap=64, d=11),
}
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
DTYPE = {"fp64": "f64", "fp32": "f32", "tf32": "tf32", "bf16": "bf16"}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=6)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="maxcut_d10_kron_cap64", choices=sorted(WORKLOADS))
    p.add_argument("--precision", default="fp64", choices=sorted(PREC))
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--forms", default="tf32,bf16",
                   help="other precisions solved on the same instance and reported beside the headline form")
    p.add_argument("--micro", default="", choices=["", "lu", "contract"],
                   help="run a kernel microbenchmark instead of the workload (lu: tt_lu_solve; contract: "
                        "environment update and local product)")
    p.add_argument("--shapes", default="16:32,64:128,128:256", help="r:R shapes of --micro contract")
    p.add_argument("--sizes", default="256,512,1024,2048,4096", help="system sizes of --micro lu")
    p.add_argument("--no-learned", dest="learned", action="store_false",
                   help="skip the FP64 solve with the learned rank predictor")
    p.add_argument("--form-time-limit", type=float, default=60.0,
                   help="wall-clock seconds per solve of the other precisions (tt_sdp_options.time_limit)")
    p.add_argument("--workers", type=int, default=16, help="host threads of the batched solve")
    p.add_argument("--sequential", type=int, default=8,
                   help="batched workload: instances also solved one at a time in FP64 (0: none)")
    p.add_argument("--shard", action="store_true",
                   help="batched workload under torchrun: split one batch over the ranks instead of one batch each")
    p.add_argument("--time-limit", type=float, default=60.0,
                   help="batched workload: wall-clock seconds per instance solve (tt_sdp_options.time_limit)")
    return p.parse_args()


def _instance(w, seed):
    from paper_2509_11890_gb300 import inputs
    if w["kind"] == "maxcut_er":
        return inputs.maxcut_kron_er(w["d"], seed)
    return inputs.maxcut_kron(w["d"], seed)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.stop = threading.Event()
        self.t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self.stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                for ln in out.stdout.strip().splitlines():
                    self.rows.append([x.strip() for x in ln.split(",")])
            except Exception:
                pass
            self.stop.wait(0.2)

    def __enter__(self):
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(seed: int, rank: int) -> int:
    """Replicas: each rank solves its own instance, drawn from seed + rank."""
    return seed + rank


def partition_batch(orders, world: int, cap: int):
    """Shards of a batch of independent instances over `world` ranks: greedy
    longest-processing-time assignment by the predicted cost d * cap^3 of an
    instance of order d (largest first, each to the least-loaded rank; ties go
    to the lower rank). Returns one list of instance indices per rank."""
    loads = [0.0] * world
    shards = [[] for _ in range(world)]
    for i in sorted(range(len(orders)), key=lambda j: (-orders[j], j)):
        r = min(range(world), key=lambda q: (loads[q], q))
        shards[r].append(i)
        loads[r] += float(orders[i]) * float(cap) ** 3
    return [sorted(sh) for sh in shards]


def gather_results(local: dict, world: int):
    """Host-side gather of per-instance results ({index: result}) on every rank
    (one all_gather of Python objects after the solves; no collective runs
    during them). Identity without a process group."""
    import torch.distributed as dist
    if world <= 1 or not (dist.is_available() and dist.is_initialized()):
        return dict(local)
    parts = [None] * world
    dist.all_gather_object(parts, local)
    out = {}
    for part in parts:
        out.update(part)
    return out


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def run_reference(a):
    """The oracle on the host cores: dense primal-dual IPM (O2) to the target gap on the same instance."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from oracle import sdp_dense as sd
    w = WORKLOADS[a.workload]
    if w["kind"] == "batch":
        return _run_reference_batch(a, w)
    sample = "the same instance"
    if w["kind"] in ("theta", "cc"):
        # the dense IPM cannot take these sizes: the oracle runs on the 2^sub_d instance
        inst = _other_instance(w["kind"], w["sub_d"], a.seed, full_d=w["d"] if w["kind"] == "cc" else None)
        p = _dense_sdp(w["kind"], inst)
        sample = f"the 2^{w['sub_d']} instance of the family (the full size is beyond the dense IPM)"
    else:
        inst = _instance(w, a.seed)
        p = sd.maxcut_sdp(inst["weights"])
    times = []
    res = None
    for _ in range(max(a.steps, 1)):
        t0 = time.perf_counter()
        res = sd.solve_dense(p, tol=1e-4)
        times.append(time.perf_counter() - t0)
    val = float(np.median(times))
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": "time-to-gap-1e-4 (s)", "value": val, "unit": "s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": val * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": a.workload, "n": 2 ** w["d"], "d": w["d"], "seed": a.seed},
        "cpu_baseline": {"value": val, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": f"dense HKM primal-dual IPM (oracle O2) on {sample} to relative gap 1e-4, "
                                   f"{res.iters} iterations, median of {len(times)} solves"},
        "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_pobj": res.pobj,
    }
    print(json.dumps(line), flush=True)
    return 0


def _run_reference_batch(a, w):
    """The oracle's dense IPM (O2) on the batch, one instance at a time. Each
    step solves one instance of every order d present in the batch; the
    batch's time is the sum over its 64 instances of the median time measured
    for their order. At most two steps run (the order-11 solve alone takes
    tens of seconds on the host)."""
    from oracle import sdp_dense as sd
    from paper_2509_11890_gb300 import inputs
    insts = inputs.batch_maxcut(w["count"], a.seed, w["d_lo"], w["d_hi"])
    rep = {}
    for i in insts:
        rep.setdefault(i["d"], i)
    steps = min(max(a.steps, 1), 2)
    times = {dd: [] for dd in rep}
    for _ in range(steps):
        for dd, i in sorted(rep.items()):
            t0 = time.perf_counter()
            sd.solve_dense(sd.maxcut_sdp(i["weights"]), tol=1e-4)
            times[dd].append(time.perf_counter() - t0)
    t_of = {dd: float(np.median(v)) for dd, v in times.items()}
    per = [t_of[i["d"]] for i in insts]
    total = float(sum(per))
    val = len(insts) / total
    desc = (f"dense HKM IPM (oracle O2) to relative gap 1e-4, one instance of each order d in {sorted(rep)} per "
            f"step ({steps} steps); batch time = sum over the {len(insts)} instances of the median time of their "
            f"order: {json.dumps({str(k): round(v, 4) for k, v in sorted(t_of.items())})} s")
    line = {
        "impl": "reference", "metric": "instances/s (batched time-to-gap-1e-4)", "value": val,
        "unit": "instances/s", "n_gpus": a.gpus, "steps": steps, "warmup": a.warmup,
        "ms_per_step": total * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": a.workload, "instances": w["count"], "d_range": [w["d_lo"], w["d_hi"]],
                   "seed": a.seed},
        "p50_time_to_gap_s": float(np.percentile(per, 50)), "p99_time_to_gap_s": float(np.percentile(per, 99)),
        "cpu_baseline": {"value": val, "unit": "instances/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": val, "unit": "instances/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _cpu_baseline_batch(insts, count=8):
    """The oracle's TT-IPM (O4, numpy FP64) on the host cores, one instance after
    another, on a bounded sample: the first `count` instances of the batch's
    smallest order (larger orders can take minutes each in numpy); instances/s
    over the sample."""
    from oracle import tt_ipm, tt_problems as tp
    t_all, n, nconv, per = 0.0, 0, 0, []
    dmin = min(i["d"] for i in insts)
    for i in [x for x in insts if x["d"] == dmin][:count]:
        ipm = tt_ipm.TTIPM(tp.maxcut(i["adjacency_cores"], i["d"]), tt_ipm.Options(rank_cap=64, max_iters=40))
        t0 = time.perf_counter()
        ok = ipm.solve()
        dt = time.perf_counter() - t0
        t_all += dt
        per.append(dt)
        n += 1
        nconv += int(ok)
    return {"value": n / t_all if t_all > 0 else None, "unit": "instances/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"TT-IPM oracle O4 (numpy FP64) on the first {n} instances of order d = {dmin} of the batch, "
                      f"one after another ({nconv} certified, {t_all:.1f} s, p50 {float(np.median(per)):.2f} s)"}


def _cpu_baseline(w, seed, budget_s=30.0):
    """Oracle O2 time-to-gap on the same instance (bounded: one solve, ~10-30 s of CPU work)."""
    from oracle import sdp_dense as sd
    inst = _instance(w, seed)
    p = sd.maxcut_sdp(inst["weights"])
    t0 = time.perf_counter()
    res = sd.solve_dense(p, tol=1e-4, max_iter=60)
    dt = time.perf_counter() - t0
    return {"value": dt, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one dense HKM IPM solve (oracle O2) of the same n={2 ** w['d']} instance to relative gap "
                      f"1e-4 ({res.iters} iterations, pobj {res.pobj:.6f})"}, res.pobj


def dual_residual_lower_bound(weights: np.ndarray, cap: int) -> dict:
    """Lower bound on the relative dual residual ||Z + C - diag(y)||_F / (1 + ||C||_F)
    of every Max-Cut iterate whose Z has TT rank <= cap + 1 (a rounded iterate
    plus its spectral shift), for any y.

    At bond k the vec_TT unfolding of Z - diag(y) has rank <= (cap + 1) +
    2^min(k, d-k) (diag(y) unfolds like the vector y), so by Eckart-Young the
    residual is at least the energy of the objective's unfolding beyond that
    rank. Plain numpy SVDs of the 4^k x 4^(d-k) unfoldings of C = L / 4."""
    n = weights.shape[0]
    d = int(round(np.log2(n)))
    C = (np.diag(weights.sum(1)) - weights) / 4.0
    T = C.reshape([2] * (2 * d)).transpose([x for i in range(d) for x in (i, d + i)])
    nC = float(np.linalg.norm(C))
    best, best_k = 0.0, 0
    for k in range(1, d):
        s = np.linalg.svd(T.reshape(4 ** k, 4 ** (d - k)), compute_uv=False)
        r = cap + 1 + 2 ** min(k, d - k)
        tail = float(np.sqrt(np.sum(s[r:] ** 2)))
        if tail / (1.0 + nC) > best:
            best, best_k = tail / (1.0 + nC), k
    return {"rel_d_lower_bound": best, "bond": best_k, "rank_cap": cap,
            "eps_d": 2e-4, "certifiable": best <= 2e-4}


def _solve_timed(tg, torch, wcores, opts, steps, stream, clocks=None):
    """One solve from the initial point, `steps` iterations, CUDA events on
    the launching stream around the loop. Returns (infos, total_s,
    time_to_gap_s or None, launches)."""
    ctx = tg.Context.maxcut(wcores, opts)
    torch.cuda.synchronize()
    l0 = tg.launch_count()
    infos = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        infos.append(ctx.newton_step())
    ev1.record(stream)
    torch.cuda.synchronize()
    ctx.close()
    total = ev0.elapsed_time(ev1) * 1e-3
    ttg = None
    for j, i in enumerate(infos):
        if i["converged"]:
            ttg = sum(x["seconds"] for x in infos[: j + 1])
            break
    return infos, total, ttg, tg.launch_count() - l0


def roofline_choice(precision, peaks, peak_kind, contraction, tc, local, gemm64):
    """The bench line's roofline kernel: the one with the most device time in
    the timed region, with its own achieved rate and peak. contraction =
    (flops, seconds) of the contraction stages; tc = (flops, seconds,
    launches) of the tcgen05 GEMM; local = (flops, seconds, systems, systems
    with FP32 factors, LU fallbacks) of the dense local solves; gemm64 =
    (flops, seconds, launches) of the timed FP64 strided GEMM launches (every
    eighth). Returns (bound, achieved, peak, unit, peak_note, kernel)."""
    cflops, csec = contraction
    tflops, tsec, tlaunch = tc
    lflops, lsec, lcalls, kkt_fp32, kkt_lu = local
    gflops64, gsec64, glaunch64 = gemm64
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    if precision == "fp64":
        bound, peak, punit = "alu", 1.25, "TFLOP/s"  # FP64 FMA rate of GB300 (nominal; 1.2547 measured)
        peak_note = "FP64 ALU peak, nominal 1.25 TFLOP/s (probe measured 1.25)"
    elif precision == "fp32":
        bound, peak, punit = "alu", fp32_peak, "TFLOP/s"
        peak_note = "FP32 ALU peak from 152 SMs x 128 lanes x 2 flops x max SM clock"
    else:
        ratio = 0.5 if precision == "tf32" else 1.0
        bound, peak, punit = "tensor", peaks["bf16_tflops_sustained"] * ratio, "TFLOP/s"
        peak_note = f"{peak_kind} bf16 sustained x {ratio} (nominal dtype ratio)"
    if precision == "fp64" and 8 * gsec64 > lsec and gsec64 > 0:
        # the FP64 strided GEMM kernel (every FP64 contraction stage, local
        # operator and block move) takes the most device time
        achieved = gflops64 / gsec64 / 1e12
        kernel = (f"gemm_nd_kernel<double> (FP64 strided SIMT GEMM of the contraction stages, local operators, "
                  f"block moves and trailing updates): {glaunch64} timed launches (every eighth), "
                  f"{gflops64 / max(glaunch64, 1) / 1e6:.3f} MFLOP and {gsec64 / max(glaunch64, 1) * 1e6:.1f} us "
                  f"per launch")
    elif lsec > csec and precision == "fp64":
        # the dense local solves take most of the FP64 iteration: block
        # elimination (bordered Cholesky, Schur-complement LU, cluster
        # triangular solves); when most of them kept FP32 factors (refined to
        # an FP64 residual of 1e-14) their peak is the FP32 ALU rate
        achieved = lflops / lsec / 1e12
        if kkt_fp32 * 2 > max(lcalls, 1):
            peak = fp32_peak
            peak_note = ("FP32 ALU peak from 152 SMs x 128 lanes x 2 flops x max SM clock (most local solves "
                         "factored in FP32 and refined in FP64)")
        kernel = (f"dense local solves (block elimination: bordered Cholesky, Schur-complement LU, cluster "
                  f"triangular solves; {kkt_fp32} of {lcalls} with FP32 factors refined in FP64, "
                  f"{kkt_lu} LU fallbacks): {lflops / max(lcalls, 1) / 1e9:.4f} GFLOP and "
                  f"{lsec / max(lcalls, 1) * 1e3:.3f} ms per system")
    elif bound == "tensor":
        # the tensor-core kernel: tcgen05 GEMM of the contraction stages
        achieved = tflops / tsec / 1e12 if tsec > 0 else 0.0
        kernel = (f"tc_gemm_kernel (tcgen05 {precision.upper()} GEMM of the contractions): "
                  f"{tlaunch} launches, {tflops / max(tlaunch, 1) / 1e9:.4f} GFLOP and "
                  f"{tsec / max(tlaunch, 1) * 1e6:.1f} us per launch")
    else:
        achieved = cflops / csec / 1e12 if csec > 0 else 0.0
        kernel = "environment / local-product contraction (three strided SIMT GEMM stages)"
    return bound, achieved, peak, punit, peak_note, kernel


def _form_record(infos, ttg, total, p_star):
    conv = [i for i in infos if i["converged"]]
    last = conv[0] if conv else infos[-1]
    rec = {"time_to_gap_s": ttg, "gap_reached": bool(conv), "iters": last["iter"],
           "timed_s": total, "pobj": last["pobj"], "dobj": last["dobj"], "rel_gap": last["rel_gap"],
           "rel_p": last["rel_p"], "rel_d": last["rel_d"], "max_rank_X": last["max_rank_X"],
           "max_rank_Z": last["max_rank_Z"], "max_rank_W": last["max_rank_W"],
           "xz_fallbacks": last["xz_fallbacks"], "gmres_iters": last["gmres_iters"],
           "iter_ms": [round(i["seconds"] * 1e3, 2) for i in infos if not i["converged"]]}
    if p_star is not None:
        rec["err_vs_oracle_p_star"] = abs(last["pobj"] - p_star) / (1.0 + abs(p_star))
    return rec


def _learned_form(tg, torch, w, a, wcores, p_star, base):
    """The plain FP64 solve with the learned per-bond rank predictor: the
    network is trained on the GPU on rounding traces of two other instances of
    the same family (seeds not used by the measured instance; untimed), then
    the measured instance is solved with it. Reported beside the plain solve:
    time-to-gap, the bonds rounded by the predicted-rank range finder and the
    fallbacks to the adaptive SVD."""
    from paper_2509_11890_gb300 import inputs
    X, t = [], []
    t0 = time.perf_counter()
    for s_ in (a.seed + 1000, a.seed + 1001):
        inst = inputs.maxcut_kron(w["d"], s_)
        c = tg.Context.maxcut(inst["adjacency_cores"], tg.default_options(rank_cap=w["cap"], max_iters=a.steps + 2,
                                                                           time_limit=a.form_time_limit))
        c.set_trace(True)
        c.solve()
        x, y = c.trace()
        c.close()
        X.append(x)
        t.append(y)
    X, t = np.concatenate(X), np.concatenate(t)
    pred = tg.RankPredictor(seed=7)
    loss = pred.train(X, t, epochs=300, batch=64, lr=2e-3, seed=1)
    train_s = time.perf_counter() - t0
    o = tg.default_options(rank_cap=w["cap"], precision=0, max_iters=a.steps + 2, time_limit=a.form_time_limit)
    c = tg.Context.maxcut(wcores, o)
    c.set_rank_predictor(pred)
    torch.cuda.synchronize()
    r = c.solve()
    torch.cuda.synchronize()
    info = c.newton_step() if r["status"] == 0 else None
    c.close()
    ok = r["status"] == 0
    rec = {"time_to_gap_s": r["seconds"] if ok else None, "gap_reached": ok, "iters": r["iters"],
           "pobj": r["pobj"], "dobj": r["dobj"], "rel_gap": r["rel_gap"], "rel_p": r["rel_p"], "rel_d": r["rel_d"],
           "trace_rows": int(len(t)), "train_loss": loss, "trace_and_train_s": train_s}
    if info is not None:
        used, fb = info["pred_used"], info["pred_fallbacks"]
        rec.update({"bonds_by_range_finder": used, "fallbacks": fb,
                    "fallback_rate": fb / (used + fb) if used + fb else None})
    if p_star is not None:
        rec["err_vs_oracle_p_star"] = abs(r["pobj"] - p_star) / (1.0 + abs(p_star))
    if ok and base.get("time_to_gap_s"):
        rec["speedup_vs_plain_fp64"] = base["time_to_gap_s"] / r["seconds"]
    return rec


def run_ours(a):
    import torch

    import paper_2509_11890_gb300 as tg

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = WORKLOADS[a.workload]
    seed = replica_seed(a.seed, rank)
    inst = _instance(w, seed)
    stream = torch.cuda.current_stream()
    # row a1 (setup, untimed): graph -> TT on the device
    if inst.get("adjacency_cores") is not None:
        wcores = inst["adjacency_cores"]
    else:
        wcores = tg.tt_from_dense(torch.from_numpy(inst["weights"]).cuda(), eps_rel=1e-13)
    w_ranks = [c.shape[0] for c in wcores] + [1]
    opts = tg.default_options(rank_cap=w["cap"], precision=PREC[a.precision], max_iters=a.steps + 2)
    # warm-up: W iterations of a throwaway solve
    ctx = tg.Context.maxcut(wcores, opts)
    for _ in range(a.warmup):
        ctx.newton_step()
    ctx.close()
    torch.cuda.synchronize()
    # the oracle's optimum of the same instance (untimed, rank 0): the error of every form
    p_star = None
    if rank == 0:
        from oracle import sdp_dense as sd
        p_star = sd.solve_dense(sd.maxcut_sdp(inst["weights"]), tol=1e-9).pobj
    # timed region: K iterations of one solve from its initial point
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    tg.contraction_stats_reset()
    tg.kkt_stats(reset=True)
    with Clocks(local) as clk:
        infos, total, ttg, launches = _solve_timed(tg, torch, wcores, opts, a.steps, stream)
    kkt_block, kkt_fp32, kkt_lu = tg.kkt_stats(reset=True)
    if world > 1:
        torch.distributed.barrier()
    cflops, csec = tg.contraction_stats()
    tflops, tsec, tlaunch = tg.tc_stats()
    lflops, lsec, lcalls = tg.lu_stats()
    gflops64, gsec64, glaunch64 = tg.gemm64_stats()
    reached = ttg is not None
    ttg_all, total = max_over_ranks([ttg if reached else float("inf"), total], device="cuda")
    head = _form_record(infos, ttg, total, p_star)
    # the other precisions on the same instance, each timed the same way
    forms = {a.precision: head}
    for f in [x for x in a.forms.split(",") if x and x != a.precision]:
        # the other precisions: one solve each through tt_sdp_solve, bounded by a
        # wall-clock limit; time-to-gap is the device time of its iterations
        o = tg.default_options(rank_cap=w["cap"], precision=PREC[f], max_iters=a.steps + 2,
                               time_limit=a.form_time_limit)
        c = tg.Context.maxcut(wcores, o)
        torch.cuda.synchronize()
        tg.contraction_stats_reset()
        t0 = time.perf_counter()
        r = c.solve()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        fcf, fcs = tg.contraction_stats()
        ftf, fts, ftl = tg.tc_stats()
        flf, fls, flc = tg.lu_stats()
        info = c.newton_step() if r["status"] == 0 else None
        c.close()
        ok = r["status"] == 0
        rec = {"time_to_gap_s": r["seconds"] if ok else None, "gap_reached": ok, "iters": r["iters"],
               "wall_s": wall, "status": r["status"], "pobj": r["pobj"], "dobj": r["dobj"], "rel_gap": r["rel_gap"],
               "rel_p": r["rel_p"], "rel_d": r["rel_d"], "time_limit_s": a.form_time_limit,
               "contraction_tflops": fcf / fcs / 1e12 if fcs > 0 else 0.0,
               "tc_gemm": {"launches": ftl, "tflops": ftf / fts / 1e12 if fts > 0 else 0.0,
                           "us_per_launch": fts / max(ftl, 1) * 1e6,
                           "frac_of_peak": (ftf / fts / 1e12) / (_peaks()[0]["bf16_tflops_sustained"] *
                                                                 (0.5 if f == "tf32" else 1.0)) if fts > 0 else 0.0},
               "lu": {"systems": flc, "tflops": flf / fls / 1e12 if fls > 0 else 0.0, "seconds": fls}}
        if info is not None:
            rec.update({k: info[k] for k in ("max_rank_X", "max_rank_Z", "xz_fallbacks", "gmres_iters")})
        if p_star is not None:
            rec["err_vs_oracle_p_star"] = abs(r["pobj"] - p_star) / (1.0 + abs(p_star))
        forms[f] = rec
    if a.learned and w["kind"] == "maxcut":
        forms["fp64_learned"] = _learned_form(tg, torch, w, a, wcores, p_star, head)
    if "fp64" in forms:
        for f, rec in forms.items():
            if f != "fp64":
                rec["pobj_rel_diff_vs_gpu_fp64"] = abs(rec["pobj"] - forms["fp64"]["pobj"]) / (
                    1.0 + abs(forms["fp64"]["pobj"]))
    # end to end through the C ABI with host buffers: H2D of the weight cores,
    # the solve, D2H of the primal iterate X
    e2e = None
    if not a.no_e2e:
        h2d = int(sum(c.size for c in wcores) * 8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2 = tg.Context.maxcut(wcores, opts)
        n_e2e = 0
        for _ in range(a.steps):
            info = ctx2.newton_step()
            n_e2e += 1
            if info["converged"]:
                break
        X = ctx2.iterate(0)
        torch.cuda.synchronize()
        e2e_t = time.perf_counter() - t0
        ctx2.close()
        e2e = {"value": e2e_t if info["converged"] else None, "unit": "s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(sum(c.size for c in X) * 8), "steps": n_e2e,
               "gap_reached": bool(info["converged"]), "timed_s": e2e_t}
    peaks, peak_kind = _peaks()
    contraction_tflops = cflops / csec / 1e12 if csec > 0 else 0.0
    lu_tflops = lflops / lsec / 1e12 if lsec > 0 else 0.0
    bound, achieved, peak, punit, peak_note, kernel = roofline_choice(
        a.precision, peaks, peak_kind, contraction=(cflops, csec), tc=(tflops, tsec, tlaunch),
        local=(lflops, lsec, lcalls, kkt_fp32, kkt_lu), gemm64=(gflops64, gsec64, glaunch64))
    line = {
        "metric": "time-to-gap-1e-4 (s)", "value": ttg_all if reached else None, "unit": "s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": total / a.steps * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[a.precision], "data": "synthetic",
        "config": {"workload": a.workload, "n": 2 ** w["d"], "d": w["d"], "rank_cap": w["cap"], "seed": a.seed,
                   "weights_tt_max_rank": max(w_ranks), "parallelism": "replicas" if world > 1 else "single",
                   "l2": "no flush: one IPM iteration streams far more than the 129 MB L2 holds between reuses"},
        "gap_reached": reached,
        "forms": forms,
        "oracle_p_star": p_star,
        "contraction_tflops": contraction_tflops,
        "contraction_share": csec / total if total > 0 else None,
        "lu_tflops": lu_tflops,
        "lu_share": lsec / total if total > 0 else None,
        "lu_systems": lcalls,
        "local_solves": {"systems": lcalls, "block_elimination": kkt_block, "fp32_factors_refined": kkt_fp32,
                         "lu_fallbacks": kkt_lu},
        "gemm64": {"timed_launches": glaunch64, "tflops": gflops64 / gsec64 / 1e12 if gsec64 > 0 else 0.0,
                   "seconds_timed": gsec64, "share_est": 8 * gsec64 / total if total > 0 else None,
                   "note": "every eighth FP64 GEMM launch is timed; share_est = 8 x its time / the timed region "
                           "(side streams overlap, so it can exceed the wall-clock share)"},
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": punit,
                     "frac": achieved / peak if peak else None, "traffic": None, "peak_source": peak_note,
                     "kernel": kernel},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    if not reached:
        line["null_reason"] = "the certified gap was not reached within the timed steps"
        if w["kind"] == "maxcut_er":
            lb = dual_residual_lower_bound(inst["weights"], w["cap"])
            line["dual_residual_bound"] = lb
            if not lb["certifiable"]:
                line["null_reason"] = (
                    f"uncertifiable at rank cap {w['cap']}: every iterate with TT rank <= {w['cap'] + 1} has "
                    f"rel_d >= {lb['rel_d_lower_bound']:.3f} (Eckart-Young at bond {lb['bond']}) > eps_d 2e-4")
    if rank == 0:
        cpu, opt = _cpu_baseline(w, a.seed)
        line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _other_context(tg, torch, kind, inst, opts):
    """theta / correlation-clustering context from dense host graphs, converted
    to TT on the device (row a1)."""
    tt = lambda m: tg.tt_from_dense(torch.from_numpy(np.ascontiguousarray(m, dtype=np.float64)).cuda(),
                                    eps_rel=1e-13)
    if kind == "theta":
        return tg.Context.theta(tt(inst["adjacency"]), opts)
    return tg.Context.cc(tt(inst["c_plus"]), tt(inst["c_minus"]), tt(inst["adjacency"]), opts)


def _other_instance(kind, d, seed, full_d=None):
    from paper_2509_11890_gb300 import inputs
    if kind == "theta":
        return inputs.theta_hypercube_kron(d, seed)
    if full_d is not None and full_d != d:
        return inputs.cc_signed_sub(full_d, d, seed)
    return inputs.cc_signed(d, seed)


def _dense_sdp(kind, inst):
    from oracle import sdp_dense as sd
    if kind == "theta":
        return sd.theta_sdp(inst["adjacency"])
    return sd.cc_sdp(inst["c_plus"], inst["c_minus"], inst["adjacency"])


def _iterate_bounded(tg, ctx, steps, limit):
    """Up to `steps` iterations, stopping at the first certified one, at a
    solver error (its status is recorded) or once `limit` wall seconds pass."""
    infos, err = [], None
    t0 = time.perf_counter()
    for _ in range(steps):
        try:
            info = ctx.newton_step()
        except tg.TTSDPError as e:
            err = {"status": e.status, "message": str(e)}
            break
        infos.append(info)
        if info["converged"] or time.perf_counter() - t0 > limit:
            break
    return infos, err, time.perf_counter() - t0


def run_other(a):
    """Lovasz theta (n = 2^10) and correlation clustering (n = 2^12): the plain
    FP64 solve with the timed steps bounded by a wall-clock limit; value is the
    time-to-gap, or null with the reason (a solver status or the limit). The
    oracle's dense IPM checks the same method on a 2^sub_d instance of the
    family (for correlation clustering the principal sub-instance of the same
    graph), which is also the CPU baseline."""
    import torch

    import paper_2509_11890_gb300 as tg

    torch.cuda.set_device(0)
    w = WORKLOADS[a.workload]
    kind = w["kind"]
    inst = _other_instance(kind, w["d"], a.seed)
    # tt_sdp_solve with the library's deadline (checked between the core steps
    # of the sweeps), so a long iteration cannot overrun the limit
    opts = tg.default_options(rank_cap=w["cap"], precision=PREC[a.precision], max_iters=a.steps,
                              time_limit=a.time_limit)
    stream = torch.cuda.current_stream()
    ctx = _other_context(tg, torch, kind, inst, opts)
    torch.cuda.synchronize()
    tg.contraction_stats_reset()
    l0 = tg.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    err = None
    t0 = time.perf_counter()
    with Clocks(0) as clk:
        ev0.record(stream)
        try:
            res = ctx.solve()
        except tg.TTSDPError as e:
            res, err = None, {"status": e.status, "message": str(e)}
        ev1.record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ranks = {"max_rank_X": max(ctx.ranks(0)), "max_rank_Z": max(ctx.ranks(3))}
    ctx.close()
    total = ev0.elapsed_time(ev1) * 1e-3
    conv = res is not None and res["status"] == 0
    ttg = res["seconds"] if conv else None
    if res is not None and res["status"] != 0 and err is None:
        err = {"status": res["status"], "message": "iteration budget or time limit reached without the gap"}
    lflops, lsec, lcalls = tg.lu_stats()
    cflops, csec = tg.contraction_stats()
    # the same method against the dense oracle on the small instance
    sub = _other_instance(kind, w["sub_d"], a.seed, full_d=w["d"] if kind == "cc" else None)
    sctx = _other_context(tg, torch, kind, sub, tg.default_options(rank_cap=w["cap"], max_iters=60,
                                                                     time_limit=a.time_limit))
    sinfos, serr, _ = _iterate_bounded(tg, sctx, 60, min(a.time_limit, 60.0))
    sctx.close()
    from oracle import sdp_dense as sd
    t0 = time.perf_counter()
    ref = sd.solve_dense(_dense_sdp(kind, sub), tol=1e-8)
    t_ref = time.perf_counter() - t0
    s_last = sinfos[-1] if sinfos else None
    line = {
        "metric": "time-to-gap-1e-4 (s)", "value": ttg, "unit": "s", "n_gpus": 1, "steps": a.steps,
        "warmup": 0, "ms_per_step": total / max(res["iters"] if res else 1, 1) * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[a.precision], "data": "synthetic",
        "config": {"workload": a.workload, "n": 2 ** w["d"], "d": w["d"], "rank_cap": w["cap"], "seed": a.seed,
                   "parallelism": "single", "l2": "no flush"},
        "gap_reached": bool(conv), "wall_s": wall, "time_limit_s": a.time_limit,
        "final": (dict({k: res[k] for k in ("iters", "rel_gap", "rel_p", "rel_d", "pobj", "dobj", "seconds")},
                       **ranks) if res is not None else ranks),
        "lu_share": lsec / total if total > 0 else None, "contraction_share": csec / total if total > 0 else None,
        "gpu_launches": tg.launch_count() - l0, "clocks": clk.summary(),
        "sub_instance": {"d": w["sub_d"], "p_star": ref.pobj,
                         "gpu_pobj": s_last["pobj"] if s_last else None,
                         "gap_reached": bool(s_last and s_last["converged"]),
                         "err_vs_oracle_p_star": (abs(s_last["pobj"] - ref.pobj) / (1 + abs(ref.pobj))
                                                  if s_last else None),
                         "error": serr},
        "cpu_baseline": {"value": t_ref, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"dense IPM (oracle O2) on the 2^{w['sub_d']} instance "
                                   f"({'principal sub-instance' if kind == 'cc' else 'same family'}) to 1e-8"},
        "e2e": None,
    }
    if not conv:
        line["null_reason"] = (f"solver status {err['status']}: {err['message']}" if err else
                               "the certified gap was not reached")
    print(json.dumps(line), flush=True)
    return 0


def run_batch(a):
    """Batched solve: every step solves all instances of the batch concurrently
    (tt_sdp_solve_batch: worker threads, one CUDA stream each); the value is
    instances per second over the timed steps. Replicas shard nothing: under
    torchrun every rank solves its own batch (seed + rank)."""
    import torch

    import paper_2509_11890_gb300 as tg
    from paper_2509_11890_gb300 import inputs

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = WORKLOADS[a.workload]
    seed = replica_seed(a.seed, rank)
    insts = inputs.batch_maxcut(w["count"], seed, w["d_lo"], w["d_hi"])
    if world > 1 and a.shard:
        # one batch split over the ranks (every rank draws the same batch)
        insts_all = inputs.batch_maxcut(w["count"], a.seed, w["d_lo"], w["d_hi"])
        mine = partition_batch([i["d"] for i in insts_all], world, w["cap"])[rank]
        insts = [insts_all[j] for j in mine]
    opts = tg.default_options(rank_cap=w["cap"], precision=PREC[a.precision], max_iters=60,
                              time_limit=a.time_limit)

    def make():
        return [tg.Context.maxcut(i["adjacency_cores"], opts) for i in insts]

    for _ in range(a.warmup):
        # warm-up on a slice of the batch (one instance of every size)
        seen, sub = set(), []
        for i in insts:
            if i["d"] not in seen:
                seen.add(i["d"])
                sub.append(tg.Context.maxcut(i["adjacency_cores"], opts))
        tg.solve_batch(sub, workers=a.workers)
        for c in sub:
            c.close()
    torch.cuda.synchronize()
    l0 = tg.launch_count()
    per, walls, creates, results = [], [], [], []
    h2d = int(sum(c.size for i in insts for c in i["adjacency_cores"]) * 8)
    with Clocks(local) as clk:
        for _ in range(a.steps):
            if world > 1:
                torch.distributed.barrier()
            # end to end: host cores -> device problem assembly -> solves -> result records
            torch.cuda.synchronize()
            tc0 = time.perf_counter()
            ctxs = make()
            torch.cuda.synchronize()
            creates.append(time.perf_counter() - tc0)
            t0 = time.perf_counter()
            res = tg.solve_batch(ctxs, workers=a.workers)
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - t0)
            per += [r["seconds"] for r in res]
            results = res
            for c in ctxs:
                c.close()
    launches = tg.launch_count() - l0
    wall = sum(walls)
    wall, create = max_over_ranks([wall, sum(creates)], device="cuda")
    sharded = world > 1 and a.shard
    n_inst = w["count"] * a.steps * (1 if sharded else world)
    if sharded:
        allres = gather_results({j: (r["status"], s_, r["iters"]) for j, r, s_ in
                                 zip(mine, results, per[-len(results):])}, world)
        results = [{"status": allres[j][0], "iters": allres[j][2]} for j in sorted(allres)]
        per = [allres[j][1] for j in sorted(allres)]
    conv = sum(r["status"] == 0 for r in results)
    line = {
        "metric": "instances/s (batched time-to-gap-1e-4)", "value": n_inst / wall, "unit": "instances/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": wall / a.steps * 1e3,
        "higher_is_better": True, "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": DTYPE[a.precision], "data": "synthetic",
        "config": {"workload": a.workload, "instances": w["count"], "d_range": [w["d_lo"], w["d_hi"]],
                   "d_values": [i["d"] for i in insts], "rank_cap": w["cap"], "seed": a.seed,
                   "workers": a.workers,
                   "parallelism": ("sharded" if sharded else "replicas") if world > 1 else "single",
                   "l2": "each instance streams its own cores; no flush"},
        "p50_time_to_gap_s": float(np.percentile(per, 50)), "p99_time_to_gap_s": float(np.percentile(per, 99)),
        "converged": int(conv), "time_limit_s": a.time_limit,
        "note": "per-instance times of instances stopped by the time limit count at their stopping time",
        "iters_mean": float(np.mean([r["iters"] for r in results])),
        "gpu_launches": launches, "clocks": clk.summary(),
        "roofline": None,
        "e2e": {"value": n_inst / (wall + create), "unit": "instances/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(64 * len(insts)),
                "note": "each step copies the instances' adjacency cores from host memory, assembles the "
                        "problems on the device, solves them and reads one result record per instance"},
    }
    if rank == 0 and world == 1:
        line["cpu_baseline"] = _cpu_baseline_batch(insts)
    if rank == 0 and a.sequential > 0:
        # one at a time in the plain FP64 form, on a bounded sample of the batch
        o64 = tg.default_options(rank_cap=w["cap"], precision=0, max_iters=60, time_limit=a.time_limit)
        sample = insts[: a.sequential]
        ts, nconv = [], 0
        for i in sample:
            c = tg.Context.maxcut(i["adjacency_cores"], o64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = c.solve()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            nconv += int(r["status"] == 0)
            c.close()
        line["sequential_fp64"] = {
            "instances": len(sample), "converged": nconv, "instances_per_s": len(sample) / sum(ts),
            "p50_time_to_gap_s": float(np.percentile(ts, 50)), "p99_time_to_gap_s": float(np.percentile(ts, 99)),
            "sample": f"the first {len(sample)} instances of the batch, solved one after another in FP64"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_micro_lu(a):
    """Dense local solve microbenchmark (tt_lu_solve): seeded well-conditioned
    systems of the sizes the AMEn sweeps form (n x n, n up to 4096), FP64 and
    FP32-factor / FP64-refined, CUDA events on the launching stream, best of
    `steps` after `warmup` untimed solves. One JSON line per size and precision."""
    import torch

    import paper_2509_11890_gb300 as tg
    from paper_2509_11890_gb300 import inputs

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    for n in [int(x) for x in a.sizes.split(",")]:
        g = inputs.rng(a.seed, 900 + n)
        K = torch.from_numpy(g.uniform(-1, 1, (n, n)) + 4.0 * np.eye(n)).cuda()
        x_true = torch.from_numpy(np.sin(0.37 * np.arange(n) + 1.0)).cuda()
        b0 = K @ x_true
        for pn in ("fp64", "tf32"):
            times, res = [], None
            for it in range(a.warmup + max(a.steps, 1)):
                b = b0.clone()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                res = tg.lu_solve(K, b, PREC[pn])
                e1.record(stream)
                torch.cuda.synchronize()
                if it >= a.warmup:
                    times.append(e0.elapsed_time(e1) * 1e-3)
            err = float(torch.linalg.norm(b - x_true) / torch.linalg.norm(x_true))
            t = min(times)
            fl = 2.0 / 3.0 * n ** 3 + 2.0 * n * n
            print(json.dumps({"micro": "dense local solve (tt_lu_solve)", "n": n, "precision": pn, "seconds": t,
                              "tflops": fl / t / 1e12, "rel_residual": res, "rel_error": err}), flush=True)
        # the same size as a reduced projected system (half dX, half multipliers)
        # solved by block elimination: SPD L_Z block, coupling blocks of unit scale
        nz = n // 2
        nm = n - nz
        if nz < 1 or nm < 1:
            continue
        Bm = g.uniform(-1, 1, (nz, nz))
        LZ = Bm @ Bm.T / nz + 2.0 * np.eye(nz)
        E = g.uniform(-1, 1, (nm, nz)) / np.sqrt(nz)
        F = g.uniform(-1, 1, (nm, nm)) / np.sqrt(nm) + 2.0 * np.eye(nm)
        G = g.uniform(-1, 1, (nz, nm)) / np.sqrt(nm)
        Ks = torch.from_numpy(np.block([[E, F], [LZ, G]])).cuda()
        bs0 = Ks @ x_true
        for pn in ("fp64", "tf32"):
            times, res = [], None
            tg.kkt_stats(reset=True)
            for it in range(a.warmup + max(a.steps, 1)):
                b = bs0.clone()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                res = tg.kkt_solve(Ks, b, nz, PREC[pn])
                e1.record(stream)
                torch.cuda.synchronize()
                if it >= a.warmup:
                    times.append(e0.elapsed_time(e1) * 1e-3)
            blocks, fp32, fallbacks = tg.kkt_stats(reset=True)
            err = float(torch.linalg.norm(b - x_true) / torch.linalg.norm(x_true))
            t = min(times)
            fl = nz ** 3 / 3.0 + 2.0 * nz * nz * nm + 2.0 * nz * nm * nm + 2.0 * nm ** 3 / 3.0
            print(json.dumps({"micro": "block elimination (tt_kkt_solve)", "n": n, "n_lz": nz, "precision": pn,
                              "seconds": t, "tflops": fl / t / 1e12, "rel_residual": res, "rel_error": err,
                              "block_solves": blocks, "fp32_factor_solves": fp32, "lu_fallbacks": fallbacks}),
                  flush=True)
    return 0


def run_micro_contract(a):
    """Contraction microbenchmark: one left and one right environment update
    and one local product (three-stage contractions, rows a6 and a7) at the shapes of the
    configured workloads: frame and vector ranks r, operator ranks R, modes
    4 x 4, with (r, R) = (16, 32), (64, 128), (128, 256). CUDA events on the
    launching stream around `steps` calls after `warmup`; algorithmic flops
    of the three stages (the library's own count). Beside each shape, the
    oracle's environment update (numpy einsum chain, FP64) timed on the host
    cores: the CPU baseline of the contraction throughput."""
    import torch

    import paper_2509_11890_gb300 as tg
    from oracle import tt as ott
    from paper_2509_11890_gb300 import inputs

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    peaks, kind = _peaks()
    for r, R in [(int(x.split(":")[0]), int(x.split(":")[1])) for x in a.shapes.split(",")]:
        dims = dict(rw=r, rw2=r, R=R, R2=R, rv=r, rv2=r, m=4, n=4)
        g = inputs.rng(a.seed, 700 + r)
        t = lambda *sh: torch.from_numpy(g.standard_normal(sh)).cuda()
        phi, u, op, v, psi = t(r, R, r), t(r, 4, r), t(R, 4, 4, R), t(r, 4, r), t(r, R, r)
        out = torch.empty(r * R * r, dtype=torch.float64, device="cuda")
        y = torch.empty(r * 4 * r, dtype=torch.float64, device="cuda")
        flops = (2.0 * r * R * r * 4 * r + 2.0 * r * r * (R * 4) * (4 * R) + 2.0 * r * R * r * r * 4)
        # CPU baseline: the oracle's update of the same operands, best of a few calls
        hp, hu, hop, hv = (x.cpu().numpy() for x in (phi, u, op, v))
        times = []
        for _ in range(3):
            t0 = time.perf_counter()
            ott.env_left_step(hp, hu, hop, hv)
            times.append(time.perf_counter() - t0)
            if sum(times) > 10.0:
                break
        cpu_s = min(times)
        print(json.dumps({"micro": "env_left (oracle, numpy einsum chain)", "r": r, "R": R, "precision": "fp64",
                          "seconds": cpu_s, "gflop": flops / 1e9, "tflops": flops / cpu_s / 1e12,
                          "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(),
                                           "sample": f"best of {len(times)} calls"}}), flush=True)
        for pn in ("fp64", "fp32", "tf32", "bf16"):
            for name, fn in (("env_left", lambda: tg.env_left_step(dims, phi, u, op, v, out, PREC[pn])),
                             ("env_right", lambda: tg.env_right_step(dims, psi, u, op, v, out, PREC[pn])),
                             ("local_apply", lambda: tg.local_apply(dims, phi, op, psi, v, y, PREC[pn]))):
                for _ in range(a.warmup):
                    fn()
                tg.contraction_stats_reset()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(max(a.steps, 1)):
                    fn()
                e1.record(stream)
                torch.cuda.synchronize()
                sec = e0.elapsed_time(e1) * 1e-3 / max(a.steps, 1)
                tf, ts, tl = tg.tc_stats()
                rec = {"micro": f"{name} (three-stage contraction)", "r": r, "R": R, "precision": pn,
                       "seconds": sec, "gflop": flops / 1e9, "tflops": flops / sec / 1e12}
                if tl:
                    tc = tf / ts / 1e12
                    pk = peaks["bf16_tflops_sustained"] * (0.5 if pn == "tf32" else 1.0)
                    rec["tc_gemm"] = {"launches_per_call": tl / max(a.steps, 1), "tflops": tc,
                                      "frac_of_peak": tc / pk, "peak": pk, "peak_source": f"{kind} bf16 sustained"}
                print(json.dumps(rec), flush=True)
    return 0


def main():
    a = _args()
    if a.micro == "lu":
        return run_micro_lu(a)
    if a.micro == "contract":
        return run_micro_contract(a)
    if a.impl == "reference":
        return run_reference(a)
    if WORKLOADS[a.workload]["kind"] == "batch":
        return run_batch(a)
    if WORKLOADS[a.workload]["kind"] in ("theta", "cc"):
        return run_other(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
