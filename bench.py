"""Benchmark: reduced-Hessian-vector products per second, FP64, 9241-bus-shaped grid.

A step is one pass of the whole hot path over the grid's current state, one
rh_reduced_hessian call: Jacobian assembly, LU refactorisation, adjoint and
projection coefficients, and the full reduced Hessian, all n_p = 2889 directions
(W = I) in flight at once in the direction kernel, whose SpMul/L/U half runs
beside the adjoint solve.  Throughput = n_p HVPs / step time.  Inputs are synthetic (seeded PEGASE9241
shape, see gridgen.py) and resident in HBM; the device workspace (~0.9 GB) is
larger than L2 and L2 is also flushed between timed steps.

e2e: the same metric through the C ABI with host buffers: parameters, loads and
the operating point copied in, the full H (66.8 MB) copied out, every step.

--impl reference times the CPU oracle (oracle/, plain C, the columns of W shared
out over the host cores) on the same workload.

--fp64-peak only measures the device's FP64 FMA rate by CTAs and warps per SM.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CASE = "case9241"
BLOCK_N = 256
# FP64 roofline of GB300, derived from unit counts at the maximum SM clock: 152 SMs x 4
# sub-partitions x 0.5 lane-FMA per clock x 2 flop x 2.070 GHz = 1258.6 GFLOP/s.  The FMA-chain
# measurement behind the 0.5 lane-FMA per clock per sub-partition (python bench.py --fp64-peak)
# is summarised in profiles/fp64_fma_rate.md; every run also reports the rate it measures.
PEAK_FP64_GFLOPS = 152 * 4 * 0.5 * 2 * 2.070


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--case", default=CASE)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass (profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 118-bus latency, scenario batching, plain-path and serving measurements")
    ap.add_argument("--fp64-peak", action="store_true",
                    help="only measure the FP64 FMA rate by CTAs and warps per SM and print the table")
    ap.add_argument("--only", choices=["case118_full_hessian", "scenario_batching", "serving", "tracking_step",
                                       "jacobian_ad"],
                    help="run only this extra measurement on one GPU and print its JSON (profiling runs)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Several GPUs run replicas: every rank computes the whole workload of a step (the
# directions and blocks are independent, no step exchanges data), so the job's
# time is the slowest rank's and its throughput is world x the per-rank units.
def max_over_ranks(value, world, device):
    """The largest of the ranks' values (all ranks call it; no-op for one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each process units_per_rank in `seconds`."""
    return world * units_per_rank / seconds


def measured_traffic():
    """DRAM bytes of one step's two k_dirs launches from the committed ncu capture, if the kernel
    source is unchanged."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "k_dirs_case9241_traffic.json")))
        csrc = os.path.join(ROOT, "paper_2201_00241_gb300", "csrc")
        sha = lambda f: hashlib.sha256(open(os.path.join(csrc, f), "rb").read()).hexdigest()
        # the kernels and the symbolic phase (ordering, schedules) both shape the traffic
        if sha("kernels.cu") == rec["kernels_cu_sha256"] and sha("symbolic.cpp") == rec.get("symbolic_cpp_sha256"):
            return int(rec["dram_bytes_per_step"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def start_clock_sampler(path):
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except (OSError, FileNotFoundError):
        return None


def read_clocks(path, dev):
    out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
    try:
        rows = [ln.split(",") for ln in open(path) if ln.strip()]
    except OSError:
        return out
    rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(dev)]
    if not rows:
        return out
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    out["sm_mhz"] = statistics.median(sm) if sm else None
    out["sm_max_mhz"] = float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = set()
    for r in rows:
        for k, name in enumerate(names):
            if r[5 + k].lower().startswith("active"):
                reasons.add(name)
    out["reasons"] = sorted(reasons)
    return out


def host_cpu():
    """Model name of the host cores (lscpu, else /proc/cpuinfo) and the cores this process may use."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                name = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    name = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return name or "unknown", int(cores or 1)


def cpu_baseline(case):
    """The oracle as it stands (plain C), timed on the whole workload of one step: all n_p
    unit directions of the full reduced Hessian, with its own per-state LU and adjoint.
    Once on one thread (like the paper's sequential CPU reference) and once with the
    columns shared out over every core the process may use (a few seconds each)."""
    from oracle import OracleGrid
    from paper_2201_00241_gb300 import gridgen as gg

    g = gg.make_case(case)
    o = OracleGrid(g)
    st = o.plant()
    W = np.eye(o.n_p)
    model, cores = host_cpu()
    t0 = time.perf_counter()
    o.hessvec(st.x, st.p, st.pd, st.qd, W)
    dt1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.hessvec(st.x, st.p, st.pd, st.qd, W, threads=cores)
    dtn = time.perf_counter() - t0
    return dict(value=o.n_p / dtn, unit="HVP/s", cores=cores, kind="oracle", host_cpu=model, nproc=os.cpu_count(),
                single_thread_value=o.n_p / dt1,
                sample=f"the whole step: all {o.n_p} unit directions of H on {case} (incl. the oracle's own LU and "
                       f"adjoint): {dtn:.2f} s on {cores} threads (columns shared out), {dt1:.1f} s on one")


def _ready(case, scale_k=None):
    from paper_2201_00241_gb300 import gridgen as gg
    from paper_2201_00241_gb300 import rh
    g = gg.make_case(case)
    lg = rh.Grid(g, device=torch_device_index())
    st = lg.plant()
    pd, qd = st.pd, st.qd
    if scale_k is not None:
        s = gg.load_scales(g.n_bus, scale_k + 1, g.seed)[scale_k]
        pd, qd = pd * s, qd * s
    lg.set_state(st.p, pd, qd)
    lg.powerflow(st.x, tol=1e-12, max_iter=20)
    lg.adjoint()
    return lg


def torch_device_index():
    import torch
    return torch.cuda.current_device()


def _colmajor(W):
    import torch
    return torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()


def _event_ms(fn, reps):
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_case118_latency(reps=20):
    """Full reduced Hessian of the 118-bus grid in blocks of N = 16 (7 blocks), per-state
    setup included: the blocks issued together in one rh_reduced_hessian call (Jacobians,
    refactorisation, adjoint beside the first direction sweeps, all 107 directions in
    flight), and, for comparison, rh_adjoint followed by one launch per block."""
    from paper_2201_00241_gb300 import rh
    lg = _ready("case118")
    lib = rh.load()
    import torch
    H = torch.empty((lg.n_p, lg.n_p), dtype=torch.float64, device="cuda").t()
    sptr = rh.C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def fused():
        rh._check(lib.rh_reduced_hessian(lg._h, rh._ptr(H), lg.n_p, None, None, sptr, rh.RH_DEVICE_PTRS))

    def blocks():
        rh._check(lib.rh_adjoint(lg._h, None, None, None))
        rh._check(lib.rh_hessian(lg._h, 16, rh._ptr(H), lg.n_p, sptr, rh.RH_DEVICE_PTRS))

    out = {"workload": "case118: full reduced Hessian, 107 columns in 7 blocks of N=16, setup included"}
    for name, fn in (("blocks_together", fused), ("block_by_block", blocks)):
        for _ in range(3):
            fn()
        t = [_event_ms(fn, 1) for _ in range(reps)]
        out[f"{name}_ms_p50"] = float(np.median(t))
        out[f"{name}_ms_min"] = float(np.min(t))
    out["latency_ms_p50"] = out["blocks_together_ms_p50"]
    return out


def measure_scenarios(n_scen=8, N=64, reps=10):
    """8 load scenarios of the 1354-bus grid, N=64 directions each: 8 plain launches vs one
    batched launch replayed from a captured CUDA graph, in the autotuned configuration
    (interleave width, CTA shape, narrow-level k-split cap and dense-tail bound)."""
    import torch
    from paper_2201_00241_gb300 import autotune
    from paper_2201_00241_gb300 import gridgen as gg
    from paper_2201_00241_gb300 import rh
    grids = [_ready("case1354", k) for k in range(n_scen)]
    resolve = measure_scenario_resolves(grids)
    for lg in grids:
        lg.adjoint()
    items = []
    for k, lg in enumerate(grids):
        W = _colmajor(gg.random_directions(lg.n_p, N, 1000 + k))
        HW = torch.empty((N, lg.n_p), dtype=torch.float64, device="cuda").t()
        work = torch.empty(rh.work_doubles(lg, N), dtype=torch.float64, device="cuda")
        items.append((lg, W, HW, work))

    def plain():
        for lg, W, HW, _ in items:
            lg.hessvec(W, HW)

    plain()
    t_plain = _event_ms(plain, reps)
    tuned = autotune.tune(items, tails=autotune.TAILS)
    default = next(r["ms"] for r in tuned["table"]
                   if (r["width"], r["threads"], r["split_lanes"], r["max_tail"]) == (0, 384, 32, int(grids[0].dims.max_tail)))
    tg = autotune.with_tail([lg for lg, _, _, _ in items], tuned["max_tail"])
    titems = [(g2,) + tuple(it[1:]) for g2, it in zip(tg, items)]
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    autotune.launch(titems, tuned)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            autotune.launch(titems, tuned, stream=rh.C.c_void_p(s.cuda_stream))
    graph.replay()
    t_batched = _event_ms(graph.replay, reps)
    total = n_scen * N
    top = sorted(tuned["table"], key=lambda r: r["ms"])[:5]
    return {"workload": f"case1354: {n_scen} load scenarios (per-bus loads x U[0.9,1.1], power flow re-solved), "
                        f"N={N} random unit directions each",
            "plain_hvp_per_s": total / (t_plain * 1e-3), "batched_hvp_per_s": total / (t_batched * 1e-3),
            "plain_ms": t_plain, "batched_ms": t_batched,
            "tuned": {k: tuned[k] for k in ("width", "threads", "ctas_per_sm", "split_lanes", "max_tail", "ms")},
            "tuning": {"configs_measured": len(tuned["table"]), "default_config_ms": default, "fastest": top,
                       "note": "tuning times are warm-L2 means of 3 launches: they rank configurations"},
            "batched_launch": "one rh_batch_hessvec_cfg, CUDA graph",
            "power_flow_resolve": resolve}


def measure_scenario_resolves(grids, reps=7):
    """Newton re-solves of the scenarios' power flows from the planted point (section 3.2,
    reading R20): each grid alone with rh_powerflow, one after another, against all of them
    in one rh_batch_powerflow call (host wall time, both synchronous)."""
    from paper_2201_00241_gb300 import rh
    import torch
    x0 = [lg.plant().x for lg in grids]

    def one_by_one():
        its = []
        for lg, x in zip(grids, x0):
            _, it, _, _ = lg.powerflow(x, tol=1e-12, max_iter=20)
            its.append(int(it))
        return its

    def batched():
        _, its, _, st = rh.batch_powerflow(grids, x0=x0, tol=1e-12, max_iter=20)
        assert (st == rh.RH_OK).all()
        return [int(v) for v in its]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            its = fn()
            ts.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(ts)), its

    t_seq, it_seq = timed(one_by_one)
    t_bat, it_bat = timed(batched)
    return {"sequential_ms": t_seq, "batched_ms": t_bat, "newton_iters": it_bat, "newton_iters_sequential": it_seq,
            "note": "re-solve of every scenario from the planted point to ||g||_inf <= 1e-12: rh_powerflow per "
                    "grid vs one rh_batch_powerflow (one host sync per iteration, graphs per active set)"}


def measure_rto(n_updates=12):
    """Real-time tracking updates (section 6.3, Table 3 workload: the 1354-bus grid).

    Each update takes new loads w_t, re-solves the power flow from the previous
    state, forms lambda and grad F (rh_adjoint), and runs rh_rto_step: the full
    reduced Hessian (Step 1), its Cholesky factorisation and the solve (Step 2).
    The step is computed but not applied: the synthetic cost has no operating
    limits, so full Newton steps would leave the region where the power flow
    has a solution."""
    import time
    import torch
    from paper_2201_00241_gb300 import gridgen as gg
    from paper_2201_00241_gb300 import rh
    g = gg.make_case("case1354")
    lg = rh.Grid(g, device=torch_device_index())
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    lg.powerflow(st.x)
    lg.adjoint()
    lib = rh.load()
    n = lg.n_p
    H = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    pn = torch.empty(n, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    sptr = rh.C.c_void_p(torch.cuda.current_stream().cuda_stream)
    noise = gg.load_scales(g.n_bus, n_updates + 3, g.seed)

    def loads(t):
        f = (1.0 + 0.03 * np.sin(2 * np.pi * t / 60.0)) * (1.0 + 0.2 * (noise[t] - 1.0))
        return st.pd * f, st.qd * f

    def rto():
        rh._check(lib.rh_rto_step(lg._h, rh._ptr(H), n, rh._ptr(d), rh._ptr(pn), rh._ptr(info), sptr, 0))

    def update(t):
        pd, qd = loads(t)
        lg.set_state(None, pd, qd)
        lg.powerflow()
        lg.adjoint()
        rto()

    for t in range(3):
        update(t)
    torch.cuda.synchronize()
    wall = []
    for t in range(3, n_updates + 3):
        t0 = time.perf_counter()
        update(t)
        torch.cuda.synchronize()
        wall.append((time.perf_counter() - t0) * 1e3)
    assert int(info.item()) == 0
    t_rto = _event_ms(rto, 10)
    t_hess = _event_ms(lambda: rh._check(lib.rh_hessian(lg._h, n, rh._ptr(H), n, sptr,
                                                        rh.RH_DEVICE_PTRS | rh.RH_HESSIAN_CONCURRENT)), 10)
    # rh_potrf alone on this H (n_p x n_p), replayed from a CUDA graph, H restored between runs
    H0 = H.clone()
    A = torch.empty_like(H0)
    gs = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(gs):
        A.copy_(H0)
        rh.potrf(A, stream=rh.C.c_void_p(gs.cuda_stream))
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=gs):
            rh.potrf(A, stream=rh.C.c_void_p(gs.cuda_stream))
    t_potrf = []
    for _ in range(20):
        A.copy_(H0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        t_potrf.append(e0.elapsed_time(e1))
    return {"workload": f"case1354: tracking updates with loads w_t = w_0 (1 + 0.03 sin(2 pi t / 60)) x per-bus "
                        f"U[0.98, 1.02]; n_p = {n}; step computed, not applied",
            "update_ms_p50": float(np.median(wall)), "update_ms_min": float(np.min(wall)),
            "rto_step_ms": t_rto, "step1_hessian_ms": t_hess, "step2_cholesky_solve_ms": t_rto - t_hess,
            "potrf_ms": float(np.median(t_potrf)), "potrf_n": n,
            "update_includes": "loads upload, warm-started Newton power flow, adjoint + gradient, "
                               "full reduced Hessian (one launch), Cholesky + solve",
            "paper_v100_s": {"step1": 0.05, "step2": 0.05, "total": 0.10, "cpu_total": 2.22}}


def measure_jacobian_ad(reps=10):
    """Coloured forward-mode Jacobian (section 4.2.2) against the analytic assembly on the
    9241-bus grid: colour counts, and the per-state setup (rh_adjoint: assembly, refactor,
    adjoint) with each assembly method."""
    from paper_2201_00241_gb300 import rh
    lg = _ready("case9241")
    lib = rh.load()
    _, _, ncx, ncp = lg.coloring()
    out = {"workload": "case9241: J_x (n_x columns) and J_p (n_p columns) at the planted point",
           "n_x": lg.n_x, "n_p": lg.n_p, "colors_x": ncx, "colors_p": ncp,
           "tangent_passes": (ncx + ncp + 7) // 8}
    for method in ("analytic", "ad"):
        lg.set_jacobian_method(method)
        rh._check(lib.rh_adjoint(lg._h, None, None, None))
        out[f"setup_ms_{method}"] = _event_ms(lambda: rh._check(lib.rh_adjoint(lg._h, None, None, None)), reps)
    lg.set_jacobian_method("analytic")
    return out


def measure_separate_calls(lg, H, sptr, reps=5):
    """The same step as two calls, rh_adjoint (synchronous) then rh_hessian, with
    nothing overlapped: the setup and the direction kernel timed apart."""
    from paper_2201_00241_gb300 import rh
    lib = rh.load()
    n_p = lg.n_p
    setup = _event_ms(lambda: rh._check(lib.rh_adjoint(lg._h, None, None, None)), reps)
    dirs = _event_ms(lambda: rh._check(lib.rh_hessian(lg._h, BLOCK_N, rh._ptr(H), n_p, sptr,
                                                       rh.RH_DEVICE_PTRS | rh.RH_HESSIAN_CONCURRENT)), reps)

    def both():
        rh._check(lib.rh_adjoint(lg._h, None, None, None))
        rh._check(lib.rh_hessian(lg._h, BLOCK_N, rh._ptr(H), n_p, sptr, rh.RH_DEVICE_PTRS | rh.RH_HESSIAN_CONCURRENT))
    step = _event_ms(both, reps)
    return {"step_ms": step, "setup_ms": setup, "hessian_ms": dirs, "hvp_per_s": n_p / (step * 1e-3)}


def measure_per_block(lg, H, sptr, reps=5):
    """The full Hessian in the metric's blocks of N = 256 columns, one launch per block (the
    plain block-by-block form of section 5.3), HVP only, state resident."""
    from paper_2201_00241_gb300 import rh
    lib = rh.load()
    rh._check(lib.rh_adjoint(lg._h, None, None, None))

    def blocks():
        rh._check(lib.rh_hessian(lg._h, BLOCK_N, rh._ptr(H), lg.n_p, sptr, rh.RH_DEVICE_PTRS))

    blocks()
    t = _event_ms(blocks, reps)
    return {"hvp_per_s": lg.n_p / (t * 1e-3), "ms": t, "blocks": -(-lg.n_p // BLOCK_N),
            "note": "HVP only (state resident): rh_hessian, one k_dirs launch per block of 256 columns"}


def measure_plain_paths(lg, n_single=32, reps=3):
    """The plain one-direction-at-a-time path and the one-launch-per-block full Hessian."""
    import torch
    from paper_2201_00241_gb300 import gridgen as gg
    from paper_2201_00241_gb300 import rh
    W = _colmajor(gg.random_directions(lg.n_p, n_single, 77))
    HW = torch.empty((n_single, lg.n_p), dtype=torch.float64, device="cuda").t()

    def singles():
        for j in range(n_single):
            lg.hessvec(W[:, j:j + 1], HW[:, j:j + 1])

    singles()
    t1 = _event_ms(singles, reps)
    lib = rh.load()
    H = torch.empty((lg.n_p, lg.n_p), dtype=torch.float64, device="cuda").t()
    sptr = rh.C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def blocks():
        rh._check(lib.rh_hessian(lg._h, BLOCK_N, rh._ptr(H), lg.n_p, sptr, rh.RH_DEVICE_PTRS))

    blocks()
    tb = _event_ms(blocks, reps)
    return {"n1_hvp_per_s": n_single / (t1 * 1e-3),
            "per_block_launches_hvp_per_s": lg.n_p / (tb * 1e-3),
            "note": "HVP only (state resident); N=1 calls one at a time / 12 launches of N=256"}


def measure_serving(factors=(0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 2.0), n_req=600, warm_req=50, seed=4, outstanding=128,
                    t_sat=2.0):
    """Poisson request stream over grids of 118, 1354, 2869 and 9241 buses (ratio 8:4:2:1),
    N ~ U{1..256} unit directions per request, through the continuous-batching server.

    Saturation is measured first, closed-loop: `outstanding` requests are kept in the
    server for t_sat seconds, each completion submitting the next from its future's
    callback (no client thread polls); its request rate is the 1x of the open-loop sweep
    that follows (Poisson arrivals at factors x saturation, the first warm_req requests of
    each rate left out of the latency percentiles)."""
    import threading
    import time as _t
    from paper_2201_00241_gb300 import autotune
    from paper_2201_00241_gb300 import gridgen as gg
    from paper_2201_00241_gb300.server import RHServer
    names = ["case118", "case1354", "case2869", "case9241"]
    weights = np.array([8, 4, 2, 1], dtype=float)
    weights /= weights.sum()
    grids = {n: _ready(n) for n in names}
    srv = RHServer(device=torch_device_index(), budget_bytes=16 << 30, max_batch=16, n_streams=4)
    for n, lg in grids.items():
        srv.register(n, lg)
    # launch configuration: tuned on a round of the mix's proportions at the mean N
    tuned = srv.tune([(n, 128) for n, c in zip(names, (8, 4, 2, 1)) for _ in range(c)], tails=autotune.TAILS)
    rng = np.random.default_rng(seed)

    def draw(k):
        name = names[rng.choice(4, p=weights)]
        N = int(rng.integers(1, 257))
        return name, gg.random_directions(grids[name].n_p, N, 10_000 + k)

    try:
        pool = [draw(k) for k in range(256)]
        for name, W in pool[:16]:
            srv.submit(name, W).result()                     # warm-up
        # each grid's request of N = 256 alone in the idle server (arrival to result)
        solo = {}
        for n in names:
            W = gg.random_directions(grids[n].n_p, 256, 77)
            ts = []
            for _ in range(5):
                t0 = _t.perf_counter()
                srv.submit(n, W).result()
                ts.append((_t.perf_counter() - t0) * 1e3)
            solo[n] = float(np.median(ts))
        lock = threading.Lock()
        st = {"k": 0, "done": 0, "hvp": 0, "live": 0, "count": False, "stop": False}
        drained = threading.Event()

        def submit_next():
            with lock:
                if st["stop"]:
                    return
                k = st["k"]
                st["k"] += 1
                st["live"] += 1
            name, W = pool[k % len(pool)]
            srv.submit(name, W).add_done_callback(lambda f, n=W.shape[1]: on_done(n))

        def on_done(n):
            with lock:
                st["live"] -= 1
                if st["count"]:
                    st["done"] += 1
                    st["hvp"] += n
                last = st["stop"] and st["live"] == 0
            if last:
                drained.set()
            submit_next()

        for _ in range(outstanding):
            submit_next()
        _t.sleep(0.3)                                        # reach the steady state
        with lock:
            st["count"] = True
        t0 = _t.perf_counter()
        _t.sleep(t_sat)
        with lock:
            st["count"] = False
            st["stop"] = True
            n_done, hvp_done = st["done"], st["hvp"]
            if st["live"] == 0:
                drained.set()
        dt = _t.perf_counter() - t0
        drained.wait(60)
        sat_req, sat_hvp = n_done / dt, hvp_done / dt
        rows = []
        # an unrecorded pass of the sweep's pattern at the first rate (allocator growth,
        # first-use costs), and a collection before each rate, so that a one-time host
        # stall does not land in the first rate's window
        for f in (None,) + tuple(factors):
            rate = (f if f is not None else factors[0]) * sat_req
            n_f = n_req if f is not None else 200
            stream = [draw(1000 * int(100 * (f if f is not None else 99)) + j) for j in range(n_f)]
            gaps = rng.exponential(1.0 / rate, n_f)
            gc.collect()
            srv.reset_latencies()
            h0 = dict(srv.host_s)
            t0 = _t.perf_counter()
            t_next = t0
            futs = []
            for (name, W), gap in zip(stream, gaps):
                t_next += gap
                wait = t_next - _t.perf_counter()
                if wait > 0:
                    _t.sleep(wait)          # releases the GIL for the server's worker thread
                futs.append(srv.submit(name, W))
            for fu in futs:
                fu.result()
            dt = _t.perf_counter() - t0
            if f is None:
                continue
            st = srv.stats(skip=warm_req)
            rows.append({"rate_factor": f, "offered_req_per_s": rate, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                         "throughput_req_per_s": n_req / dt,
                         "throughput_hvp_per_s": sum(W.shape[1] for _, W in stream) / dt,
                         "per_grid": {n: (round(v["p50_ms"], 3), round(v["p99_ms"], 3)) for n, v in st["per_grid"].items()},
                         "worker_busy": {k: (srv.host_s[k] - h0[k]) / dt for k in h0}})
        return {"workload": "Poisson requests over case118/1354/2869/9241 (8:4:2:1), N ~ U{1..256}",
                "saturated_req_per_s": sat_req, "saturated_hvp_per_s": sat_hvp,
                "saturation": f"closed loop, {outstanding} requests outstanding for {t_sat:.0f} s, each "
                              "completion submitting the next from its callback",
                "sweep": rows, "sweep_requests": f"{n_req} per rate, percentiles over all but the first {warm_req}; an "
                                                  "unrecorded pass of 200 at the first rate before the sweep",
                "alone_n256_ms": solo,
                "batches": srv.batches, "waited_for_budget": srv.waited_for_budget,
                "tuned": {k: tuned[k] for k in ("width", "threads", "ctas_per_sm", "split_lanes", "max_tail", "ms")},
                "tuned_on": "one round of 15 requests (8:4:2:1 over the four grids), N = 128 each"}
    finally:
        srv.close()


def workload_config(case, n_x, n_p, nnz_l, nnz_u, world):
    return {"workload": f"{case}: full reduced Hessian ({n_p} HVPs) per step, W = I, all {n_p} directions "
                        f"in flight in one pair of direction launches (at most 10 per CTA), per-state setup "
                        f"(Jacobian, refactor, adjoint) included; the metric's blocks of N={BLOCK_N}, one "
                        f"launch each, are reported beside it (per_block_n256)",
            "n_x": n_x, "n_p": n_p, "block_n": BLOCK_N, "nnz_l": nnz_l, "nnz_u": nnz_u,
            "l2": "flushed between steps; workspace > L2", "parallelism": "replicas" if world > 1 else "1 GPU"}


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, on the same workload: every step is the
    whole full reduced Hessian (all n_p unit directions, with the oracle's own per-state
    LU and adjoint), timed after W untimed warm-up steps."""
    if rank != 0:
        return
    from oracle import OracleGrid
    from paper_2201_00241_gb300 import gridgen as gg
    g = gg.make_case(args.case)
    o = OracleGrid(g)
    st = o.plant()
    per = o.n_p
    W = np.eye(o.n_p)
    model, cores = host_cpu()
    for _ in range(args.warmup):
        o.hessvec(st.x, st.p, st.pd, st.qd, W, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.hessvec(st.x, st.p, st.pd, st.qd, W, threads=cores)
        times.append(time.perf_counter() - t0)
    value = per * len(times) / sum(times)
    sym = o.symbolic()
    line = {"impl": "reference", "metric": "reduced-Hessian HVPs/sec FP64 (9241-bus-shaped grid, N=256)",
            "value": value, "unit": "HVP/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.case, o.n_x, o.n_p, len(sym["Lj"]), len(sym["Uj"]), 1),
            "cpu_baseline": {"value": value, "unit": "HVP/s", "cores": cores, "kind": "oracle", "host_cpu": model,
                             "nproc": os.cpu_count(),
                             "sample": f"each step: all {per} unit directions of the full Hessian, "
                                       f"with the oracle's own LU and adjoint; columns shared out over {cores} "
                                       "threads"},
            "e2e": {"value": value, "unit": "HVP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fp64_peak_table(device):
    """FP64 FMA rate (8 independent chains per thread) by CTAs and threads per SM."""
    from paper_2201_00241_gb300 import rh
    rows = []
    for ctas, threads in [(1, 128), (1, 256), (2, 128), (1, 384), (2, 256), (1, 768), (2, 384), (3, 384),
                          (2, 512), (4, 384), (2, 1024)]:
        best = 0.0
        for _ in range(3):
            gf, ms = rh.fp64_fma_rate(device, ctas, threads, 1 << 16)
            best = max(best, gf)
        rows.append({"ctas_per_sm": ctas, "threads_per_cta": threads, "warps_per_sm": ctas * threads // 32,
                     "gflops": best})
    return rows


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    if args.fp64_peak:
        torch.cuda.set_device(local)
        clk_path = os.path.join(tempfile.gettempdir(), f"rh_peak_clocks_{os.getpid()}.csv")
        sampler = start_clock_sampler(clk_path)
        time.sleep(1.0)
        rows = fp64_peak_table(local)
        if sampler:
            sampler.terminate()
            sampler.wait()
        print(json.dumps({"fp64_fma_rate": rows, "derived_peak_gflops": PEAK_FP64_GFLOPS,
                          "clocks": read_clocks(clk_path, local)}), flush=True)
        return

    if args.only:
        torch.cuda.set_device(local)
        fn = {"case118_full_hessian": measure_case118_latency, "scenario_batching": measure_scenarios,
              "serving": measure_serving, "tracking_step": measure_rto, "jacobian_ad": measure_jacobian_ad}
        print(json.dumps({args.only: fn[args.only]()}), flush=True)
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2201_00241_gb300 import gridgen as gg
    from paper_2201_00241_gb300 import rh

    g = gg.make_case(args.case)
    lg = rh.Grid(g, device=local)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    lg.powerflow(st.x, tol=1e-12, max_iter=20)
    dm = lg.dims
    n_p = lg.n_p
    lib = rh.load()
    # FP64 flops of the two direction launches of a step, counted by the library from the
    # symbolic data: Algorithm 2 for n_p dense directions, and what the kernels issue with W = I
    flops_alg, flops_exec = lg.reduced_hessian_flops()
    # the FP64 FMA rate of this device, in the direction kernel's shape (2 CTAs of 384 threads per SM)
    peak_meas = max(rh.fp64_fma_rate(local, 2, 384, 1 << 14)[0] for _ in range(3))

    H = torch.empty((n_p, n_p), dtype=torch.float64, device=f"cuda:{local}").t()   # column-major
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()
    sptr = rh.C.c_void_p(stream.cuda_stream)

    def step():
        rh._check(lib.rh_reduced_hessian(lg._h, rh._ptr(H), n_p, None, None, sptr, rh.RH_DEVICE_PTRS))

    # the clock sampler starts before the warm-up, so that its start-up (NVML initialisation)
    # is over before the timed steps; it keeps sampling through them
    # the raw samples go to RH_BENCH_CLOCKS_CSV (with _rank<r> before .csv) when it is set, else to a
    # temporary file; the JSON line carries their summary
    clk_env = os.environ.get("RH_BENCH_CLOCKS_CSV")
    clk_path = (clk_env[:-4] if clk_env and clk_env.endswith(".csv") else clk_env) + f"_rank{rank}.csv" if clk_env \
        else os.path.join(tempfile.gettempdir(), f"rh_bench_clocks_{os.getpid()}_rank{rank}.csv")
    sampler = start_clock_sampler(clk_path)
    time.sleep(1.0)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # kernels per timed step: those of rh_reduced_hessian's captured graph (counted by the library)
    dm_run = rh.Dims()
    rh._check(lib.rh_grid_dims(lg._h, rh.C.byref(dm_run)))
    launches_per_step = int(dm_run.hessian_kernels)
    if world > 1:
        torch.distributed.barrier()
    step_ms, dirs_ms, phase_ms = [], [], []
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)           # L2 flush, outside the timed events
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        # the direction launches, timed by the library's CUDA events on the stream they run on
        times = lg.reduced_hessian_times()
        dirs_ms.append(times[0])
        phase_ms.append(times[1:])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    if sampler:
        sampler.terminate()
        sampler.wait()
    t_step = max_over_ranks(sum(step_ms) / len(step_ms), world, f"cuda:{local}")
    value = replica_throughput(n_p, world, t_step * 1e-3)
    t_dirs = sum(dirs_ms) / len(dirs_ms)
    achieved = flops_alg / (t_dirs * 1e-3) * 1e-9
    achieved_exec = flops_exec / (t_dirs * 1e-3) * 1e-9
    # the plain form of the metric's N = 256 blocks: one launch per block of 256 columns
    per_block = measure_per_block(lg, H, sptr)

    # e2e through the C ABI with host buffers: H lands in pinned host memory (column-major)
    import torch
    Hh_t = torch.empty(n_p * n_p, dtype=torch.float64).pin_memory()
    Hh = Hh_t.numpy().reshape(n_p, n_p, order="F")
    x0 = st.x.copy()
    e2e_t = []
    for i in range(0 if args.no_e2e else args.warmup + args.steps):
        t0 = time.perf_counter()
        lg.set_state(st.p, st.pd, st.qd)
        lg.powerflow(x0, tol=1e-12, max_iter=20)
        rh._check(lib.rh_reduced_hessian(lg._h, rh._ptr(Hh), n_p, None, None, None, rh.RH_HOST_PTRS))
        if i >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_t) / len(e2e_t), world, f"cuda:{local}") if e2e_t else None
    e2e_value = replica_throughput(n_p, world, e2e_s) if e2e_t else None
    h2d = 8 * (n_p + 2 * g.n_bus + lg.n_x)
    d2h = 8 * n_p * n_p + 8 * (lg.n_x + n_p + 1)

    if rank != 0:
        return
    clocks = read_clocks(clk_path, local)
    line = {
        "metric": "reduced-Hessian HVPs/sec FP64 (9241-bus-shaped grid, N=256)",
        "value": value, "unit": "HVP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.case, lg.n_x, n_p, dm.nnz_l, dm.nnz_u, world),
        "per_block_n256": per_block,
        "roofline": {"bound": "alu", "kernel": "k_dirs (two launches per step: SpMul + L + U sweeps, then "
                                                 "projection + U^T + L^T sweeps + SpMulAdd)",
                     "achieved": achieved, "peak": PEAK_FP64_GFLOPS,
                     "unit": "GFLOP/s", "frac": achieved / PEAK_FP64_GFLOPS,
                     "traffic": measured_traffic() if args.case == CASE else None,
                     "kernel_ms": t_dirs, "flops_per_direction": flops_alg / n_p,
                     "achieved_executed": achieved_exec, "frac_executed": achieved_exec / PEAK_FP64_GFLOPS,
                     "flops_executed_per_step": flops_exec, "flops_algorithmic_per_step": flops_alg,
                     "peak_measured": peak_meas, "frac_of_measured_peak": achieved / peak_meas,
                     "frac_executed_of_measured_peak": achieved_exec / peak_meas,
                     "peak_note": "peak derived from unit counts at 2070 MHz (152 SMs x 4 sub-partitions x 0.5 "
                                  "lane-FMA/clk x 2); peak_measured: FMA chains in 2 x 384 threads per SM, "
                                  "this run",
                     "first_launch_end_ms": float(np.mean([p[0] for p in phase_ms])),
                     "adjoint_branch_end_ms": float(np.mean([p[1] for p in phase_ms])),
                     "note": "frac: Algorithm 2's flops for n_p dense directions (rh_reduced_hessian_flops); "
                             "frac_executed: the flops the launches issue with W = I (forward L sweep over each "
                             "CTA's reach, last L^T sweep over the rows SpMulAdd reads, no multiplications in "
                             "SpMul)"},
        "e2e": {"value": e2e_value, "unit": "HVP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step,
        "clocks": clocks,
    }
    if not args.no_extras:
        line["separate_calls"] = measure_separate_calls(lg, H, sptr)
        line["plain_paths"] = measure_plain_paths(lg)
        line["case118_full_hessian"] = measure_case118_latency()
        line["scenario_batching"] = measure_scenarios()
        line["serving"] = measure_serving()
        line["tracking_step"] = measure_rto()
        line["jacobian_ad"] = measure_jacobian_ad()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.case)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
