"""Benchmark of the HEOM-2DVS hot path on GB300 (one JSON line on rank 0).

Metric: HEOM ADO-updates/s (one ADO of one branch advanced by one full RK4
step) and the derived 2D spectra/hour, for the mixed-precision and plain FP64
GPU paths.

A timed "step" is one sample period of the t3 phase of the 2D scan over the
whole batched branch set of the workload: m RK4 steps of all 2*n1 branches
(rephasing + non-rephasing) x all ADOs, then the FP64 trace of every branch.
This is the loop that carries >99% of a spectrum's work; the remaining rows of
the path (equilibration, kicks, t1 trunk, t2, 2D DFT) run inside the e2e
measurement, which calls the public C ABI (heom_response_2d_rows) on a block of
t1 rows with the equilibrium state uploaded from pinned host memory each step.

--impl reference times the FP64 CPU oracle (tests' reference implementation)
on the host cores on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOADS = {
    # name: (config, precision code, e2e rows per step)
    "c3-mixed": ("c3", 2, 16),
    "c3-fp32": ("c3", 1, 16),
    "c2-fp64": ("c2", 0, 2),
    "c3-fp64": ("c3", 0, 2),
    "c1-fp64": ("c1", 0, 64),
    "c4-grad": ("c4", 0, 0),       # adjoint gradient of the spectrum misfit (own JSON line)
    "c5-window": ("c5", 0, 0),     # c5 RK4 steps on a few branches, projected spectra/hour
}
PREC_NAME = {0: "f64", 1: "f32", 2: "fp16x2-tc-f32acc"}


def describe(cfg, model, grid, d, nado):
    return {"workload": "%s: %d-mode MAB, d=%d, %d ADOs (L=%d), %dx%d t1xt3, t2=%s fs, dt=%g fs, m=%d"
            % (cfg, len(model["modes"]), d, nado, model["depth_L"], grid["n1"], grid["n3"],
               grid["t2_fs"], grid["dt_fs"], grid["steps_per_sample"]),
            "branches": 2 * grid["n1"], "d": d, "n_ado": nado}


def ado_updates_per_spectrum(grid, nado, n_t2_index=0):
    """ADO-updates of one full spectrum (one t2): trunk + t2 + t3 for both pathways."""
    n1, n3, m = grid["n1"], grid["n3"], grid["steps_per_sample"]
    t2 = sorted(grid["t2_fs"])[n_t2_index]
    n2 = int(round(t2 / grid["dt_fs"]))
    B = 2 * n1
    return nado * ((n1 - 1) * m + B * n2 + B * (n3 - 1) * m)


def rows_ado_updates(grid, nado, j0, j1):
    m, n3 = grid["steps_per_sample"], grid["n3"]
    B = 2 * (j1 - j0)
    n2 = max(int(round(t / grid["dt_fs"])) for t in grid["t2_fs"])
    return nado * ((j1 - 1) * m + B * n2 + len(grid["t2_fs"]) * B * (n3 - 1) * m)


# ---------------------------------------------------------------------------
# Algorithmic cost per ADO-update of the fused stage kernel
# ---------------------------------------------------------------------------
def algorithmic_costs(model, d, nado, ado_table, nb_counts, prec):
    """Algorithmic flops and bytes of one ADO-update (one ADO advanced by one RK4 step).

    bytes: 20 d^2 b -- four RK4 stages, each reading the stage input, the step-start
    state and the accumulator and writing two arrays (5 passes of d^2 complex, b = 16
    for complex128, 8 for complex64), neighbour re-reads served from L2.
    flops: 4 stages x ([H, w] with a real H: 8 d^3; per mode s the neighbour sums
    (8 d^2 per coupling entry) and V_s applied to A_s, B_s from both sides
    (16 d^2 n_s); decay and update 8 d^2).
    The byte count is that of the classic tableau; the nested (Horner) form the
    library runs needs 11 d^2 b (each stage reads its input and y and writes its
    output; the last stage reads y once), which the caller reports beside it.
    """
    dims = [md["n_levels"] for md in model["modes"]]
    avg_nb = nb_counts.sum(axis=0) / nado   # per mode
    stage = 8.0 * d ** 3 + 8.0 * d * d
    for s, n in enumerate(dims):
        stage += 8.0 * d * d * avg_nb[s] + (16.0 * d * d * n if avg_nb[s] > 0 else 0.0)
    flops = 4.0 * stage
    b = 16.0 if prec == 0 else 8.0
    return flops, 20.0 * d * d * b


# Measured DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per work item
# (one ADO of one branch) of one RK4 stage of the tensor-core path: one ncu capture
# of a 4-branch c3 case, scaled per item (the per-branch working set is the same at
# 256 branches), keyed by the stage kernels' source tag (heom_source_tag: any edit of
# their source gives another tag) and the coupling kernel's shape (rows per thread,
# row groups, ADOs per block, flags).  A build or shape without a capture reports none.
TC_STAGE_TRAFFIC_BYTES_PER_ITEM = {("004539086727f616", (8, 1, 1, 1)): 758.2e3}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(cfg, budget_s=12.0, max_steps=50):
    """Time oracle RK4 steps of one branch of the workload (FP64, host cores)."""
    from oracle import heom as OH
    from oracle import model as OM
    model, grid = W.config(cfg)
    prob = OM.Problem(model)
    rng = np.random.default_rng(3)
    x = (rng.standard_normal((1, prob.nado, prob.d, prob.d))
         + 1j * rng.standard_normal((1, prob.nado, prob.d, prob.d))) * 1e-3
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        x = OH.rk4_step(prob, x, grid["dt_fs"])
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": steps * prob.nado / dt, "unit": "ADO-updates/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "%d FP64 RK4 step(s) of one branch (%d ADOs, d=%d) of %s, numpy/BLAS on %d "
                      "host threads" % (steps, prob.nado, prob.d, cfg, os.cpu_count()),
            "seconds": dt}


def run_reference(args, cfg, rank, world):
    if rank != 0:
        return
    vals = []
    t_all = time.perf_counter()
    for i in range(args.warmup + args.steps):
        r = oracle_sample(cfg, budget_s=max(2.0, 30.0 / (args.warmup + args.steps)), max_steps=20)
        if i >= args.warmup:
            vals.append(r)
    value = float(np.mean([v["value"] for v in vals]))
    model, grid = W.config(cfg)
    # the native arm's config for the same workload (the oracle times a bounded sample of it)
    from oracle import model as OM
    prob = OM.Problem(model)
    prec = WORKLOADS[args.workload][1]
    conf = describe(cfg, model, grid, prob.d, prob.nado)
    B = 2 * grid["n1"]
    conf.update({"parallelism": "replicas" if world > 1 else "single-gpu",
                 "l2": "inputs larger than L2 (state %.1f GB)"
                       % (B * prob.nado * prob.d ** 2 * (16 if prec == 0 else 8) / 1e9),
                 "precision": PREC_NAME[prec]})
    line = {"impl": "reference", "metric": "HEOM ADO-updates/s (2D spectra/hour derived)",
            "value": value, "unit": "ADO-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean([v["seconds"] for v in vals])),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded water-like MAB model)",
            "config": dict(conf, precision="f64"),
            "cpu_baseline": {"value": value, "unit": "ADO-updates/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": value, "unit": "ADO-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
def run_grad(args, local):
    """One heom_response_2d_grad call on the c4 model (FP64), timed end to end.

    S_ref is the library's own S_C at theta_ref = theta (1 + 0.05 U(-1, 1)), seed 2604;
    the grid is the c4 grid cut to --grad-n x --grad-n (t1 x t3).  value = ADO-updates of
    the forward procedure (equilibration, trunk, both pathways' t3 scans) per second of
    the whole gradient call (forward, recomputation, reverse pass, host chain rule).
    """
    import torch
    torch.cuda.set_device(local)
    from paper_2601_20550_gb300 import heom as H
    model, grid = W.config("c4")
    grid["n1"] = grid["n3"] = args.grad_n
    th = H.theta_of(model)
    rng = np.random.default_rng(2604)
    m_ref = H.with_theta(model, th * (1 + 0.05 * rng.uniform(-1, 1, th.size)))
    h_ref = H.heom_build_hierarchy(m_ref, 0)
    eq_ref = H.heom_equilibrate(h_ref, grid["dt_fs"], grid["t_eq_fs"], 0.0)
    S_ref = H.heom_response_2d(h_ref, eq_ref, grid)[2]
    h = H.heom_build_hierarchy(model, 0)
    eq = H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0)
    nado, m, n1, n3 = h.n_ado, grid["steps_per_sample"], grid["n1"], grid["n3"]
    fwd = (round(grid["t_eq_fs"] / grid["dt_fs"]) + (n1 - 1) * m + 2 * n1 * (n3 - 1) * m) * nado
    torch.cuda.synchronize()
    n_launch0 = H.heom_launch_count()
    t0 = time.perf_counter()
    loss, g = H.heom_response_2d_grad(h, eq, grid, S_ref, 64)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    launches = H.heom_launch_count() - n_launch0
    # optional check against Richardson-extrapolated central differences of the
    # library's own FP64 loss (step 1e-3 |theta_i| and half of it: O(step^4))
    fd_check = None
    if args.grad_fd > 0:
        def lib_loss(t):
            hh = H.heom_build_hierarchy(H.with_theta(model, t), 0)
            e = H.heom_equilibrate(hh, grid["dt_fs"], grid["t_eq_fs"], 0.0)
            return float(np.sum((H.heom_response_2d(hh, e, grid)[2] - S_ref) ** 2))

        w = np.maximum(np.abs(th), 1.0)

        def central(i, step):
            tp, tm = th.copy(), th.copy()
            tp[i] += step
            tm[i] -= step
            return (lib_loss(tp) - lib_loss(tm)) / (2 * step)

        scale = float(np.max(np.abs(g * w)))
        entries = []
        t_fd = time.perf_counter()
        for i in (0, 4, 7, 10)[:args.grad_fd]:
            step = 1e-3 * w[i]
            fd = (4 * central(i, step / 2) - central(i, step)) / 3
            entries.append({"theta": i, "adjoint": float(g[i]), "fd": float(fd),
                            "rel_err": abs(g[i] - fd) / max(abs(fd), 1e-300),
                            "err_over_max_theta_grad": abs(g[i] - fd) * w[i] / scale})
        fd_check = {"method": "Richardson central differences of the library's FP64 loss",
                    "entries": entries, "seconds": time.perf_counter() - t_fd}
    print(json.dumps({
        "metric": "c4 misfit gradient, forward-equivalent HEOM ADO-updates/s", "value": fwd / el,
        "unit": "ADO-updates/s", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True,
        "dtype": "f64", "data": "synthetic (seeded water-like MAB model; S_ref from seeded theta_ref)",
        "config": {"workload": "c4: 3-mode MAB, d=%d, %d ADOs (L=4), %dx%d t1xt3, t2=0, dt=0.5 fs, m=8, "
                               "12 parameters, checkpoints every 64 steps" % (h.d, nado, n1, n3)},
        "seconds_per_gradient": el, "forward_ado_updates": fwd, "loss": loss,
        "dtheta": list(map(float, g)), "gpu_launches": int(launches), "fd_check": fd_check}))


def run_c5_window(args, local):
    """c5 (d = 216, 24310 ADOs) on a window: --steps RK4 steps of --branches branches
    (default 2) after --warmup steps, FP64 (--c5-precision 0) or FP32 coupling basis (1),
    device-timed; spectra/hour projected from ADO-updates per spectrum (t2 = 0).  The
    state is a kicked unit hierarchy (timing does not depend on the values)."""
    import torch
    torch.cuda.set_device(local)
    from paper_2601_20550_gb300 import heom as H
    model, grid = W.config("c5")
    prec = args.c5_precision
    h = H.heom_build_hierarchy(model, prec)
    d, nado = h.d, h.n_ado
    B = args.branches if args.branches > 0 else 2
    cdt = torch.complex128 if prec == 0 else torch.complex64
    y = torch.zeros((B, nado, d, d), dtype=cdt, device="cuda")
    y[:, 0, 0, 1] = 1.0
    y[:, 0, 1, 0] = 1.0
    wa, wb = torch.empty_like(y), torch.empty_like(y)
    sp = torch.cuda.current_stream().cuda_stream
    for _ in range(args.warmup):
        H.heom_propagate_dev(h, y.data_ptr(), wa.data_ptr(), wb.data_ptr(), B, prec, grid["dt_fs"], 1, sp)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = H.heom_launch_count()
    s.record()
    H.heom_propagate_dev(h, y.data_ptr(), wa.data_ptr(), wb.data_ptr(), B, prec, grid["dt_fs"], args.steps, sp)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / args.steps
    value = B * nado / (ms / 1e3)
    per_spec = ado_updates_per_spectrum(grid, nado)
    print(json.dumps({
        "metric": "HEOM ADO-updates/s (c5 window, projected 2D spectra/hour)", "value": value,
        "unit": "ADO-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "dtype": "f64" if prec == 0 else "f32",
        "data": "synthetic (seeded water-like MAB model; no dataset)",
        "config": {"workload": "c5: 3-mode MAB, d=%d, %d ADOs (L=8, K_s=2), %d branches, dt=0.25 fs"
                               % (d, nado, B), "state_GB": B * nado * d * d * (16 if prec == 0 else 8) / 1e9},
        "projected_spectra_per_hour": 3600.0 * value / per_spec, "ado_updates_per_spectrum": per_spec,
        "gpu_launches": int(H.heom_launch_count() - n0)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="c3-mixed", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--e2e-rows", type=int, default=0, help="t1 rows per e2e step (default per workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--grad-n", type=int, default=16, help="t1 and t3 samples of the c4-grad workload")
    ap.add_argument("--grad-fd", type=int, default=0,
                    help="c4-grad: check this many gradient entries (<= 4) against finite differences")
    ap.add_argument("--c5-precision", type=int, default=0, choices=[0, 1], help="c5-window: 0 FP64, 1 FP32")
    ap.add_argument("--tc-shape", type=int, default=-1,
                    help="force the tensor-core path's coupling-kernel shape 0-16 (profiling runs only)")
    ap.add_argument("--branches", type=int, default=0,
                    help="override the batch (profiling runs only; default 2*n1)")
    args = ap.parse_args()
    cfg, prec, e2e_rows = WORKLOADS[args.workload]

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, cfg, rank, world)
        return
    if args.workload == "c4-grad":
        if rank == 0:
            run_grad(args, local)
        return
    if args.workload == "c5-window":
        if rank == 0:
            run_c5_window(args, local)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2601_20550_gb300 import heom as H

    model, grid = W.config(cfg)
    h = H.heom_build_hierarchy(model, prec)
    d, nado = h.d, h.n_ado
    if args.tc_shape >= 0:
        H.heom_debug_force_tc_shape(args.tc_shape)
    # the FP64 equilibration of Sec. II.C.1 (timed: its share enters spectra/hour)
    H.heom_state_create(h, 1, 0)
    torch.cuda.synchronize()
    t_eq0 = time.perf_counter()
    eq = H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0)
    torch.cuda.synchronize()
    eq_seconds = time.perf_counter() - t_eq0
    m = grid["steps_per_sample"]
    B = args.branches if args.branches > 0 else 2 * grid["n1"]
    cdt = torch.complex128 if prec == 0 else torch.complex64
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    # batched t3 state: every branch starts from mu_plus^x rho_eq (the third kick)
    eqB = H.heom_state_create(h, B, prec)
    H.heom_state_broadcast(eq, eqB)
    y = torch.empty((B, nado, d, d), dtype=cdt, device=dev)
    H.heom_kick_dev(h, H.heom_state_device_ptr(eqB), y.data_ptr(), B, prec, 1, sp)
    torch.cuda.synchronize()
    del eqB
    wa = torch.empty_like(y)
    wb = torch.empty_like(y)
    traces = torch.zeros((args.warmup + args.steps, B), dtype=torch.complex128, device=dev)
    torch.cuda.synchronize()

    ops = H.heom_get_operators(h)
    nb = np.zeros((nado, len(model["modes"])))
    bath = ops["bath"]
    ado = ops["ado"]
    for i in range(nado):
        for j in range(h.n_exp):
            s = int(bath[j, 0])
            nb[i, s] += (ado[i, j] > 0)
            nb[i, s] += (ado[i].sum() < model["depth_L"])
    flops_upd, bytes_upd = algorithmic_costs(model, d, nado, ado, nb, prec)

    def one_step(i, ev=None):
        if ev is not None:
            ev[0].record(stream)
        H.heom_propagate_dev(h, y.data_ptr(), wa.data_ptr(), wb.data_ptr(), B, prec,
                             grid["dt_fs"], m, sp)
        if ev is not None:
            ev[1].record(stream)
        H.heom_trace_dev(h, y.data_ptr(), B, prec, 3, traces[i].data_ptr(), sp)

    for i in range(args.warmup):
        one_step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    n_launch0 = H.heom_launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(args.steps):
        one_step(args.warmup + i, evs[i])
    stop.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = H.heom_launch_count() - n_launch0
    clocks = clk.stop()
    t_ms = start.elapsed_time(stop)
    prop_ms = sum(a.elapsed_time(b) for a, b in evs)
    if dist:
        t = torch.tensor([t_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    if not torch.isfinite(traces.real).all():
        raise RuntimeError("non-finite traces in the timed region")
    units = float(B) * nado * m * args.steps * world
    value = units / (t_ms / 1000.0)
    per_spec = ado_updates_per_spectrum(grid, nado)
    stage_launches = 4 * m * args.steps
    stage_s = prop_ms / 1000.0 / stage_launches
    per_launch_units = B * nado / 4.0       # one stage = a quarter of an ADO-update per ADO
    # (for the tensor-core path a "stage" is the launch pair tc_stage_kernel + vterm_kernel)
    peaks, peak_kind = measured_peaks()
    if prec == 0:
        achieved = flops_upd * per_launch_units / stage_s / 1e12
        peak = 1.25
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "stage_kernel<double>",
                "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s); cuBLAS DGEMM measured 1.10",
                "algorithmic_flops_per_ado_update": flops_upd}
    else:
        achieved = bytes_upd * per_launch_units / stage_s / 1e9
        peak = peaks["hbm_gbs"]
        traffic = None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "RK4 stage (tc_stage_kernel + vterm_kernel)" if prec == 2 else "stage_kernel_vb",
                "peak_source": "%s hbm_gbs (MEASURED_PEAKS.json)" % peak_kind,
                "algorithmic_bytes_per_ado_update": bytes_upd,
                "algorithmic_bytes_basis": "classic RK4 tableau, 20 d^2 b per ADO-update",
                "frac_nested_form": achieved * (11.0 / 20.0) / peak,
                "nested_form_bytes_per_ado_update": bytes_upd * 11.0 / 20.0,
                "flops_TFLOPs": flops_upd * per_launch_units / stage_s / 1e12}
        if prec == 2:
            # the coupling kernel's launch shape the autotuner chose for this batch
            tuned = [e for e in H.heom_get_tuning(h) if e[0] == 2 and e[1] == B * nado * d * d]
            if args.tc_shape >= 0:
                roof["coupling_kernel_shape"] = {"forced": args.tc_shape}
            elif tuned:
                shape = H.heom_get_tc_shape(h, tuned[0][1])
                roof["coupling_kernel_shape"] = {"rows_per_thread": shape[0], "row_groups": shape[1],
                                                 "ados_per_block": shape[2], "l2_prefetch": shape[3] & 1,
                                                 "two_sources_in_flight": shape[3] >> 1,
                                                 "threads": tuned[0][2], "blocks": tuned[0][3]}
                tag = H.heom_source_tag()
                roof["kernel_source_tag"] = tag
                per_item = TC_STAGE_TRAFFIC_BYTES_PER_ITEM.get((tag, tuple(shape)))
                if per_item and cfg == "c3":
                    roof["traffic"] = per_item * B * nado

    # ---------------- error against the FP64 path ----------------
    # (a) the timed traces: every branch of the timed batch started from the same
    #     kicked state, so one FP64 branch propagated through the same (warm-up +
    #     timed) sample periods is the reference for all of them;
    # (b) the full t3 length of the workload (n3 samples of m RK4 steps) on one
    #     branch in the same precision, against the same FP64 branch continued.
    # (The FP64 path matches the oracle to 1e-10 on the test models.)
    error = None
    if prec != 0 and not args.no_fp64:
        h64e = H.heom_build_hierarchy(model, 0)
        s64 = H.heom_state_create(h64e, 1, 0)
        H.heom_state_broadcast(eq, s64)
        y1 = torch.empty((1, nado, d, d), dtype=torch.complex128, device=dev)
        H.heom_kick_dev(h64e, H.heom_state_device_ptr(s64), y1.data_ptr(), 1, 0, 1, sp)
        a1, b1 = torch.empty_like(y1), torch.empty_like(y1)
        n3 = grid["n3"]
        nt = max(n3, args.warmup + args.steps)
        ref = torch.zeros(nt, dtype=torch.complex128, device=dev)
        for i in range(nt):
            H.heom_propagate_dev(h64e, y1.data_ptr(), a1.data_ptr(), b1.data_ptr(), 1, 0,
                                 grid["dt_fs"], m, sp)
            H.heom_trace_dev(h64e, y1.data_ptr(), 1, 0, 3, ref[i:i + 1].data_ptr(), sp)
        # one branch in the benched precision from the same kicked state
        sM = H.heom_state_create(h, 1, prec)
        H.heom_state_broadcast(eq, sM)
        yM = torch.empty((1, nado, d, d), dtype=cdt, device=dev)
        H.heom_kick_dev(h, H.heom_state_device_ptr(sM), yM.data_ptr(), 1, prec, 1, sp)
        aM, bM = torch.empty_like(yM), torch.empty_like(yM)
        trM = torch.zeros(n3, dtype=torch.complex128, device=dev)
        for i in range(n3):
            H.heom_propagate_dev(h, yM.data_ptr(), aM.data_ptr(), bM.data_ptr(), 1, prec,
                                 grid["dt_fs"], m, sp)
            H.heom_trace_dev(h, yM.data_ptr(), 1, prec, 3, trM[i:i + 1].data_ptr(), sp)
        torch.cuda.synchronize()
        nw = args.warmup + args.steps
        timed = (traces - ref[:nw, None]).abs().max().item() / ref[:nw].abs().max().item()
        full = (trM - ref[:n3]).abs().max().item() / ref[:n3].abs().max().item()
        error = {"timed_traces": {"max_abs_over_max_ref": timed, "rk4_steps": nw * m,
                                  "branches_compared": B},
                 "full_t3_length": {"max_abs_over_max_ref": full, "rk4_steps": n3 * m, "branches": 1},
                 "vs": "FP64 GPU path (same kicked initial state, same RK4 steps)"}
        del y1, a1, b1, s64, h64e, yM, aM, bM, sM

    # ---------------- plain FP64 GPU path on the same model (mixed vs FP64) ----------------
    fp64 = None
    if prec != 0 and not args.no_fp64:
        h64 = H.heom_build_hierarchy(model, 0)
        Bf = min(B, 16)
        s64 = H.heom_state_create(h64, Bf, 0)
        H.heom_state_broadcast(eq, s64)
        y64 = torch.empty((Bf, nado, d, d), dtype=torch.complex128, device=dev)
        H.heom_kick_dev(h64, H.heom_state_device_ptr(s64), y64.data_ptr(), Bf, 0, 1, sp)
        del s64
        a64, b64 = torch.empty_like(y64), torch.empty_like(y64)
        H.heom_propagate_dev(h64, y64.data_ptr(), a64.data_ptr(), b64.data_ptr(), Bf, 0, grid["dt_fs"], 1, sp)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        H.heom_propagate_dev(h64, y64.data_ptr(), a64.data_ptr(), b64.data_ptr(), Bf, 0, grid["dt_fs"], 2, sp)
        e1.record(stream)
        torch.cuda.synchronize()
        v64 = Bf * nado * 2 / (e0.elapsed_time(e1) / 1000.0)
        fp64 = {"value": v64, "unit": "ADO-updates/s", "branches": Bf, "steps": 2,
                "mixed_over_fp64": value / v64}
        del y64, a64, b64, h64

    # ---------------- e2e through the public C ABI with host buffers ----------------
    e2e = None
    if not args.no_e2e:
        eq_host = H.heom_state_download(eq)
        pinned = torch.from_numpy(eq_host.view(np.float64)).pin_memory()
        eq_up = H.heom_state_create(h, 1, 0)
        rows = min(args.e2e_rows or e2e_rows, grid["n1"])
        # warm-up call of the timed size (the first call of a batch size tunes the
        # coupling kernel's launch shape once; repeated calls reuse it)
        H.heom_response_2d_rows(h, eq, grid, 0, rows)
        tt = []
        d2h = 0
        for i in range(args.e2e_steps):
            j0 = (i * rows) % grid["n1"]
            j1 = min(grid["n1"], j0 + rows)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            H.lib().heom_state_upload(eq_up.h, H.ct.cast(pinned.data_ptr(), H._D))
            RI, RII = H.heom_response_2d_rows(h, eq_up, grid, j0, j1)
            tt.append((time.perf_counter() - t0, rows_ado_updates(grid, nado, j0, j1)))
            d2h = RI.nbytes + RII.nbytes
        e2e = {"value": sum(u for _, u in tt) / sum(s for s, _ in tt), "unit": "ADO-updates/s",
               "h2d_bytes_per_step": int(pinned.numel() * 8), "d2h_bytes_per_step": int(d2h),
               "call": "heom_state_upload + heom_response_2d_rows (%d t1 rows, both pathways, all "
                       "t3 and t2, trunk recomputed)" % rows,
               "seconds_per_step": sum(s for s, _ in tt) / len(tt)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(cfg, budget_s=15.0, max_steps=30)
        cpu.pop("seconds", None)

    if rank == 0:
        conf = describe(cfg, model, grid, d, nado)
        conf["branches"] = B
        conf.update({"parallelism": "replicas" if world > 1 else "single-gpu",
                     "l2": "inputs larger than L2 (state %.1f GB)" % (y.numel() * y.element_size() / 1e9),
                     "precision": PREC_NAME[prec]})
        line = {
            "metric": "HEOM ADO-updates/s (2D spectra/hour derived)",
            "value": value, "unit": "ADO-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": PREC_NAME[prec],
            "data": "synthetic (seeded water-like MAB model; no dataset)",
            "config": conf,
            # one spectrum = its ADO-updates at the measured rate plus one equilibration
            "spectra_per_hour": 3600.0 / (per_spec / value + eq_seconds),
            "spectra_per_hour_excl_equilibration": 3600.0 * value / per_spec,
            "equilibration_s": eq_seconds,
            "ado_updates_per_spectrum": per_spec,
            "error": error,
            "roofline": roof, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
            "fp64_gpu": fp64,
            "gpu_launches": int(launches),
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
