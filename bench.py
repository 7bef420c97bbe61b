"""Benchmark of the fused phi + u lattice Boltzmann step on GB300.

Default workload: the 3D precision form, 512^3 periodic, D3Q15 (phi) / D3Q7
(u), FP32 arithmetic with the populations stored as FP16 deviations from
w_i phi and w_i u, the <110> form of Eq. (As_MatSci) with eps = 0,
gamma = -0.02, Delta = 0.4, centred seed of radius 8 (Younsi & Cartalade's 3D
parameter set, Sec. 5.2).  A step is one time step of the whole domain; the
metric is MLUPS (million lattice-site updates per second) with the fraction
of the measured HBM copy bandwidth that the step kernel's algorithmic bytes
reach.  The timed steps go through lbpf_step in runs of 16, which the library
replays from CUDA graphs.

Under torchrun every rank advances its own independent domain (replicas of
the workload; weak scaling, no data-path collective).

--impl reference times the FP64 CPU oracle (the method written plainly from
the paper) on the host cores: each step is one oracle time step of a 64^3
periodic crop of the same workload (for the batched 2D workload: of its
first domain).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (description, lattice, precision, n)
    "c2-256-fp32": ("3D single crystal 256^3 periodic, D3Q15/D3Q7, FP32, <100> eps=0.05, Delta=0.3, seed R=8", 1, 1, 256),
    "c2-256-d3q19-fp32": ("3D single crystal 256^3 periodic, D3Q19/D3Q7, FP32, <100> eps=0.05, Delta=0.3, seed R=8",
                          2, 1, 256),
    "c2-256-d3q27-fp32": ("3D single crystal 256^3 periodic, D3Q27/D3Q7, FP32, <100> eps=0.05, Delta=0.3, seed R=8",
                          3, 1, 256),
    "c3-512-fp16dev": ("3D 512^3 periodic, D3Q15/D3Q7, FP32 arithmetic with FP16 deviation storage, "
                       "<110> form eps=0, gamma=-0.02, Delta=0.4, seed R=8", 1, 2, 512),
    "c3-512-bf16dev": ("3D 512^3 periodic, D3Q15/D3Q7, FP32 arithmetic with BF16 deviation storage, "
                       "<110> form eps=0, gamma=-0.02, Delta=0.4, seed R=8", 1, 3, 512),
    "c3-512-fp16dev-sr": ("3D 512^3 periodic, D3Q15/D3Q7, FP32 arithmetic with FP16 deviation storage rounded "
                          "stochastically, <110> form eps=0, gamma=-0.02, Delta=0.4, seed R=8", 1, 4, 512),
    "c3-512-fp32": ("3D 512^3 periodic, D3Q15/D3Q7, FP32, <110> form eps=0, gamma=-0.02, Delta=0.4, seed R=8", 1, 1, 512),
    "octant-351-fp32": ("3D octant of dendrite B (Sec. 5.3): 351^3, zero-flux walls on all faces, seed R=8 at the "
                        "origin, D3Q15/D3Q7, FP32, <110> form eps=0, gamma=-0.02, Delta=0.25", 1, 1, 351),
    "octant-351-fp16dev": ("3D octant of dendrite B (Sec. 5.3): 351^3, zero-flux walls on all faces, seed R=8 at the "
                           "origin, D3Q15/D3Q7, FP32 arithmetic with FP16 deviation storage, <110> form eps=0, "
                           "gamma=-0.02, Delta=0.25", 1, 2, 351),
    "c4-batch64-fp32": ("batched 2D multi-crystal: 64 periodic domains, sides U{128..1024} (24.4 M sites), D2Q9/D2Q5, "
                        "FP32, 1-12 seeds each with its own angle-form crystal (q=4, theta, eps), Delta per domain, "
                        "one launch per step, CUDA graphs", 0, 1, 0),
}
DTYPE = {0: "f64", 1: "f32", 2: "f32 arithmetic, f16 storage", 3: "f32 arithmetic, bf16 storage",
         4: "f32 arithmetic, f16 storage (stochastic rounding)"}
METRIC = "fused phi+u LB step MLUPS"
KERNEL_SOURCES = ["step_kernel.cuh", "staged_kernel.cuh", "lbpf_internal.cuh"]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def rank_max(x: float, dist=None, device="cuda") -> float:
    """The largest x over all ranks (x itself without a process group): the
    job's time is that of its slowest rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, sites: float, steps: int, seconds: float) -> float:
    """Whole-job MLUPS: every rank advances its own replica of `sites` sites
    by `steps` steps; `seconds` is the max over ranks."""
    return world * sites * steps / seconds / 1e6


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1606_09432_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """dram bytes per launch of the step kernel from the committed ncu summary,
    or None when there is none or the kernel changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"step_kernel_{workload}.md")
    if not os.path.exists(path):
        return None
    info = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            info[k.strip()] = v.strip().strip("`")
    if info.get("kernel_source_hash") != kernel_hash():
        return None
    try:
        return float(info["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def make_batch(L, W, stream, precision=1):
    doms, seeds = [], []
    for w in W.c4():
        prm = dict(w["params"])
        lam = prm.pop("lam")
        _, L_, _ = w["shape"][0], w["shape"][1], w["shape"][2]
        crs = [L.make_crystal(**c) for c in w["crystals"]]
        doms.append(L.make_domain(L_, L_, 1, lam=lam, crystals=crs, **prm))
        seeds.append(w["seeds"])
    s = L.Solver(doms, L.LBPF_D2Q9_D2Q5, L.LBPF_GRAD_DD, precision, stream=stream)
    for k, sd in enumerate(seeds):
        s.seed(sd, domain=k)
    c = seeds[0][0]
    return s, {"centre": (int(c[0]), int(c[1]), 0)}


def workload_recipe(W, workload, n):
    if workload.startswith("c2"):
        return W.c2(n)
    if workload.startswith("octant"):
        return W.octant(n)
    return W.c3(n, eps=0.0, gamma=-0.02)


def make_solver(L, W, workload, stream, size=0):
    if workload.startswith("c4"):
        return make_batch(L, W, stream)
    desc, lattice, precision, n = WORKLOADS[workload]
    n = size or n
    w = workload_recipe(W, workload, n)
    prm = dict(w["params"])
    lam = prm.pop("lam")
    dom = L.make_domain(n, n, n, lam=lam, crystals=[L.make_crystal(**w["aniso"])], bc=w.get("bc", 0), **prm)
    s = L.Solver(dom, lattice, L.LBPF_GRAD_DD, precision, stream=stream)
    s.seed(w["seeds"])
    return s, w


def oracle_threads() -> int:
    """Threads the OpenMP oracle runs with: OMP_NUM_THREADS when set, else
    every host core."""
    try:
        return max(1, int(os.environ["OMP_NUM_THREADS"]))
    except (KeyError, ValueError):
        return os.cpu_count() or 1


def oracle_sample(workload: str, n: int):
    """The oracle on a bounded sample of the workload: a periodic n^3 crop of
    a 3D workload (same parameters and centred seed), or the first domain of
    the batched 2D workload.  Returns (oracle, sites, description)."""
    from oracle import oracle as O
    from paper_1606_09432_gb300 import workloads as W
    O.build()
    desc, lattice, precision, _ = WORKLOADS[workload]
    if workload.startswith("c4"):
        w = W.c4()[0]
        prm = dict(w["params"])
        lam = prm.pop("lam")
        side = w["shape"][1]
        p = O.make_params(O.D2Q9_D2Q5, side, side, 1, lam=lam, crystals=[O.make_crystal(**c) for c in w["crystals"]],
                          **prm)
        o = O.Oracle(p).seed([list(s) for s in w["seeds"]])
        return o, side * side, f"first domain of the batch ({side}^2, {len(w['seeds'])} crystals)"
    w = workload_recipe(W, workload, n)
    prm = dict(w["params"])
    lam = prm.pop("lam")
    p = O.make_params(lattice, n, n, n, lam=lam, crystals=[O.make_crystal(**w["aniso"])], bc=w.get("bc", 0), **prm)
    o = O.Oracle(p).seed([list(s) for s in w["seeds"]])
    kind = "walled octant" if w.get("bc") else "periodic crop"
    return o, n ** 3, f"{n}^3 {kind} of the workload"


def cpu_oracle_rate(workload: str, budget_s: float, n: int = 64, max_steps: int | None = None):
    """Oracle MLUPS on a bounded sample of the workload (host cores)."""
    o, sites, what = oracle_sample(workload, n)
    o.step(1)  # warm
    steps, t0 = 0, time.perf_counter()
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and steps >= max_steps):
            break
    return sites * steps / el / 1e6, steps, el, what


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    desc = WORKLOADS[args.workload][0]
    o, sites, what = oracle_sample(args.workload, 64)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    v = sites * args.steps / el / 1e6
    cores = oracle_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "oracle_sample": f"{what}, one oracle step per bench step"},
        "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{what}, {args.steps} steps"},
        "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_surrogate(args, size=1024):
    K, M, kv, alpha = args.sur_k, args.sur_m, args.sur_kv, args.sur_alpha
    train_size, steps_total = args.sur_train_size, args.sur_steps
    n_draws, traj = args.sur_draws, args.sur_traj
    """Surrogate + LB vs plain LB on one 2D domain of the batched
    configuration's distributions: same final time, tip velocity from the
    last LB measurements, wall-clock time to solution."""
    import torch
    from paper_1606_09432_gb300 import build as B
    B.build()
    from paper_1606_09432_gb300 import lbpf as L
    from paper_1606_09432_gb300 import surrogate as S
    from paper_1606_09432_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    X, Y = S.generate_pairs(W.surrogate_draws(n_draws, size=train_size, seed=7), traj, K, torch)
    arch = dict(levels=args.sur_levels, base=args.sur_base)
    net = L.Net(train_size, train_size, batch=8, seed=1, **arch)
    net.set_loss_weight(alpha)
    hist = S.train(net, X, Y, args.sur_train, lr=1e-3, torch=torch)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    d = W.surrogate_draws(1, size=size, seed=99)[0]
    d["seeds"] = [(size / 2, size / 2, 0.0, 10.0, 0)]
    d["crystals"] = d["crystals"][:1]
    centre = (size // 2, size // 2, 0)
    inf = L.Net(size, size, batch=1, seed=0, **arch)
    inf.set_params(net.params())

    def solver():
        s = L.Solver([S._domain(d)], L.LBPF_D2Q9_D2Q5, L.LBPF_GRAD_DD, L.LBPF_FP32)
        s.seed(d["seeds"])
        return s

    def tipv(s, window=200):
        a = np.max(s.measure(*centre)[0][:4])
        s.step(window)
        b = np.max(s.measure(*centre)[0][:4])
        return (b - a) / window

    sp = solver()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    sp.step(steps_total)
    sp.measure(*centre)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t1
    sc = solver()
    ctl = S.Controller(sc, inf, d, centre, torch, K=K, M=M, kv=kv)
    st = ctl.run(steps_total)
    v_plain, v_sur = tipv(sp), tipv(sc)
    xx = torch.zeros((1, size, size, 5), device="cuda")
    yy = torch.empty((1, size, size, 2), device="cuda")
    inf.forward(xx, yy)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for _ in range(10):
        inf.forward(xx, yy)
    torch.cuda.synchronize()
    t_net = (time.perf_counter() - t2) / 10
    line = {"metric": "surrogate + LB vs plain LB time to solution", "value": round(t_plain / st.seconds, 4),
            "unit": "x (plain LB time / surrogate+LB time)", "higher_is_better": True, "n_gpus": 1,
            "config": {"workload": f"2D {size}^2 periodic, D2Q9/D2Q5 FP32, one seed R=10, {steps_total} steps, "
                                   f"K={K}, M={M}, k_v={kv}, network trained on {n_draws} draws at {train_size}^2 "
                                   f"({traj} LB steps each, pairs every K steps, {args.sur_train} Adam steps, "
                                   f"interface loss weight {alpha}), U-Net {args.sur_levels} levels, "
                                   f"base {args.sur_base} channels"},
            "plain_lb_s": round(t_plain, 4), "surrogate_lb_s": round(st.seconds, 4),
            "jumps_accepted": st.jumps_accepted, "blocks_rejected": st.blocks_rejected,
            "tip_velocity_rel_err": round(abs(v_sur - v_plain) / abs(v_plain), 4) if v_plain else None,
            "net_forward_ms": round(t_net * 1e3, 3), "train_s": round(t_train, 2),
            "train_loss_last": float(np.mean(hist[-50:])), "predict_zero_loss": float((Y ** 2).mean().item()),
            "rejected_range": st.rejected_range, "rejected_velocity": st.rejected_velocity,
            "v_dev_median": float(np.median(np.abs(st.v_dev))) if st.v_dev else None}
    print(json.dumps(line), flush=True)
    return 0


CONV_SHAPES = [(1, 1024, 1024, 32, 32), (1, 512, 512, 64, 64), (1, 256, 256, 128, 128), (1, 128, 128, 256, 256),
               (1, 128, 128, 384, 128), (8, 128, 128, 32, 32)]


def run_conv(args):
    """The surrogate's 3x3 convolution kernels alone (tensor cores): forward
    (bias + ReLU) and weight gradient for the 4-level network's layer shapes
    at 1024^2 and a training batch; one JSON line a shape with TFLOP/s and
    the fraction of the measured BF16 peak (a kernel timed alone: burst)."""
    import torch
    from paper_1606_09432_gb300 import build as B
    B.build()
    from paper_1606_09432_gb300 import lbpf as L
    L.load()
    peak = (peaks() or {}).get("bf16_tflops")
    torch.manual_seed(0)
    for n, H, W, cin, cout in CONV_SHAPES:
        x = torch.randn((n, H, W, cin), device="cuda")
        w = (torch.randn((9, cout, cin), device="cuda") / (3 * cin ** 0.5)).to(torch.bfloat16)
        b = torch.zeros(cout, device="cuda")
        y = torch.empty((n, H, W, cout), device="cuda")
        dy = torch.randn((n, H, W, cout), device="cuda")
        dw = torch.zeros((9, cout, cin), device="cuda")
        flops = 2.0 * n * H * W * 9 * cin * cout
        line = {"metric": "surrogate 3x3 convolution", "shape_nhwc_cin_cout": [n, H, W, cin, cout],
                "flop_per_call": flops, "unit": "TFLOP/s"}
        for name, fn in (("forward", lambda: L.nn_conv3x3(x, w, b, y, relu=True)),
                         ("weight_grad", lambda: L.nn_conv3x3_wgrad(x, dy, dw))):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps if args.steps > 0 else 10):
                fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / (args.steps if args.steps > 0 else 10)
            tf = flops / ms / 1e9
            line[name] = {"us": round(ms * 1e3, 1), "tflops": round(tf, 1),
                          "frac_of_bf16_peak": round(tf / peak, 4) if peak else None}
        line["error_word"] = L.nn_conv_error()
        line["peak_source"] = ("MEASURED_PEAKS.json bf16_tflops (burst, of measured)" if peak else
                               "no MEASURED_PEAKS.json")
        print(json.dumps(line), flush=True)
    return 0


def run_replicate(args):
    """Paper-scale runs of Secs. 4.2 and 5.2 (paper_1606_09432_gb300.replicate):
    one JSON line per run, with the paper's values as context."""
    import torch
    from paper_1606_09432_gb300 import build as B
    B.build()
    from paper_1606_09432_gb300 import lbpf as L
    from paper_1606_09432_gb300 import replicate as R
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    paper42 = {"FD": {"err_l2": 1.71e-1, "rot60_max": 1.446, "rot60_min": -1.454},
               "DD": {"err_l2": 3.04e-3, "rot60_max": 0.1, "rot60_min": -0.103}}
    if args.replicate in ("sec42", "all"):
        for grad in (L.LBPF_GRAD_FD, L.LBPF_GRAD_DD):
            t0 = time.perf_counter()
            r = R.sec42(L, grad, precision=L.LBPF_FP64, steps=args.rep_steps or 100000)
            r.update(seconds=round(time.perf_counter() - t0, 1), precision="f64", paper=paper42[r["grad"]],
                     experiment="Sec. 4.2 sixfold crystal 800^2, walls, q=6, eps=0.05, Delta=0.30")
            print(json.dumps(r), flush=True)
    if args.replicate in ("sec52", "all"):
        for which in "ABC":
            t0 = time.perf_counter()
            r = R.sec52(L, which, precision=L.LBPF_FP32)
            r.update(seconds=round(time.perf_counter() - t0, 1), precision="f32",
                     experiment="Sec. 5.2 dendrite 351^3, walls, Delta=0.30, seed R=8 at the centre",
                     paper="slices superimposed (Fig. 8)")
            print(json.dumps(r), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=512)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="c3-512-fp16dev", choices=sorted(WORKLOADS))
    ap.add_argument("--size", type=int, default=0, help="override the cube edge of the workload (profiling runs)")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sur-k", type=int, default=50, help="surrogate jump length K (LB steps)")
    ap.add_argument("--sur-m", type=int, default=4, help="surrogate jumps per validation")
    ap.add_argument("--sur-kv", type=int, default=20, help="LB validation steps after M jumps")
    ap.add_argument("--sur-alpha", type=float, default=0.0, help="interface weight of the training loss")
    ap.add_argument("--sur-draws", type=int, default=16, help="training draws")
    ap.add_argument("--sur-traj", type=int, default=2000, help="LB steps per training trajectory")
    ap.add_argument("--sur-train", type=int, default=1500, help="Adam steps")
    ap.add_argument("--sur-train-size", type=int, default=128, help="side of the training domains")
    ap.add_argument("--sur-steps", type=int, default=4400, help="LB steps to solution of the timed run")
    ap.add_argument("--sur-levels", type=int, default=3, help="U-Net levels")
    ap.add_argument("--sur-base", type=int, default=16, help="U-Net channels at the top level")
    ap.add_argument("--replicate", choices=["sec42", "sec52", "all"],
                    help="paper-scale isotropy runs of Secs. 4.2 / 5.2 instead of the benchmark")
    ap.add_argument("--rep-steps", type=int, default=0, help="steps of the Sec. 4.2 run (default 1e5)")
    ap.add_argument("--conv", action="store_true",
                    help="time the surrogate's tensor-core 3x3 convolution kernels alone")
    ap.add_argument("--surrogate", action="store_true",
                    help="time-to-solution of surrogate + LB vs plain LB (trains a network first)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.conv:
        return run_conv(args)
    if args.surrogate:
        return run_surrogate(args)
    if args.replicate:
        return run_replicate(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1606_09432_gb300 import build as B
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    from paper_1606_09432_gb300 import lbpf as L
    from paper_1606_09432_gb300 import workloads as W

    stream = torch.cuda.Stream()
    desc, lattice, precision, n = WORKLOADS[args.workload]
    if args.size:
        desc = desc.replace(f"{n}^3", f"{args.size}^3")
    with torch.cuda.stream(stream):
        s, w = make_solver(L, W, args.workload, stream.cuda_stream, args.size)
    sites = s.query(L.LBPF_Q_SITES)
    bps = s.query(L.LBPF_Q_BYTES_PER_SITE)

    # warm-up, then K timed steps through lbpf_step in runs of 16 (replayed
    # from CUDA graphs by the library), an event after every run
    G = 16
    s.step(args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    chunks = [G] * (args.steps // G) + ([args.steps % G] if args.steps % G else [])
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(chunks) + 1)]
    k0 = s.query(L.LBPF_Q_STEP_KERNELS)
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for k, c in enumerate(chunks):
            s.step(c)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
    launches = int(s.query(L.LBPF_Q_STEP_KERNELS) - k0)
    per = np.array([ev[k].elapsed_time(ev[k + 1]) / c for k, c in enumerate(chunks)])  # ms per step, per run
    total_ms = rank_max(float(ev[0].elapsed_time(ev[-1])), dist)
    value = job_rate(world, sites, args.steps, total_ms * 1e-3)
    tip, sf, cons = s.measure(*w["centre"])

    # end to end through the public API with host buffers: write the initial
    # fields from pinned host memory, advance K steps, read phi and u back
    # (every domain of the batched workload).
    ndom = len(s.domains)
    tdt = torch.float64 if precision == L.LBPF_FP64 else torch.float32
    bufs = []
    for k in range(ndom):
        shape = s.shape(k)
        bufs.append(torch.empty((2,) + shape, dtype=tdt).pin_memory())
        L.lbpf_read_fields(s.ctx, k, L.LBPF_READ_PHI | L.LBPF_READ_U, bufs[k])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(ndom):
        L.lbpf_write_fields(s.ctx, k, bufs[k][0], bufs[k][1])
    s.step(args.steps)
    for k in range(ndom):
        L.lbpf_read_fields(s.ctx, k, L.LBPF_READ_PHI | L.LBPF_READ_U, bufs[k])
    el = rank_max(time.perf_counter() - t0, dist)
    nb = sum(b.numel() * b.element_size() for b in bufs)
    e2e = {"value": round(job_rate(world, sites, args.steps, el), 2), "unit": "MLUPS",
           "h2d_bytes_per_step": round(nb / args.steps, 1), "d2h_bytes_per_step": round(nb / args.steps, 1),
           "note": f"lbpf_write_fields from pinned host + {args.steps} steps + lbpf_read_fields(phi|u) to pinned "
                   f"host, {ndom} domain(s)"}

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    avg_kernel_s = float(ev[0].elapsed_time(ev[-1])) * 1e-3 / args.steps  # this rank's mean step time
    achieved = bps * sites / avg_kernel_s / 1e9
    traffic = profiled_traffic(args.workload)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, st, el, what = cpu_oracle_rate(args.workload, args.cpu_budget, n=96)
        cpu = {"value": round(v, 3), "unit": "MLUPS", "cores": oracle_threads(), "kind": "oracle",
               "sample": f"{what}, {st} FP64 oracle steps in {el:.1f} s"}
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[precision], "data": "synthetic",
        "config": {"workload": desc, "sites_per_gpu": int(sites), "parallelism": f"replicas x{world}",
                   "l2": f"state {s.query(L.LBPF_Q_DEVICE_BYTES) / 1e9:.2f} GB per GPU, larger than L2 (no flush)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": "step_kernel", "bytes_per_site": bps,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if pk else "fallback 6.8 TB/s"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "check": {"tip_x": round(float(tip[0]), 4), "solid_fraction": sf, "conserved": cons},
        "step_ms": {"median": round(float(np.median(per)), 4), "min": round(float(per.min()), 4),
                    "max": round(float(per.max()), 4),
                    "note": "CUDA events around every run of 16 steps (graph replays), per step"},
        "schedule": {"tile_rows": s.query(L.LBPF_Q_TILE_ROWS), "segment": s.query(L.LBPF_Q_SEGMENT),
                     "blocks": s.query(L.LBPF_Q_BLOCKS)},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
