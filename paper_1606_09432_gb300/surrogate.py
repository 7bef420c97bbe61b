"""Learned surrogate of the lattice Boltzmann step: training data from LB
trajectories, training, and the jump / validate / fall-back controller.

This module orchestrates C-ABI calls (include/lbpf.h); every arithmetic step
runs in the library's CUDA kernels.  PyTorch provides device buffers only.

Controller, per block of M jumps of K steps on one 2D domain:
  1. checkpoint phi, u;
  2. M network jumps: (phi, u) += net(phi, u, cos 4 theta, sin 4 theta, eps),
     the populations restarted at equilibrium from the new fields; a jump that
     leaves phi outside [-1 - 1e-2, 1 + 1e-2] rejects the block;
  3. validation: k_v plain LB steps from the jumped state; the tip velocity of
     the jumps is compared with the LB tip velocity over those steps (LB is
     the reference); a relative deviation above v_tol rejects the block;
  4. a rejected block is restored from the checkpoint and redone with plain LB.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import lbpf as L
from . import workloads as W


def _domain(d):
    prm = dict(d["params"])
    lam = prm.pop("lam")
    n = d["shape"][1]
    return L.make_domain(n, n, 1, lam=lam, crystals=[L.make_crystal(**c) for c in d["crystals"]], **prm)


def crystal_table(d, torch):
    tab = np.array([[c["eps"], c["phi0"]] for c in d["crystals"]], dtype=np.float32)
    return torch.from_numpy(tab).cuda()


def read_state(solver, k, torch, index=True):
    shape = solver.shape(k)
    phi = torch.empty(shape, dtype=torch.float32, device="cuda")
    u = torch.empty(shape, dtype=torch.float32, device="cuda")
    L.lbpf_read_field(solver.ctx, k, L.LBPF_FIELD_PHI, phi)
    L.lbpf_read_field(solver.ctx, k, L.LBPF_FIELD_U, u)
    I = None
    if index:
        I = torch.empty(shape, dtype=torch.int32, device="cuda")
        L.lbpf_read_field(solver.ctx, k, L.LBPF_FIELD_INDEX, I)
    return phi, u, I


def generate_pairs(draws, total_steps, K, torch, stream=None):
    """Run all draws in one batched LB context; every K steps build the network
    input and, K steps later, the target increment.  Returns X (M, H, W, 5) and
    Y (M, H, W, 2) as CUDA tensors."""
    s = L.Solver([_domain(d) for d in draws], L.LBPF_D2Q9_D2Q5, L.LBPF_GRAD_DD, L.LBPF_FP32, stream=stream)
    for k, d in enumerate(draws):
        s.seed(d["seeds"], domain=k)
    n = draws[0]["shape"][1]
    tabs = [crystal_table(d, torch) for d in draws]
    prev = [None] * len(draws)
    X, Y = [], []
    for t in range(0, total_steps + 1, K):
        for k, d in enumerate(draws):
            phi, u, I = read_state(s, k, torch)
            if prev[k] is not None:
                y = torch.empty((n, n, 2), dtype=torch.float32, device="cuda")
                L.net_delta(prev[k][0], prev[k][1], phi, u, y, stream)
                Y.append(y)
            if t < total_steps:
                x = torch.empty((n, n, 5), dtype=torch.float32, device="cuda")
                L.net_assemble(phi, u, I, tabs[k], x, stream)
                X.append(x)
            prev[k] = (phi, u)
        if t < total_steps:
            s.step(K)
    s.close()
    return torch.stack(X), torch.stack(Y)


def train(net, X, Y, steps, lr=2e-3, seed=0, torch=None, log_every=0):
    """Adam on random minibatches of net.batch pairs; returns the loss history."""
    rng = np.random.default_rng(seed)
    hist = []
    B = net.batch
    for it in range(steps):
        idx = torch.from_numpy(rng.choice(X.shape[0], B, replace=False)).cuda()
        xb = X.index_select(0, idx).contiguous()
        yb = Y.index_select(0, idx).contiguous()
        hist.append(net.train_step(xb, yb, lr))
        if log_every and it % log_every == 0:
            print(f"step {it}: loss {hist[-1]:.3e}")
    return hist


@dataclass
class Stats:
    steps: int = 0
    jumps_accepted: int = 0
    blocks_rejected: int = 0
    rejected_range: int = 0
    rejected_velocity: int = 0
    v_dev: list = field(default_factory=list)
    lb_steps: int = 0
    seconds: float = 0.0
    tip_history: list = field(default_factory=list)


class Controller:
    """Advances one 2D domain (a single-domain Solver) with network jumps under
    LB validation and fall-back (see the module docstring)."""

    def __init__(self, solver, net, draw, centre, torch, K=50, M=4, kv=20, v_tol=0.05, margin=1e-2, stream=None):
        self.s, self.net, self.torch = solver, net, torch
        self.K, self.M, self.kv, self.v_tol, self.margin = K, M, kv, v_tol, margin
        self.centre, self.stream = centre, stream
        self.tab = crystal_table(draw, torch)
        self.dt = draw["params"]["dt"]
        n = draw["shape"][1]
        self.x = torch.empty((1, n, n, 5), dtype=torch.float32, device="cuda")
        self.y = torch.empty((1, n, n, 2), dtype=torch.float32, device="cuda")
        self.cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.stats = Stats()

    def _tip(self):
        tip = self.s.measure(*self.centre)[0][:4]
        return float(np.max(tip))

    def _write(self, phi, u, I):
        L.lbpf_write_fields(self.s.ctx, 0, phi, u, I)

    def block(self):
        st = self.stats
        phi0, u0, I0 = read_state(self.s, 0, self.torch)
        ck = (phi0.clone(), u0.clone(), I0.clone())
        tip_start = self._tip()
        phi, u, I = phi0, u0, I0
        ok = True
        for _ in range(self.M):
            L.net_assemble(phi, u, I, self.tab, self.x, self.stream)
            self.net.forward(self.x, self.y)
            L.net_apply(self.y, phi, u, self.stream)
            L.net_range_check(phi, -1.0 - self.margin, 1.0 + self.margin, self.cnt, self.stream)
            self._write(phi, u, I)
            if int(self.cnt.item()) > 0:
                ok = False
                st.rejected_range += 1
                break
        if ok:
            tip_jump = self._tip()
            v_sur = (tip_jump - tip_start) / (self.M * self.K)
            self.s.step(self.kv)
            v_lb = (self._tip() - tip_jump) / self.kv
            st.v_dev.append((v_sur - v_lb) / v_lb if v_lb != 0 else float("inf"))
            if not (v_lb > 0 and abs(v_sur - v_lb) <= self.v_tol * abs(v_lb)):
                ok = False
                st.rejected_velocity += 1
        if ok:
            st.jumps_accepted += self.M
            st.lb_steps += self.kv
        else:
            st.blocks_rejected += 1
            self._write(*ck)
            self.s.step(self.M * self.K + self.kv)
            st.lb_steps += self.M * self.K + self.kv
        st.steps += self.M * self.K + self.kv
        st.tip_history.append((st.steps, self._tip()))

    def run(self, total_steps):
        t0 = time.perf_counter()
        while self.stats.steps + self.M * self.K + self.kv <= total_steps:
            self.block()
        rest = total_steps - self.stats.steps
        if rest > 0:
            self.s.step(rest)
            self.stats.lb_steps += rest
            self.stats.steps += rest
        self.torch.cuda.synchronize()
        self.stats.seconds = time.perf_counter() - t0
        return self.stats
