"""GPU tests of the batched / scheduled step: ragged multi-domain multi-crystal
parity with the oracle, bit-identical results across CUDA-graph replay and
across work schedules (tile height, z-segment length), and the 64-domain
batched 2D workload's invariants at full size."""
import numpy as np
import pytest

from helpers import gpu_run, maxabs, oracle_run
from paper_1606_09432_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1606_09432_gb300 import build as B
    from paper_1606_09432_gb300 import lbpf
    B.build()
    lbpf.load()
    return lbpf


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("xi", [0.1, 1e-7])
def test_batched_multicrystal_parity(L, O, xi):
    """Three ragged 2D domains, each with its own crystals and index field,
    advanced by one launch per step, against one oracle run per domain; the
    index threshold xi at 0.1 and at the paper's 1e-7 (Sec. 4.3)."""
    specs = [((1, 45, 70), [(15.0, 14.0, 0, 5.0, 0), (50.0, 30.0, 0, 6.0, 1)]),
             ((1, 64, 33), [(16.0, 20.0, 0, 4.0, 0), (16.0, 48.0, 0, 5.5, 1), (5.0, 5.0, 0, 4.0, 2)]),
             ((1, 40, 52), [(26.0, 20.0, 0, 6.0, 0)])]
    prm = dict(W.C4_PARAMS, delta=0.35)
    lam = prm.pop("lam")
    doms, oracles, crys = [], [], []
    for k, (shape, seeds) in enumerate(specs):
        cr = [dict(kind=1, eps=0.03 + 0.01 * j, q=4 + j, phi0=0.2 * j + 0.1 * k) for j in range(len(seeds))]
        crys.append(cr)
        doms.append(L.make_domain(shape[2], shape[1], 1, lam=lam, xi=xi, crystals=[L.make_crystal(**c) for c in cr],
                                  **prm))
        oracles.append(oracle_run(O, 0, shape, dict(prm, lam=lam), cr, seeds=seeds, xi=xi))
    s = L.Solver(doms, 0, 0, L.LBPF_FP64)
    for k, (_, seeds) in enumerate(specs):
        s.seed(seeds, domain=k)
    for rnd in range(2):
        s.step(100)
        for k, o in enumerate(oracles):
            o.step(100)
            ophi, ou, oI = o.fields()
            assert maxabs(s.field(0, domain=k), ophi) <= 1e-10, (rnd, k)
            assert maxabs(s.field(1, domain=k), ou) <= 1e-10, (rnd, k)
            assert np.array_equal(s.field(2, domain=k), oI), (rnd, k)


def test_graph_replay_matches_plain_launches(L):
    import torch
    w = W.c2(40)
    cr = [w["aniso"]]
    st = torch.cuda.Stream()
    a = gpu_run(L, 1, w["shape"], w["params"], cr, seeds=w["seeds"], precision=L.LBPF_FP32,
                stream=st.cuda_stream)
    b = gpu_run(L, 1, w["shape"], w["params"], cr, seeds=w["seeds"], precision=L.LBPF_FP32)
    a.step(70)  # 1 plain (load) step, 4 graph batches of 16, 5 plain
    b.step(70)
    torch.cuda.synchronize()
    assert np.array_equal(a.field(0), b.field(0)) and np.array_equal(a.field(1), b.field(1))
    assert a.query(L.LBPF_Q_STEP_KERNELS) == 70 and a.query(L.LBPF_Q_STEPS) == 70


@pytest.mark.parametrize("lattice,shape", [(1, (30, 41, 70)), (0, (1, 77, 100))])
def test_schedules_give_identical_results(L, lattice, shape):
    prm = dict(W.C3D_PARAMS, delta=0.3) if lattice == 1 else W.C1_PARAMS
    seeds = [(shape[2] / 2, shape[1] / 2, shape[0] / 2, 6.0, 0)]
    cr = [dict(kind=0, eps=0.05)]
    runs = []
    for rows, seg in ((8, 7), (16, 3), (8, 1000), (16, 16)):
        s = gpu_run(L, lattice, shape, prm, cr, seeds=seeds, precision=L.LBPF_FP32)
        L.lbpf_set_schedule(s.ctx, rows, seg)
        assert s.query(L.LBPF_Q_TILE_ROWS) == rows
        s.step(40)
        runs.append(s.fields())
    for r in runs[1:]:
        assert np.array_equal(r[0], runs[0][0]) and np.array_equal(r[1], runs[0][1])
    with pytest.raises(L.LbpfError):
        L.lbpf_set_schedule(s.ctx, 12, 8)


@pytest.mark.parametrize("lattice,shape", [(1, (36, 40, 44)), (0, (1, 90, 130))])
def test_autotune_at_first_step_leaves_state(L, tmp_path, monkeypatch, lattice, shape):
    """The schedule trials run at the first step on the live state: the run
    is bit-identical to one with the rule schedule and no trials, and the
    choice is cached for the next context of the same configuration."""
    prm = dict(W.C3D_PARAMS, delta=0.3) if lattice == 1 else W.C1_PARAMS
    seeds = [(shape[2] / 2, shape[1] / 2, shape[0] / 2, 6.0, 0)]
    cr = [dict(kind=0, eps=0.05)]
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("LBPF_TUNE_CACHE", str(cache))
    runs = []
    for tune in ("1", "0"):
        monkeypatch.setenv("LBPF_AUTOTUNE", tune)
        s = gpu_run(L, lattice, shape, prm, cr, seeds=seeds, precision=L.LBPF_FP32)
        s.step(25)
        runs.append(s.fields())
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert cache.exists() and len(cache.read_text().split()) == 3


def test_batch64_workload_invariants(L):
    """The 64-domain batched 2D configuration at full size (24.4 M sites), FP32:
    per-domain conservation of sum(u - phi/2) and growth, after 300 steps."""
    import torch
    st = torch.cuda.Stream()
    doms, seeds = [], []
    for w in W.c4():
        prm = dict(w["params"])
        lam = prm.pop("lam")
        n = w["shape"][1]
        doms.append(L.make_domain(n, n, 1, lam=lam, crystals=[L.make_crystal(**c) for c in w["crystals"]], **prm))
        seeds.append(w["seeds"])
    s = L.Solver(doms, 0, 0, L.LBPF_FP32, stream=st.cuda_stream)
    for k, sd in enumerate(seeds):
        s.seed(sd, domain=k)
    before = [s.measure(int(sd[0][0]) % doms[k].nx, int(sd[0][1]) % doms[k].ny, 0, domain=k) for k, sd in enumerate(seeds)]
    s.step(300)
    torch.cuda.synchronize()
    for k, sd in enumerate(seeds):
        tip, sf, cs = s.measure(int(sd[0][0]) % doms[k].nx, int(sd[0][1]) % doms[k].ny, 0, domain=k)
        # FP32 rounding: drift of the sum bounded per site and step (the sum
        # itself can nearly cancel when u - phi/2 ~ 0, so no relative bound)
        nk = doms[k].nx * doms[k].ny
        assert abs(cs - before[k][2]) <= 1e-8 * nk * 300, k
        assert sf > before[k][1], k  # undercooled crystals grow
