"""The 3D precision form on its 64^3 crop: the <110>/<111> anisotropy of Eq.
(As_MatSci) with (eps_1, eps_2) = (eps_s, gamma) over {-0.02, 0, 0.02}^2,
Delta = 0.4, centred seed of radius 8, 120 steps, against the FP64 oracle.
At this undercooling the crystal grows fast and the growth amplifies
rounding: by 500 steps the tips reach 28 of the 32 sites to the periodic
images, and FP32 then differs from FP64 by up to 7e-2 (1.1e-4 at 200
steps, at the point (0.02, -0.02)).

FP32 is gated (1e-4 on phi and u, tips within 0.5 lattice unit).  The 16-bit
deviation forms (FP16, BF16) change the rounding of the stored populations;
their errors are stated: max |phi|, |u| differences, and the relative errors
of the tip velocity (FP64 least-squares slope over the last 8 measurements,
every 12 steps) and of the tip radius (parabola fit of the crossings, J = 3)
along +x.  (At 200 steps BF16 moved one tip of the (0, -0.02) crystal by
3.2 sites: the growth instability picks up BF16-sized noise.)
"""
import itertools

import numpy as np
import pytest

from helpers import gpu_run, maxabs, oracle_run
from paper_1606_09432_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PAIRS = list(itertools.product([-0.02, 0.0, 0.02], repeat=2))
STEPS, EVERY = 120, 12


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


def measured_run(run, centre, dt, dx):
    """Step a run to STEPS, measuring every EVERY steps; returns tips along
    +x over time, the final tip6, the tip velocity along +x."""
    times, tips = [], []
    for k in range(STEPS // EVERY):
        run.step(EVERY)
        t = run.measure(*centre)[0]
        times.append((k + 1) * EVERY * dt)
        tips.append(t)
    return np.array(times), np.array(tips)


@pytest.mark.parametrize("eps,gamma", PAIRS)
def test_c3_sweep_point(L, O, eps, gamma):
    w = W.c3(64, eps=eps, gamma=gamma)
    cr = [w["aniso"]]
    dt, dx = w["params"]["dt"], w["params"]["dx"]
    o = oracle_run(O, 1, w["shape"], w["params"], cr, seeds=w["seeds"])
    ot, otips = measured_run(o, w["centre"], dt, dx)
    ophi, ou, _ = o.fields()
    ov = O.tip_velocity(ot[-8:], otips[-8:, 0] * dx)
    orad = O.tip_radius(ophi, w["centre"], 0, J=3)
    assert otips[-1, 0] > 8.5 and ov > 0 and orad > 1.0
    rows = []
    for prec, name in ((1, "FP32"), (2, "FP16 dev"), (3, "BF16 dev")):
        s = gpu_run(L, 1, w["shape"], w["params"], cr, seeds=w["seeds"], precision=prec)
        _, tips = measured_run(s, w["centre"], dt, dx)
        phi, u = s.fields()
        v = s.tip_velocity(window=8)[0]
        r = s.tip_radius(*w["centre"], 0, J=3)
        e = dict(phi=maxabs(phi, ophi), u=maxabs(u, ou), tip=float(np.abs(tips[-1] - otips[-1]).max()),
                 v=abs(v - ov) / abs(ov), rho=abs(r - orad) / abs(orad))
        rows.append((name, e))
        print(f"C3 sweep (eps1, eps2) = ({eps:+.2f}, {gamma:+.2f}) {name:9s}: phi {e['phi']:.2e}  u {e['u']:.2e}  "
              f"tips {e['tip']:.2e}  V_tip rel {e['v']:.2e}  rho rel {e['rho']:.2e}  "
              f"(oracle V_tip {ov:.4e}, rho {orad:.3f})")
        if prec == 1:
            assert e["phi"] <= 1e-4 and e["u"] <= 1e-4 and e["tip"] <= 0.5
        else:  # stated, with sanity bounds
            assert np.isfinite(phi).all() and e["phi"] < 1.0 and e["u"] < 0.5
        s.close()
