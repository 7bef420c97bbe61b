"""Scaled-down GPU runs of the paper's isotropy experiments (the full-size
runs are `bench.py --replicate`): the sixfold crystal of Sec. 4.2 on 400^2
for 2.5e4 steps is markedly more isotropic with directional derivatives than
with central differences, by both of the paper's measures; the slices of a
Sec. 5.2 dendrite related by a cube symmetry agree to FP32 rounding."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1606_09432_gb300 import build as B
    from paper_1606_09432_gb300 import lbpf
    B.build()
    lbpf.load()
    return lbpf


def test_sec42_dd_beats_fd(L):
    from paper_1606_09432_gb300 import replicate as R
    fd = R.sec42(L, L.LBPF_GRAD_FD, precision=L.LBPF_FP32, n=400, steps=25000)
    dd = R.sec42(L, L.LBPF_GRAD_DD, precision=L.LBPF_FP32, n=400, steps=25000)
    print("Sec. 4.2 at 400^2, 2.5e4 steps:", fd, dd)
    assert fd["tip_x"] > 40 and dd["tip_x"] > 40
    assert dd["err_l2"] < 0.5 * fd["err_l2"]
    assert max(dd["rot60_max"], -dd["rot60_min"]) < 0.5 * max(fd["rot60_max"], -fd["rot60_min"])


@pytest.mark.parametrize("which", ["A", "B", "C"])
def test_sec52_slices_match(L, which):
    from paper_1606_09432_gb300 import replicate as R
    r = R.sec52(L, which, n=95, steps=1500)
    print(f"Sec. 5.2 dendrite {which} at 95^3, 1500 steps:", r)
    assert r["slice_max_diff"] <= 1e-4 and r["solid_fraction"] > 0.0
