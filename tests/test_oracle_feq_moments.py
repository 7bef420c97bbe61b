"""Pin of the phase-field equilibrium of the oracle through its moments.

Sec. 3.2 fixes the moments of the equilibrium distribution of Eq. (Feq_Phase):
  sum_i g_i^(0)               = phi,
  sum_i g_i^(0) e_i           = -(dt/dx)(W0^2/tau0) N,
  sum_i g_i^(0) e_i e_i       = e^2 phi I,
with N the vector of Eq. (TermesAnisotropes).  The populations the oracle
starts from after set_fields are g^(0)(phi, N), so on a curved interface
(where N != 0) their first moment pins the scale and the sign with which N
enters Eq. (Feq_Phase): a factor 1/2, a dropped 1/e^2 or a flipped sign each
break it.  N itself is taken from the oracle's gradient and anisotropy
routines (pinned separately against numerical derivatives of a_s).
"""
import numpy as np
import pytest

FORMS_3D = {
    "cubic": dict(kind=0, eps=0.05),
    "y66": dict(kind=2, eps=0.05),
    "hoyt110": dict(kind=3, eps=0.02, gamma=-0.02),
    "s111": dict(kind=4, gamma=0.02),
}
# in 2D the <111> form is isotropic (S = nx^2 ny^2 nz^2 = 0), so N = 0 there
FORMS_2D = {k: v for k, v in FORMS_3D.items() if k != "s111"}
FORMS_2D["angle"] = dict(kind=1, eps=0.05, q=4, phi0=0.3)

# physical parameter sets of the paper: the 2D validation set (Sec. 3.4) and
# the 3D set of Sec. 5.2
P2 = dict(dx=0.4, dt=0.008, W0=1.0, tau0=1.0, kappa=2.0)
P3 = dict(dx=0.01, dt=1.5e-5, W0=0.0125, tau0=1.5625e-4, kappa=1.0)


def curved_field(shape, dx, W0):
    """Off-centre tanh sphere (circle in 2D) of radius 6 sites: every
    interface normal direction occurs, so N is non-zero on most of the rim."""
    nz, ny, nx = shape
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(float)
    cz = (nz - 1) / 2 + 0.37 if nz > 1 else 0.0
    r = np.sqrt((x - nx / 2 + 0.21) ** 2 + (y - ny / 2 - 0.43) ** 2 + (z - cz) ** 2)
    return np.tanh((6.0 - r) * dx / (np.sqrt(2.0) * W0))


CASES = [(0, f) for f in FORMS_2D] + [(lat, f) for lat in (1, 2, 3) for f in FORMS_3D]


@pytest.mark.parametrize("lattice,form", CASES)
def test_equilibrium_moments(orc, lattice, form):
    O = orc
    D, e, w, e2 = O.lattice(lattice, 0)
    shape = (1, 20, 22) if D == 2 else (16, 17, 18)
    prm = P2 if D == 2 else P3
    crystal = (FORMS_2D if D == 2 else FORMS_3D)[form]
    p = O.make_params(lattice, shape[2], shape[1], shape[0], crystals=[O.make_crystal(**crystal)], **prm)
    phi = curved_field(shape, prm["dx"], prm["W0"])
    u = np.full(shape, -0.3)
    o = O.Oracle(p).set_fields(phi, u)
    g, _ = o.populations()  # (Q, nz, ny, nx)

    # N at every site from the oracle's gradient and anisotropy routines
    G = O.gradient(p, phi)
    cr = O.make_crystal(**crystal)
    N = np.zeros(shape + (3,))
    for idx in np.ndindex(*shape):
        N[idx] = O.anisotropy(cr, D, G[idx], prm["dx"])[1]
    coef = (prm["dt"] / prm["dx"]) * (prm["W0"] ** 2 / prm["tau0"])
    nmax = np.abs(coef * N).max()
    assert nmax > 1e-4, "the test field must have a non-zero N"

    m0 = g.sum(axis=0)
    m1 = np.einsum("qa,qzyx->zyxa", e.astype(float), g)
    m2 = np.einsum("qa,qb,qzyx->zyxab", e.astype(float), e.astype(float), g)
    assert np.abs(m0 - phi).max() <= 1e-13
    assert np.abs(m1 - (-coef * N)).max() <= 1e-13 * max(1.0, nmax)
    want2 = e2 * phi[..., None, None] * np.eye(3)
    if D == 2:
        want2[..., 2, 2] = 0.0
    assert np.abs(m2 - want2).max() <= 1e-13


def test_moments_fix_the_n_term_scale(orc):
    """The first moment alone decides between the printed e.d.f. and its
    plausible misreadings: on the same populations, N scaled by 1/2, by e^2
    (no 1/e^2) or with the opposite sign would each miss by far more than
    rounding."""
    O = orc
    lattice = 1
    D, e, w, e2 = O.lattice(lattice, 0)
    shape = (16, 17, 18)
    crystal = FORMS_3D["hoyt110"]
    p = O.make_params(lattice, 18, 17, 16, crystals=[O.make_crystal(**crystal)], **P3)
    phi = curved_field(shape, P3["dx"], P3["W0"])
    g, _ = O.Oracle(p).set_fields(phi, np.zeros(shape)).populations()
    G = O.gradient(p, phi)
    cr = O.make_crystal(**crystal)
    N = np.stack([O.anisotropy(cr, D, G[idx], P3["dx"])[1] for idx in np.ndindex(*shape)]).reshape(shape + (3,))
    coef = (P3["dt"] / P3["dx"]) * (P3["W0"] ** 2 / P3["tau0"])
    m1 = np.einsum("qa,qzyx->zyxa", e.astype(float), g)
    err = np.abs(m1 + coef * N).max()
    for wrong in (0.5 * coef, e2 * coef, -coef):
        assert np.abs(m1 + wrong * N).max() > 1e6 * max(err, 1e-18)
