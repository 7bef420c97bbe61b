"""Thin Python binding of the lbpf C ABI (include/lbpf.h).

Argument marshalling only: every step of the solver runs in the CUDA library
liblbpf.so.  Device buffers may be passed as torch CUDA tensors, host buffers
as numpy arrays.  There is no CPU fallback: if the library is missing, loading
fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LBPF_LIB") or os.path.join(_HERE, "liblbpf.so")

# enums (include/lbpf.h)
LBPF_OK, LBPF_EINVAL, LBPF_ENOMEM, LBPF_ECUDA, LBPF_ETIMEOUT, LBPF_ENONFINITE, LBPF_ERANGE = 0, -1, -2, -3, -4, -5, -6
LBPF_D2Q9_D2Q5, LBPF_D3Q15_D3Q7, LBPF_D3Q19_D3Q7, LBPF_D3Q27_D3Q7 = 0, 1, 2, 3
LBPF_GRAD_DD, LBPF_GRAD_FD = 0, 1
LBPF_FP64, LBPF_FP32, LBPF_FP32_FP16DEV, LBPF_FP32_BF16DEV, LBPF_FP32_FP16DEV_SR = range(5)
LBPF_AS_CUBIC100, LBPF_AS_ANGLE, LBPF_AS_Y66, LBPF_AS_HOYT110, LBPF_AS_S111 = 0, 1, 2, 3, 4
LBPF_FIELD_PHI, LBPF_FIELD_U, LBPF_FIELD_INDEX, LBPF_FIELD_AS = 0, 1, 2, 3
LBPF_READ_PHI, LBPF_READ_U, LBPF_READ_AS, LBPF_READ_INDEX = 1, 2, 4, 8
(LBPF_Q_SITES, LBPF_Q_STEPS, LBPF_Q_BYTES_PER_SITE, LBPF_Q_DEVICE_BYTES, LBPF_Q_LAMBDA, LBPF_Q_STEP_KERNELS,
 LBPF_Q_TILE_ROWS, LBPF_Q_SEGMENT, LBPF_Q_BLOCKS, LBPF_Q_KERNEL) = range(10)
LBPF_MAX_CRYSTALS = 16
LBPF_BC_WALL_X, LBPF_BC_WALL_Y, LBPF_BC_WALL_Z = 1, 2, 4
EXPORTED = ["lbpf_create", "lbpf_seed", "lbpf_write_fields", "lbpf_step", "lbpf_read_fields", "lbpf_read_field",
            "lbpf_read_populations", "lbpf_measure", "lbpf_query", "lbpf_destroy", "lbpf_last_error",
            "lbpf_field_sums_static", "lbpf_set_schedule", "lbpf_tip_velocity", "lbpf_tip_radius",
            "lbpf_net_create", "lbpf_net_create_arch", "lbpf_net_destroy", "lbpf_net_last_error", "lbpf_net_num_params",
            "lbpf_net_get_params", "lbpf_net_set_params", "lbpf_net_forward", "lbpf_net_backward",
            "lbpf_net_train_step", "lbpf_net_assemble", "lbpf_net_apply", "lbpf_net_delta",
            "lbpf_net_range_check", "lbpf_net_set_loss_weight", "lbpf_nn_conv3x3", "lbpf_nn_conv3x3_wgrad",
            "lbpf_nn_conv_error"]


class lbpf_crystal(C.Structure):
    _fields_ = [("kind", C.c_int), ("eps", C.c_double), ("gamma", C.c_double), ("q", C.c_int), ("phi0", C.c_double)]


class lbpf_domain(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("bc", C.c_int),
                ("dx", C.c_double), ("dt", C.c_double), ("W0", C.c_double), ("tau0", C.c_double),
                ("kappa", C.c_double), ("lam", C.c_double), ("delta", C.c_double), ("xi", C.c_double),
                ("n_crystals", C.c_int), ("crystals", lbpf_crystal * LBPF_MAX_CRYSTALS),
                ("adv", C.c_double * 3)]


class lbpf_seed_t(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z", C.c_double), ("radius", C.c_double), ("crystal", C.c_int)]


class LbpfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbpf error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load liblbpf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1606_09432_gb300.build.build()")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.lbpf_create.argtypes = [C.POINTER(lbpf_domain), C.c_int, C.c_int, C.c_int, C.c_int, vp, C.POINTER(vp)]
    lib.lbpf_seed.argtypes = [vp, C.c_int, C.POINTER(lbpf_seed_t), C.c_int]
    lib.lbpf_write_fields.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int]
    lib.lbpf_step.argtypes = [vp, C.c_int]
    lib.lbpf_read_fields.argtypes = [vp, C.c_int, C.c_uint, vp, C.c_int, C.c_size_t]
    lib.lbpf_read_field.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, C.c_size_t]
    lib.lbpf_read_populations.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, C.c_size_t]
    d = C.POINTER(C.c_double)
    lib.lbpf_measure.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, d, d, d]
    lib.lbpf_query.argtypes = [vp, C.c_int, d]
    lib.lbpf_destroy.argtypes = [vp]
    lib.lbpf_last_error.argtypes = [vp]
    lib.lbpf_last_error.restype = C.c_char_p
    lib.lbpf_field_sums_static.argtypes = [vp, vp, C.c_longlong, C.c_int, vp, vp]
    lib.lbpf_set_schedule.argtypes = [vp, C.c_int, C.c_int]
    lib.lbpf_tip_velocity.argtypes = [vp, C.c_int, C.c_int, d]
    lib.lbpf_tip_radius.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, d]
    lib.lbpf_net_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_ulonglong, vp, C.POINTER(vp)]
    lib.lbpf_net_create_arch.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_ulonglong, vp,
                                         C.POINTER(vp)]
    lib.lbpf_net_destroy.argtypes = [vp]
    lib.lbpf_net_last_error.argtypes = [vp]
    lib.lbpf_net_num_params.argtypes = [vp, C.POINTER(C.c_longlong)]
    lib.lbpf_net_get_params.argtypes = [vp, vp, C.c_int]
    lib.lbpf_net_set_params.argtypes = [vp, vp]
    lib.lbpf_net_forward.argtypes = [vp, vp, vp]
    lib.lbpf_net_backward.argtypes = [vp, vp]
    lib.lbpf_net_train_step.argtypes = [vp, vp, vp, C.c_float, d]
    lib.lbpf_net_set_loss_weight.argtypes = [vp, C.c_float]
    lib.lbpf_net_assemble.argtypes = [vp, vp, vp, vp, C.c_int, vp, C.c_longlong, vp]
    lib.lbpf_net_apply.argtypes = [vp, vp, vp, C.c_longlong, vp]
    lib.lbpf_net_delta.argtypes = [vp, vp, vp, vp, vp, C.c_longlong, vp]
    lib.lbpf_net_range_check.argtypes = [vp, C.c_longlong, C.c_float, C.c_float, vp, vp]
    lib.lbpf_nn_conv3x3.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp]
    lib.lbpf_nn_conv3x3_wgrad.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp]
    lib.lbpf_nn_conv_error.argtypes = [C.POINTER(C.c_int)]
    for name in EXPORTED:
        lib[name].restype = C.c_int
    lib.lbpf_last_error.restype = C.c_char_p
    lib.lbpf_net_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def lbpf_last_error(ctx=None) -> str:
    return load().lbpf_last_error(ctx).decode()


def _check(rc, ctx=None):
    if rc != LBPF_OK:
        raise LbpfError(rc, lbpf_last_error(ctx))


def make_crystal(kind=LBPF_AS_CUBIC100, eps=0.0, gamma=0.0, q=4, phi0=0.0) -> lbpf_crystal:
    return lbpf_crystal(kind, eps, gamma, q, phi0)


def make_domain(nx, ny, nz=1, *, dx, dt, W0, tau0, kappa, lam=0.0, delta=0.0, xi=1e-7, crystals=None,
                bc=0, adv=(0.0, 0.0, 0.0)) -> lbpf_domain:
    """lam <= 0 selects lambda* (the library applies Eq. (Kinetic-Coeff) with
    beta = 0); bc: LBPF_BC_WALL_* bits (0: periodic); adv: uniform velocity
    of the advective heat equilibrium (physical units)."""
    d = lbpf_domain()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.bc = bc
    d.dx, d.dt, d.W0, d.tau0, d.kappa = dx, dt, W0, tau0, kappa
    d.lam = 0.0 if lam is None else lam
    d.delta, d.xi = delta, xi
    d.adv[0], d.adv[1], d.adv[2] = (float(v) for v in adv)
    cl = list(crystals) if crystals else [make_crystal()]
    d.n_crystals = len(cl)
    for k, c in enumerate(cl):
        d.crystals[k] = c
    return d


def _ptr(a):
    """(address, on_device) of a numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), int(a.is_cuda)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data), 0


def lbpf_create(domains, lattice, grad=LBPF_GRAD_DD, precision=LBPF_FP32, stream=None):
    doms = list(domains) if isinstance(domains, (list, tuple)) else [domains]
    arr = (lbpf_domain * len(doms))(*doms)
    ctx = C.c_void_p()
    s = C.c_void_p(stream) if stream else None
    _check(load().lbpf_create(arr, len(doms), lattice, grad, precision, s, C.byref(ctx)))
    return ctx


def lbpf_seed(ctx, domain, seeds):
    rows = [lbpf_seed_t(*(float(v) for v in s[:4]), int(s[4]) if len(s) > 4 else 0) for s in seeds]
    arr = (lbpf_seed_t * len(rows))(*rows)
    _check(load().lbpf_seed(ctx, domain, arr, len(rows)), ctx)


def lbpf_write_fields(ctx, domain, phi, u, index=None):
    pp, dev = _ptr(phi)
    up, dev2 = _ptr(u)
    ip = None
    if index is not None:
        ip, dev3 = _ptr(index)
        if dev3 != dev:
            raise ValueError("index must live where phi does")
    if dev != dev2:
        raise ValueError("phi and u must both be host or both device buffers")
    _check(load().lbpf_write_fields(ctx, domain, pp, up, ip, dev), ctx)


def lbpf_step(ctx, n_steps=1):
    _check(load().lbpf_step(ctx, int(n_steps)), ctx)


def lbpf_read_fields(ctx, domain, mask, out):
    """Fields selected by mask (LBPF_READ_* bits) into out, back to back in
    bit order (phi, u, a_s in the arithmetic type, then int32 index); out is a
    host array or device tensor of enough bytes."""
    p, dev = _ptr(out)
    nbytes = out.numel() * out.element_size() if hasattr(out, "numel") else out.nbytes
    _check(load().lbpf_read_fields(ctx, domain, mask, p, dev, nbytes), ctx)
    return out


def lbpf_read_field(ctx, domain, field, out):
    p, dev = _ptr(out)
    nbytes = out.numel() * out.element_size() if hasattr(out, "numel") else out.nbytes
    _check(load().lbpf_read_field(ctx, domain, field, p, dev, nbytes), ctx)
    return out


def lbpf_read_populations(ctx, domain, which, out):
    p, dev = _ptr(out)
    nbytes = out.numel() * out.element_size() if hasattr(out, "numel") else out.nbytes
    _check(load().lbpf_read_populations(ctx, domain, which, p, dev, nbytes), ctx)
    return out


def lbpf_measure(ctx, domain, cx, cy, cz=0):
    tip = (C.c_double * 6)()
    sf, cs = C.c_double(), C.c_double()
    _check(load().lbpf_measure(ctx, domain, cx, cy, cz, tip, C.byref(sf), C.byref(cs)), ctx)
    return np.array(tip[:]), sf.value, cs.value


def lbpf_tip_velocity(ctx, domain, window=10):
    v = (C.c_double * 6)()
    _check(load().lbpf_tip_velocity(ctx, domain, window, v), ctx)
    return np.array(v[:])


def lbpf_tip_radius(ctx, domain, cx, cy, cz, direction, J=3):
    r = C.c_double()
    _check(load().lbpf_tip_radius(ctx, domain, cx, cy, cz, direction, J, C.byref(r)), ctx)
    return r.value


def lbpf_set_schedule(ctx, tile_rows, segment):
    _check(load().lbpf_set_schedule(ctx, tile_rows, segment), ctx)


def lbpf_query(ctx, what):
    v = C.c_double()
    _check(load().lbpf_query(ctx, what, C.byref(v)), ctx)
    return v.value


def lbpf_field_sums_static(phi, u, precision, out, stream=None):
    """Measurement sums over device tensors phi, u into the device tensor out
    (3 float64), with no device allocation by the library; see include/lbpf.h."""
    pp, d1 = _ptr(phi)
    up, d2 = _ptr(u)
    op, d3 = _ptr(out)
    if not (d1 and d2 and d3):
        raise ValueError("phi, u and out must be device tensors")
    n = phi.numel()
    rc = load().lbpf_field_sums_static(pp, up, n, precision, op, C.c_void_p(stream) if stream else None)
    if rc != LBPF_OK:
        raise LbpfError(rc, "lbpf_field_sums_static failed")


def lbpf_destroy(ctx):
    if ctx:
        load().lbpf_destroy(ctx)


class Solver:
    """Convenience owner of one context (all domains share lattice, gradient
    and precision)."""

    Q = {LBPF_D2Q9_D2Q5: (9, 5), LBPF_D3Q15_D3Q7: (15, 7), LBPF_D3Q19_D3Q7: (19, 7), LBPF_D3Q27_D3Q7: (27, 7)}

    def __init__(self, domains, lattice, grad=LBPF_GRAD_DD, precision=LBPF_FP32, stream=None):
        self.domains = list(domains) if isinstance(domains, (list, tuple)) else [domains]
        self.precision = precision
        self.lattice = lattice
        self.ctx = lbpf_create(self.domains, lattice, grad, precision, stream)

    @property
    def dtype(self):
        return np.float64 if self.precision == LBPF_FP64 else np.float32

    def shape(self, domain=0):
        d = self.domains[domain]
        return (d.nz, d.ny, d.nx)

    def seed(self, seeds, domain=0):
        lbpf_seed(self.ctx, domain, seeds)
        return self

    def write_fields(self, phi, u, index=None, domain=0):
        if not hasattr(phi, "data_ptr"):
            phi = np.ascontiguousarray(phi, dtype=self.dtype)
            u = np.ascontiguousarray(u, dtype=self.dtype)
            if index is not None:
                index = np.ascontiguousarray(index, dtype=np.int32)
        lbpf_write_fields(self.ctx, domain, phi, u, index)
        return self

    def step(self, n=1):
        lbpf_step(self.ctx, n)
        return self

    def field(self, which, domain=0):
        dt = np.int32 if which == LBPF_FIELD_INDEX else self.dtype
        out = np.empty(self.shape(domain), dtype=dt)
        return lbpf_read_field(self.ctx, domain, which, out)

    def fields(self, domain=0):
        """(phi, u) read by one lbpf_read_fields call."""
        shp = self.shape(domain)
        out = np.empty((2,) + shp, dtype=self.dtype)
        lbpf_read_fields(self.ctx, domain, LBPF_READ_PHI | LBPF_READ_U, out)
        return out[0], out[1]

    def anisotropy_field(self, domain=0):
        """a_s of the current phi at every site (LBPF_FIELD_AS)."""
        return self.field(LBPF_FIELD_AS, domain)

    def populations(self, which, domain=0):
        out = np.empty((self.Q[self.lattice][which],) + self.shape(domain), dtype=self.dtype)
        return lbpf_read_populations(self.ctx, domain, which, out)

    def measure(self, cx, cy, cz=0, domain=0):
        return lbpf_measure(self.ctx, domain, cx, cy, cz)

    def query(self, what):
        return lbpf_query(self.ctx, what)

    def tip_velocity(self, window=10, domain=0):
        return lbpf_tip_velocity(self.ctx, domain, window)

    def tip_radius(self, cx, cy, cz, direction, J=3, domain=0):
        return lbpf_tip_radius(self.ctx, domain, cx, cy, cz, direction, J)

    def close(self):
        if self.ctx:
            lbpf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Learned surrogate network (include/lbpf.h, "Learned surrogate").
# ---------------------------------------------------------------------------

def _dptr(t):
    if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Net:
    """The surrogate U-Net for batches of `batch` H x W images (NHWC float32
    CUDA tensors: input (N, H, W, 5), output (N, H, W, 2)); `levels` levels
    with base * 2^l channels at level l."""

    def __init__(self, H, W, batch=1, seed=0, stream=None, levels=3, base=16):
        self.H, self.W, self.batch = H, W, batch
        self.levels, self.base = levels, base
        self.stream = stream
        self.h = C.c_void_p()
        rc = load().lbpf_net_create_arch(H, W, batch, levels, base, seed, C.c_void_p(stream) if stream else None,
                                         C.byref(self.h))
        if rc != LBPF_OK:
            raise LbpfError(rc, load().lbpf_net_last_error(None).decode())
        n = C.c_longlong()
        load().lbpf_net_num_params(self.h, C.byref(n))
        self.n_params = n.value

    def _chk(self, rc):
        if rc != LBPF_OK:
            raise LbpfError(rc, load().lbpf_net_last_error(self.h).decode())

    def params(self, which=0):
        out = np.empty(self.n_params, dtype=np.float32)
        self._chk(load().lbpf_net_get_params(self.h, C.c_void_p(out.ctypes.data), which))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._chk(load().lbpf_net_set_params(self.h, C.c_void_p(p.ctypes.data)))

    def forward(self, x, y=None):
        self._chk(load().lbpf_net_forward(self.h, _dptr(x), _dptr(y) if y is not None else None))
        return y

    def backward(self, dy):
        self._chk(load().lbpf_net_backward(self.h, _dptr(dy)))
        return self.params(which=1)

    def set_loss_weight(self, alpha):
        self._chk(load().lbpf_net_set_loss_weight(self.h, float(alpha)))

    def train_step(self, x, target, lr):
        loss = C.c_double()
        self._chk(load().lbpf_net_train_step(self.h, _dptr(x), _dptr(target), lr, C.byref(loss)))
        return loss.value

    def close(self):
        if self.h:
            load().lbpf_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def net_assemble(phi, u, index, crystal_tab, x, stream=None):
    """x (P, 5) from phi, u (P,), index (P,) int32 or None and the crystal table (nc, 2) = (eps, theta)."""
    tab = crystal_tab.reshape(-1)
    rc = load().lbpf_net_assemble(_dptr(phi), _dptr(u), _dptr(index) if index is not None else None, _dptr(tab),
                                  tab.numel() // 2, _dptr(x), phi.numel(), C.c_void_p(stream) if stream else None)
    if rc != LBPF_OK:
        raise LbpfError(rc, "lbpf_net_assemble failed")


def net_apply(y, phi, u, stream=None):
    rc = load().lbpf_net_apply(_dptr(y), _dptr(phi), _dptr(u), phi.numel(), C.c_void_p(stream) if stream else None)
    if rc != LBPF_OK:
        raise LbpfError(rc, "lbpf_net_apply failed")


def net_delta(phi0, u0, phi1, u1, y, stream=None):
    rc = load().lbpf_net_delta(_dptr(phi0), _dptr(u0), _dptr(phi1), _dptr(u1), _dptr(y), phi0.numel(),
                               C.c_void_p(stream) if stream else None)
    if rc != LBPF_OK:
        raise LbpfError(rc, "lbpf_net_delta failed")


def net_range_check(phi, lo, hi, count, stream=None):
    """count: a 1-element int32 CUDA tensor; returns nothing (read count after synchronising)."""
    rc = load().lbpf_net_range_check(_dptr(phi), phi.numel(), lo, hi, _dptr(count),
                                     C.c_void_p(stream) if stream else None)
    if rc != LBPF_OK:
        raise LbpfError(rc, "lbpf_net_range_check failed")


def nn_conv3x3(x, wt, bias, y, relu=False, stream=None):
    """One periodic 3x3 convolution on the tensor cores: x (n, H, W, cin) and
    y (n, H, W, cout) float32 CUDA tensors, wt a (9, cout, cin) bfloat16 (or
    int16 bit-pattern) CUDA tensor, bias a (cout,) float32 CUDA tensor or None."""
    n, H, W, cin = x.shape
    cout = y.shape[-1]
    rc = load().lbpf_nn_conv3x3(_dptr(x), _dptr(wt), _dptr(bias) if bias is not None else None, _dptr(y), n, H, W,
                                cin, cout, int(bool(relu)), C.c_void_p(stream) if stream else None)
    if rc != LBPF_OK:
        raise LbpfError(rc, "lbpf_nn_conv3x3 failed")


def nn_conv3x3_wgrad(x, dy, dwt, stream=None):
    """dwt (9, cout, cin) float32 += the weight gradient of one 3x3 layer with
    input x (n, H, W, cin) and output gradient dy (n, H, W, cout) (CUDA tensors)."""
    n, H, W, cin = x.shape
    cout = dy.shape[-1]
    rc = load().lbpf_nn_conv3x3_wgrad(_dptr(x), _dptr(dy), _dptr(dwt), n, H, W, cin, cout,
                                      C.c_void_p(stream) if stream else None)
    if rc != LBPF_OK:
        raise LbpfError(rc, "lbpf_nn_conv3x3_wgrad failed")


def nn_conv_error():
    """The convolution kernels' device error word (synchronises the device)."""
    w = C.c_int(0)
    rc = load().lbpf_nn_conv_error(C.byref(w))
    if rc != LBPF_OK:
        raise LbpfError(rc, "lbpf_nn_conv_error failed")
    return w.value
