"""GB300 (sm_103a) pseudo-potential lattice Boltzmann step (arXiv 2504.15018).

Thin ctypes binding of the C ABI in ``include/plb.h``: every ``plb_*`` function
here has the C function's name and arguments and only marshals them; all work
of the method runs in the CUDA library ``_lib/libplb.so`` (built in-tree by
``builder.py``).  There is no CPU fallback: using the binding without the built
library raises.

:class:`Lattice` is a convenience wrapper that owns a torch device workspace
and calls the same entry points.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libplb.so")
_lock = threading.Lock()
_lib = None

# status codes and enums (include/plb.h)
PLB_OK, PLB_EINVAL, PLB_ENOMEM, PLB_ECUDA, PLB_ENONFINITE, PLB_EPSI_DOMAIN, PLB_ETIMEOUT, PLB_EUNSUPPORTED = range(8)
PLB_D2Q9, PLB_D3Q19 = 0, 1
PLB_EOS_PR, PLB_EOS_PAPER = 0, 1
PLB_FP64, PLB_FP32, PLB_FP16S = 0, 1, 2
PLB_BGK, PLB_MRT = 0, 1
PLB_STREAM_AA, PLB_STREAM_FUSED = 0, 1
PLB_MASS, PLB_MOMENTUM, PLB_UMAX, PLB_UL1, PLB_UL2, PLB_MEAN_RHO, PLB_MEAN_P = range(7)

STATUS_NAMES = {0: "PLB_OK", 1: "PLB_EINVAL", 2: "PLB_ENOMEM", 3: "PLB_ECUDA", 4: "PLB_ENONFINITE",
                5: "PLB_EPSI_DOMAIN", 6: "PLB_ETIMEOUT", 7: "PLB_EUNSUPPORTED"}


class PlbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class plb_eos_params(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
                ("omega", ctypes.c_double), ("T_over_Tc", ctypes.c_double),
                ("rho_v", ctypes.c_double), ("rho_l", ctypes.c_double), ("pc_over_rhoc3", ctypes.c_double),
                ("p_scale", ctypes.c_double)]


class plb_opts(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("tau_v", ctypes.c_double),
                ("tau_rho_v", ctypes.c_double), ("tau_rho_l", ctypes.c_double),
                ("collision", ctypes.c_int),
                ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
                ("s_pi", ctypes.c_double), ("s_m", ctypes.c_double),
                ("precision", ctypes.c_int), ("rho_ref", ctypes.c_double), ("wall_y", ctypes.c_int),
                ("body_force", ctypes.c_double * 3), ("fp16_rounding", ctypes.c_int), ("streaming", ctypes.c_int),
                ("wall_rho", ctypes.c_double)]


class plb_instance(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 3), ("eos", plb_eos_params), ("tau", ctypes.c_double),
                ("G", ctypes.c_double), ("eps", ctypes.c_double), ("opts", plb_opts)]


class plb_xfer(ctypes.Structure):
    _fields_ = [("send_off", ctypes.c_longlong), ("recv_off", ctypes.c_longlong), ("bytes", ctypes.c_longlong),
                ("face", ctypes.c_int), ("region", ctypes.c_int)]


_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_VP = ctypes.c_void_p

# name -> (restype, argtypes)
_SIGNATURES = {
    "plb_default_opts": (None, [ctypes.POINTER(plb_opts)]),
    "plb_velocity_set": (ctypes.c_int, [ctypes.c_int, _IP, _DP]),
    "plb_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, _IP, ctypes.POINTER(plb_opts)]),
    "plb_create": (ctypes.c_int, [ctypes.c_int, _IP, ctypes.POINTER(plb_eos_params), ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.POINTER(plb_opts), _VP, ctypes.c_size_t,
                                  _VP, ctypes.POINTER(_VP)]),
    "plb_destroy": (None, [_VP]),
    "plb_init": (ctypes.c_int, [_VP, _DP, _DP]),
    "plb_init_physical": (ctypes.c_int, [_VP, _DP, _DP]),
    "plb_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "plb_step_timed": (ctypes.c_int, [_VP, ctypes.c_int, _DP]),
    "plb_status": (ctypes.c_int, [_VP]),
    "plb_time": (ctypes.c_longlong, [_VP]),
    "plb_moments": (ctypes.c_int, [_VP, _DP, _DP, _DP]),
    "plb_reduce": (ctypes.c_int, [_VP, ctypes.c_int, _IP, _IP, _DP]),
    "plb_get_populations": (ctypes.c_int, [_VP, _DP]),
    "plb_set_populations": (ctypes.c_int, [_VP, _DP]),
    "plb_state_bytes": (ctypes.c_size_t, [_VP]),
    "plb_get_state": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "plb_set_state": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "plb_solve_params": (ctypes.c_int, [ctypes.POINTER(plb_eos_params), _DP, _DP, _DP]),
    "plb_si_convert": (ctypes.c_int, [_DP, _DP, ctypes.c_double, _DP]),
    "plb_step_pairs_static": (ctypes.c_int, [ctypes.c_int, _IP, ctypes.POINTER(plb_eos_params), ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.POINTER(plb_opts), _VP,
                                             ctypes.c_int, ctypes.c_longlong, _VP]),
    "plb_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(plb_instance)]),
    "plb_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(plb_instance), _VP, ctypes.c_size_t,
                                        _VP, ctypes.POINTER(_VP)]),
    "plb_batch_destroy": (None, [_VP]),
    "plb_batch_instance": (_VP, [_VP, ctypes.c_int]),
    "plb_batch_init": (ctypes.c_int, [_VP, ctypes.c_int, _DP, _DP]),
    "plb_batch_init_physical": (ctypes.c_int, [_VP, ctypes.c_int, _DP, _DP]),
    "plb_batch_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "plb_batch_status": (ctypes.c_int, [_VP]),
    "plb_batch_reset_error": (ctypes.c_int, [_VP]),
    "plb_batch_configure": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_uint]),
    "plb_batch_autotune": (ctypes.c_int, [_VP, ctypes.c_int, _IP, _IP, _DP]),
    "plb_batch_withhold_arrivals": (ctypes.c_int, [_VP, ctypes.c_uint]),
    "plb_batch_time": (ctypes.c_longlong, [_VP]),
    "plb_batch_launch_counts": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    "plb_slab_plan": (ctypes.c_int, [ctypes.c_int, _IP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(plb_xfer), ctypes.c_int, _IP]),
    "plb_slab_bind": (ctypes.c_int, [_VP, ctypes.c_int]),
    "plb_slab_pass": (ctypes.c_int, [_VP, ctypes.c_int]),
    "plb_slab_regions": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "plb_slab_exchange": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "plb_last_error": (ctypes.c_char_p, []),
}


def build(force: bool = False) -> str:
    from . import builder
    return builder.build(force=force)


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run paper_2504_15018_gb300.build())")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


def _check(code: int):
    if code != PLB_OK:
        raise PlbError(code, lib().plb_last_error().decode())


def _dptr(a):
    if a is None:
        return _DP()
    if hasattr(a, "data_ptr"):                      # torch tensor (pinned host memory)
        return ctypes.cast(a.data_ptr(), _DP)
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _iptr(v):
    if v is None:
        return _IP()
    return (ctypes.c_int * len(v))(*[int(x) for x in v])


# ------------------------------------------------------------ C-ABI functions

def plb_default_opts() -> plb_opts:
    o = plb_opts()
    lib().plb_default_opts(ctypes.byref(o))
    return o


def plb_velocity_set(lattice: int):
    q = 9 if lattice == PLB_D2Q9 else 19
    c = (ctypes.c_int * (3 * q))()
    w = (ctypes.c_double * q)()
    r = lib().plb_velocity_set(lattice, c, w)
    if r < 0:
        raise PlbError(PLB_EINVAL, "unknown lattice")
    return np.array(c[:], dtype=np.int32).reshape(q, 3), np.array(w[:])


def plb_workspace_bytes(lattice: int, dims, opts: plb_opts | None = None) -> int:
    return lib().plb_workspace_bytes(lattice, _iptr(dims), ctypes.byref(opts) if opts is not None else None)


def plb_create(lattice: int, dims, eos: plb_eos_params, tau: float, G: float, eps: float, opts: plb_opts | None,
               dev_workspace: int, ws_bytes: int, cuda_stream: int):
    h = _VP()
    _check(lib().plb_create(lattice, _iptr(dims), ctypes.byref(eos), tau, G, eps,
                            ctypes.byref(opts) if opts is not None else None, _VP(dev_workspace), ws_bytes,
                            _VP(cuda_stream), ctypes.byref(h)))
    return h


def plb_destroy(h):
    lib().plb_destroy(h)


def plb_init(h, rho0, u0=None):
    _check(lib().plb_init(h, _dptr(rho0), _dptr(u0)))


def plb_init_physical(h, rho0, u0=None):
    _check(lib().plb_init_physical(h, _dptr(rho0), _dptr(u0)))


def plb_step(h, n: int):
    _check(lib().plb_step(h, int(n)))


def plb_step_timed(h, n: int):
    """Returns (ms of the psi passes, ms of the fused force/collide/stream passes)."""
    ms = np.zeros(2)
    _check(lib().plb_step_timed(h, int(n), _dptr(ms)))
    return float(ms[0]), float(ms[1])


def plb_status(h):
    _check(lib().plb_status(h))


def plb_time(h) -> int:
    return lib().plb_time(h)


def plb_moments(h, rho=None, u=None, p=None):
    _check(lib().plb_moments(h, _dptr(rho), _dptr(u), _dptr(p)))


def plb_reduce(h, what: int, lo=None, hi=None) -> np.ndarray:
    out = np.zeros(3)
    _check(lib().plb_reduce(h, what, _iptr(lo), _iptr(hi), _dptr(out)))
    return out if what == PLB_MOMENTUM else out[:1]


def plb_get_populations(h, f):
    _check(lib().plb_get_populations(h, _dptr(f)))


def plb_set_populations(h, f):
    _check(lib().plb_set_populations(h, _dptr(f)))


def plb_state_bytes(h) -> int:
    return lib().plb_state_bytes(h)


def plb_get_state(h, buf: np.ndarray):
    _check(lib().plb_get_state(h, buf.ctypes.data_as(_VP), buf.nbytes))


def plb_set_state(h, buf: np.ndarray):
    _check(lib().plb_set_state(h, buf.ctypes.data_as(_VP), buf.nbytes))


def plb_solve_params(eos: plb_eos_params):
    rv, rl, p0 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().plb_solve_params(ctypes.byref(eos), ctypes.byref(rv), ctypes.byref(rl), ctypes.byref(p0)))
    return rv.value, rl.value, p0.value


def plb_si_convert(si, lat, xi: float) -> dict:
    out = (ctypes.c_double * 11)()
    _check(lib().plb_si_convert((ctypes.c_double * 6)(*si), (ctypes.c_double * 3)(*lat), float(xi), out))
    keys = ["C_L", "C_T", "C_M", "C_U", "C_VF", "C_gamma", "rho_v", "tau_v", "gamma_lat", "P", "kappa"]
    return dict(zip(keys, out[:]))


def plb_step_pairs_static(lattice: int, dims, eos: plb_eos_params, tau: float, G: float, eps: float,
                          opts: plb_opts | None, dev_pops: int, npairs: int, t0: int, cuda_stream: int):
    """Allocation-free stepping of a caller-owned device population array (2 * npairs steps from
    time step t0)."""
    _check(lib().plb_step_pairs_static(lattice, _iptr(dims), ctypes.byref(eos), tau, G, eps,
                                       ctypes.byref(opts) if opts is not None else None, _VP(dev_pops),
                                       int(npairs), int(t0), _VP(cuda_stream)))


def plb_batch_workspace_bytes(lattice: int, instances) -> int:
    arr = (plb_instance * len(instances))(*instances)
    return lib().plb_batch_workspace_bytes(lattice, len(instances), arr)


def plb_batch_create(lattice: int, instances, dev_workspace: int, ws_bytes: int, cuda_stream: int):
    arr = (plb_instance * len(instances))(*instances)
    b = _VP()
    _check(lib().plb_batch_create(lattice, len(instances), arr, _VP(dev_workspace), ws_bytes, _VP(cuda_stream),
                                  ctypes.byref(b)))
    return b


def plb_batch_destroy(b):
    lib().plb_batch_destroy(b)


def plb_batch_instance(b, k: int):
    h = lib().plb_batch_instance(b, int(k))
    if not h:
        raise PlbError(PLB_EINVAL, f"no instance {k}")
    return _VP(h)


def plb_batch_init(b, k: int, rho0, u0=None):
    _check(lib().plb_batch_init(b, int(k), _dptr(rho0), _dptr(u0)))


def plb_batch_init_physical(b, k: int, rho0, u0=None):
    _check(lib().plb_batch_init_physical(b, int(k), _dptr(rho0), _dptr(u0)))


def plb_batch_step(b, nsteps: int):
    _check(lib().plb_batch_step(b, int(nsteps)))


def plb_batch_status(b):
    _check(lib().plb_batch_status(b))


def plb_batch_reset_error(b):
    _check(lib().plb_batch_reset_error(b))


def plb_batch_configure(b, tile_cells: int = 0, blocks_per_sm: int = 0, spin_limit: int = 0):
    _check(lib().plb_batch_configure(b, int(tile_cells), int(blocks_per_sm), int(spin_limit)))


def plb_batch_autotune(b, steps_per_candidate: int = 5):
    tc, bps, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().plb_batch_autotune(b, int(steps_per_candidate), ctypes.byref(tc), ctypes.byref(bps),
                                    ctypes.byref(ms)))
    return tc.value, bps.value, ms.value


def plb_batch_withhold_arrivals(b, count: int):
    _check(lib().plb_batch_withhold_arrivals(b, int(count)))


def plb_batch_time(b) -> int:
    return lib().plb_batch_time(b)


def plb_batch_launch_counts(b) -> dict:
    c = (ctypes.c_longlong * 3)()
    _check(lib().plb_batch_launch_counts(b, c))
    return {"graph_captures": c[0], "graph_launches": c[1], "direct_launches": c[2]}


def plb_slab_plan(lattice: int, dims, precision: int, wall_y: int, pass_: int, odd: int) -> list:
    """The exchange plan of a slab (host-only): a list of dicts with send_off, recv_off, bytes,
    face and region."""
    out = (plb_xfer * 16)()
    n = ctypes.c_int(0)
    _check(lib().plb_slab_plan(lattice, _iptr(dims), precision, int(wall_y), int(pass_), int(odd), out, 16,
                               ctypes.byref(n)))
    return [{k: getattr(out[i], k) for k, _ in plb_xfer._fields_} for i in range(n.value)]


def plb_slab_bind(h, z_first: int):
    _check(lib().plb_slab_bind(h, int(z_first)))


def plb_slab_pass(h, pass_: int):
    _check(lib().plb_slab_pass(h, int(pass_)))


def plb_slab_regions(h):
    a, b = _VP(), _VP()
    _check(lib().plb_slab_regions(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def plb_slab_exchange(lower, upper, pass_: int):
    _check(lib().plb_slab_exchange(lower, upper, int(pass_)))


# ------------------------------------------------------------------- helpers

def pr_eos(T_over_Tc: float, a: float = 2.0 / 49.0, b: float = 2.0 / 21.0, R: float = 1.0, omega: float = 0.327,
           p_scale: float = 1.0) -> plb_eos_params:
    e = plb_eos_params()
    e.kind, e.a, e.b, e.R, e.omega, e.T_over_Tc, e.p_scale = PLB_EOS_PR, a, b, R, omega, T_over_Tc, p_scale
    return e


def paper_eos(rho_v: float, rho_l: float, pc_over_rhoc3: float, p_scale: float = 1.0) -> plb_eos_params:
    e = plb_eos_params()
    e.kind, e.rho_v, e.rho_l, e.pc_over_rhoc3, e.p_scale = PLB_EOS_PAPER, rho_v, rho_l, pc_over_rhoc3, p_scale
    return e


def make_opts(**kw) -> plb_opts:
    o = plb_default_opts()
    for k, v in kw.items():
        if k == "body_force":
            for a in range(3):
                o.body_force[a] = v[a] if a < len(v) else 0.0
        else:
            setattr(o, k, v)
    return o


def make_instance(dims, eos: plb_eos_params, tau: float = 1.0, G: float = -1.0, eps: float = 2.0,
                  opts: plb_opts | None = None) -> plb_instance:
    inst = plb_instance()
    d = (list(dims) + [1, 1])[:3]
    for a in range(3):
        inst.dims[a] = int(d[a])
    inst.eos = eos
    inst.tau, inst.G, inst.eps = tau, G, eps
    inst.opts = opts if opts is not None else plb_default_opts()
    return inst


class Batch:
    """A batch of independent lattices advanced by one persistent launch per step call."""

    def __init__(self, lattice: int, instances, device: str = "cuda", stream=None):
        import torch
        self.lattice = lattice
        self.instances = list(instances)
        nbytes = plb_batch_workspace_bytes(lattice, self.instances)
        if nbytes == 0:
            raise PlbError(PLB_EINVAL, "bad batch description")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        aligned = (self.ws.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.ws.device)
        self.b = plb_batch_create(lattice, self.instances, aligned, nbytes, self.stream.cuda_stream)
        self.Q = 9 if lattice == PLB_D2Q9 else 19
        self.D = 2 if lattice == PLB_D2Q9 else 3

    def __del__(self):
        b = getattr(self, "b", None)
        if b:
            try:
                plb_batch_destroy(b)
            except Exception:
                pass
            self.b = None

    def __len__(self):
        return len(self.instances)

    def cells(self, k: int) -> int:
        d = self.instances[k].dims
        return d[0] * d[1] * d[2]

    def init(self, k: int, rho0, u0=None, physical: bool = False):
        """physical: plb_batch_init_physical (the velocity of Eq. Momentum is u0 at t = 0)."""
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64).reshape(-1)
        u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
        (plb_batch_init_physical if physical else plb_batch_init)(self.b, k, rho0, u0)

    def step(self, n: int = 1):
        plb_batch_step(self.b, n)

    def status(self):
        plb_batch_status(self.b)

    def autotune(self, steps_per_candidate: int = 5):
        return plb_batch_autotune(self.b, steps_per_candidate)

    def configure(self, tile_cells: int = 0, blocks_per_sm: int = 0, spin_limit: int = 0):
        plb_batch_configure(self.b, tile_cells, blocks_per_sm, spin_limit)

    def populations(self, k: int) -> np.ndarray:
        f = np.zeros((self.Q, self.cells(k)))
        plb_get_populations(plb_batch_instance(self.b, k), f)
        return f

    def moments(self, k: int):
        n = self.cells(k)
        rho, u, p = np.zeros(n), np.zeros((self.D, n)), np.zeros(n)
        plb_moments(plb_batch_instance(self.b, k), rho, u, p)
        return rho, u, p

    def reduce(self, k: int, what: int, lo=None, hi=None):
        return plb_reduce(plb_batch_instance(self.b, k), what, lo, hi)


class Lattice:
    """One P-LBM lattice on the current CUDA device, workspace owned by torch."""

    def __init__(self, lattice: int, dims, eos: plb_eos_params, tau: float = 1.0, G: float = -1.0, eps: float = 2.0,
                 opts: plb_opts | None = None, device: str = "cuda", stream=None):
        import torch
        self.lattice = lattice
        self.dims = tuple(int(d) for d in (list(dims) + [1, 1])[:3])
        self.Q = 9 if lattice == PLB_D2Q9 else 19
        self.D = 2 if lattice == PLB_D2Q9 else 3
        self.n = self.dims[0] * self.dims[1] * self.dims[2]
        self.opts = opts if opts is not None else plb_default_opts()
        nbytes = plb_workspace_bytes(lattice, self.dims, self.opts)
        if nbytes == 0:
            raise PlbError(PLB_EINVAL, "bad lattice, dims or precision")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.ws.device)
        self.h = plb_create(lattice, self.dims, eos, tau, G, eps, self.opts, aligned, nbytes,
                            self.stream.cuda_stream)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            try:
                plb_destroy(h)
            except Exception:
                pass
            self.h = None

    def init(self, rho0, u0=None, physical: bool = False):
        """physical: plb_init_physical (the velocity of Eq. Momentum is u0 at t = 0)."""
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64).reshape(-1)
        u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
        (plb_init_physical if physical else plb_init)(self.h, rho0, u0)

    def step(self, n: int = 1):
        plb_step(self.h, n)

    def step_timed(self, n: int):
        return plb_step_timed(self.h, n)

    def status(self):
        plb_status(self.h)

    @property
    def time(self) -> int:
        return plb_time(self.h)

    def moments(self):
        rho, u, p = np.zeros(self.n), np.zeros((self.D, self.n)), np.zeros(self.n)
        plb_moments(self.h, rho, u, p)
        return rho, u, p

    def reduce(self, what: int, lo=None, hi=None):
        return plb_reduce(self.h, what, lo, hi)

    def populations(self) -> np.ndarray:
        f = np.zeros((self.Q, self.n))
        plb_get_populations(self.h, f)
        return f

    def set_populations(self, f):
        plb_set_populations(self.h, np.ascontiguousarray(f, dtype=np.float64))

    def get_state(self) -> np.ndarray:
        buf = np.zeros(plb_state_bytes(self.h), dtype=np.uint8)
        plb_get_state(self.h, buf)
        return buf

    def set_state(self, buf: np.ndarray):
        plb_set_state(self.h, np.ascontiguousarray(buf))
