"""FP64 CPU oracle of the pseudo-potential LBM time step (arXiv 2504.15018).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2504_15018_gb300``: the step lives in
``lbm.c`` (plain C, FP64, ``-ffp-contract=off``) and the parameter solve in
``params.py`` (numpy / scipy).

Population layout of the oracle: ``f[cell, i]`` (cell-major), cell index
``x + nx * (y + ny * z)``.  Velocity ordering: :func:`velocity_set`.

Parity status per function (see the tests that pin each one):
  - orc_feq, orc_guo: pinned by exact moment identities.
  - orc_psi_moments (M1, M2, F^SC, F^int): pinned by exactness on quadratic psi,
    by the closed form F^SC = -G psi grad psi on linear psi, and by the plain
    Shan-Chen reduction at eps = 0, kappa = 1.
  - orc_run: pinned by mass / momentum balance, shear-wave decay (nu = (tau-1/2)/3),
    the parabolic Poiseuille profile between bounce-back walls, MRT == BGK when all
    rates equal 1/tau, and planar-interface coexistence at the Maxwell densities.
  - MRT rates: inputs without a paper value; their placement is pinned by each basis mode
    of a uniform lattice relaxing as (1 - s_k)^n with the other moments at equilibrium, and
    by Poiseuille flow between bounce-back walls being exact at Lambda = 3/16.
  - Wetting walls (wall_rho): not in the paper; pinned by a uniform state at the wall density
    staying at rest, by the mirror-rule limit and by the order of contact angles.  The
    contact angle value itself: parity unpinned (no closed form for this scheme).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_lbm.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EPSI_DOMAIN, ENONFINITE = 0, 1, 2, 3
D2Q9, D3Q19 = 0, 1
EOS_PR, EOS_PAPER = 0, 1


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall_y", ctypes.c_int),
        ("eos_kind", ctypes.c_int),
        ("pr_a", ctypes.c_double), ("pr_b", ctypes.c_double), ("pr_R", ctypes.c_double),
        ("pr_omega", ctypes.c_double), ("pr_T", ctypes.c_double),
        ("pe_rho_v", ctypes.c_double), ("pe_rho_l", ctypes.c_double), ("pe_P", ctypes.c_double),
        ("p_scale", ctypes.c_double),
        ("G", ctypes.c_double), ("eps", ctypes.c_double), ("kappa", ctypes.c_double),
        ("tau_l", ctypes.c_double), ("tau_v", ctypes.c_double),
        ("tau_rho_v", ctypes.c_double), ("tau_rho_l", ctypes.c_double),
        ("mrt", ctypes.c_int),
        ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
        ("s_pi", ctypes.c_double), ("s_m", ctypes.c_double),
        ("fext", ctypes.c_double * 3),
        ("eps_printed", ctypes.c_int),
        ("wall_rho", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile ``lbm.c`` into ``liboracle_lbm.so`` next to it (gcc, -O2, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_variant(path: str, mutant: int) -> str:
    """Compile ``lbm.c`` with the planted mistake ``ORC_MUTANT=mutant`` into ``path``
    (tests only: the pins must fail on every such build)."""
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-fopenmp", f"-DORC_MUTANT={int(mutant)}", _SRC, "-o", path, "-lm"]
    subprocess.run(cmd, check=True)
    return path


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORC_LIB_OVERRIDE: a build_variant() library, set only by the planted-mistake tests
            L = ctypes.CDLL(os.environ.get("ORC_LIB_OVERRIDE") or build())
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(OrcParams)
            L.orc_velocity_set.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]
            L.orc_mrt_matrix.argtypes = [ctypes.c_int, dp, dp]
            L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
            L.orc_feq.restype = None
            L.orc_guo.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp]
            L.orc_guo.restype = None
            L.orc_pressure.argtypes = [pp, ctypes.c_double]
            L.orc_pressure.restype = ctypes.c_double
            for name, nargs in (("orc_force_field", 3), ("orc_psi_moments", 3), ("orc_psi_field", 1),
                                ("orc_moments", 3)):
                getattr(L, name).argtypes = [pp, dp] + [dp] * nargs
            L.orc_init.argtypes = [pp, dp, dp, dp]
            L.orc_run.argtypes = [pp, dp, ctypes.c_int]
            _lib = L
    return _lib


def _dp(a: np.ndarray | None):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(lattice: int, dims, *, wall_y: bool = False, eos: dict, G: float = -1.0,
                eps: float = 2.0, kappa: float = 1.0, tau: float = 1.0, tau_v: float | None = None,
                tau_rho=(0.0, 1.0), mrt: bool = False, rates=None, fext=(0.0, 0.0, 0.0),
                p_scale: float = 1.0, eps_printed: bool = False, wall_rho: float = 0.0) -> OrcParams:
    """Build the C parameter block.

    ``eos`` is ``{"kind": "pr", "a", "b", "R", "omega", "T"}`` (absolute T) or
    ``{"kind": "paper", "rho_v", "rho_l", "P"}`` with P = p_c / rho_c^3.
    ``rates`` = dict(s_e, s_eps, s_q, s_pi, s_m) for MRT.
    ``wall_rho`` > 0: psi on the wall nodes is psi(wall_rho) (wetting walls); 0: mirror rule.
    """
    P = OrcParams()
    P.lattice = lattice
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    P.nx, P.ny, P.nz = int(nx), int(ny), int(nz)
    P.wall_y = int(bool(wall_y))
    if eos["kind"] == "pr":
        P.eos_kind = EOS_PR
        P.pr_a, P.pr_b, P.pr_R, P.pr_omega, P.pr_T = eos["a"], eos["b"], eos.get("R", 1.0), eos["omega"], eos["T"]
    else:
        P.eos_kind = EOS_PAPER
        P.pe_rho_v, P.pe_rho_l, P.pe_P = eos["rho_v"], eos["rho_l"], eos["P"]
    P.p_scale = p_scale
    P.G, P.eps, P.kappa = G, eps, kappa
    P.tau_l = tau
    P.tau_v = tau if tau_v is None else tau_v
    P.tau_rho_v, P.tau_rho_l = tau_rho
    P.mrt = int(bool(mrt))
    r = {"s_e": 1.0, "s_eps": 1.0, "s_q": 1.0, "s_pi": 1.0, "s_m": 1.0}
    if rates:
        r.update(rates)
    P.s_e, P.s_eps, P.s_q, P.s_pi, P.s_m = r["s_e"], r["s_eps"], r["s_q"], r["s_pi"], r["s_m"]
    for a in range(3):
        P.fext[a] = fext[a]
    P.eps_printed = int(bool(eps_printed))
    P.wall_rho = wall_rho
    return P


def ncells(P: OrcParams) -> int:
    return P.nx * P.ny * P.nz


def q_of(lattice: int) -> int:
    return 9 if lattice == D2Q9 else 19


def velocity_set(lattice: int):
    q = q_of(lattice)
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    lib().orc_velocity_set(lattice, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w))
    return c, w


def mrt_matrix(lattice: int):
    q = q_of(lattice)
    M = np.zeros((q, q))
    Minv = np.zeros((q, q))
    lib().orc_mrt_matrix(lattice, _dp(M), _dp(Minv))
    return M, Minv


def feq(lattice: int, rho: float, u) -> np.ndarray:
    out = np.zeros(q_of(lattice))
    lib().orc_feq(lattice, float(rho), _dp(np.ascontiguousarray(u, dtype=np.float64)), _dp(out))
    return out


def guo(lattice: int, tau: float, F, u) -> np.ndarray:
    out = np.zeros(q_of(lattice))
    lib().orc_guo(lattice, float(tau), _dp(np.ascontiguousarray(F, dtype=np.float64)),
                  _dp(np.ascontiguousarray(u, dtype=np.float64)), _dp(out))
    return out


def pressure(P: OrcParams, rho: float) -> float:
    return lib().orc_pressure(ctypes.byref(P), float(rho))


def _check(st: int, what: str):
    if st != OK:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def init(P: OrcParams, rho0: np.ndarray, u0: np.ndarray | None = None) -> np.ndarray:
    """f = f^eq(rho0, u0); rho0 shape (N,), u0 shape (d, N). Returns f shape (N, Q)."""
    n = ncells(P)
    f = np.zeros((n, q_of(P.lattice)))
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64).reshape(-1)
    u0c = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
    _check(lib().orc_init(ctypes.byref(P), _dp(rho0), _dp(u0c), _dp(f)), "init")
    return f


def run(P: OrcParams, f: np.ndarray, nsteps: int) -> np.ndarray:
    """Advance a copy of f (shape (N, Q)) by nsteps time steps."""
    g = np.ascontiguousarray(f, dtype=np.float64).copy()
    _check(lib().orc_run(ctypes.byref(P), _dp(g), int(nsteps)), "run")
    return g


def run_status(P: OrcParams, f: np.ndarray, nsteps: int) -> int:
    g = np.ascontiguousarray(f, dtype=np.float64).copy()
    return lib().orc_run(ctypes.byref(P), _dp(g), int(nsteps))


def moments(P: OrcParams, f: np.ndarray):
    """rho (N,), u (d, N), p (N,)."""
    n = ncells(P)
    d = 2 if P.lattice == D2Q9 else 3
    rho, u, p = np.zeros(n), np.zeros((d, n)), np.zeros(n)
    _check(lib().orc_moments(ctypes.byref(P), _dp(np.ascontiguousarray(f)), _dp(rho), _dp(u), _dp(p)),
           "moments")
    return rho, u, p


def force_field(P: OrcParams, f: np.ndarray):
    """M1 (N,3), M2 (N,3,3), F (N,3) of the psi field of populations f."""
    n = ncells(P)
    M1, M2, F = np.zeros((n, 3)), np.zeros((n, 3, 3)), np.zeros((n, 3))
    _check(lib().orc_force_field(ctypes.byref(P), _dp(np.ascontiguousarray(f)), _dp(M1), _dp(M2), _dp(F)),
           "force_field")
    return M1, M2, F


def psi_moments(P: OrcParams, psi: np.ndarray):
    """M1, M2, F for a psi field given directly (shape (N,))."""
    n = ncells(P)
    M1, M2, F = np.zeros((n, 3)), np.zeros((n, 3, 3)), np.zeros((n, 3))
    psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(-1)
    _check(lib().orc_psi_moments(ctypes.byref(P), _dp(psi), _dp(M1), _dp(M2), _dp(F)), "psi_moments")
    return M1, M2, F


def psi_field(P: OrcParams, f: np.ndarray) -> np.ndarray:
    psi = np.zeros(ncells(P))
    _check(lib().orc_psi_field(ctypes.byref(P), _dp(np.ascontiguousarray(f)), _dp(psi)), "psi_field")
    return psi
