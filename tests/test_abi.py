"""C-ABI library checks that need no GPU: every symbol declared in include/*.h is
exported, the host-side entry points (velocity set, workspace layout, parameter
solve, SI converter) agree with the oracle, and invalid arguments are rejected
before any device work."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import paper_2504_15018_gb300 as plb
from oracle import params as pp
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    plb.build()
    return plb.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(plb_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(plb.exported_symbols()) | {n for n in names if hasattr(L, n)}


def test_binding_covers_every_declared_function():
    assert set(declared_functions()) <= set(plb.exported_symbols())


@pytest.mark.parametrize("lattice", [plb.PLB_D2Q9, plb.PLB_D3Q19])
def test_velocity_set_matches_oracle_as_a_set(L, lattice):
    c, w = plb.plb_velocity_set(lattice)
    oc, ow = oracle.velocity_set(lattice)
    lib_set = {tuple(v): wi for v, wi in zip(c.tolist(), w)}
    orc_set = {tuple(v): wi for v, wi in zip(oc.tolist(), ow)}
    assert lib_set.keys() == orc_set.keys()
    for k in lib_set:
        assert lib_set[k] == pytest.approx(orc_set[k], abs=1e-16)
    # opposite directions are adjacent
    for i in range(1, len(w), 2):
        assert (c[i] == -c[i + 1]).all()


@pytest.mark.parametrize("t_ratio", [0.7, 0.8, 0.9])
def test_library_maxwell_matches_oracle(L, t_ratio):
    rv, rl, p0 = plb.plb_solve_params(plb.pr_eos(t_ratio))
    T = t_ratio * pp.pr_Tc(2 / 49, 2 / 21)
    orv, orl, op0 = pp.pr_maxwell(2 / 49, 2 / 21, 1.0, 0.327, T)
    assert rv == pytest.approx(orv, rel=1e-9)
    assert rl == pytest.approx(orl, rel=1e-11)
    assert p0 == pytest.approx(op0, rel=1e-10)


def test_library_paper_eos_coexistence(L):
    rv, rl, p0 = plb.plb_solve_params(plb.paper_eos(0.0375, 1.187, 0.044))
    assert (rv, rl) == (0.0375, 1.187)
    assert p0 == pytest.approx(0.044 * 0.0375 * 1.187 ** 2, rel=1e-15)


def test_supercritical_has_no_coexistence(L):
    with pytest.raises(plb.PlbError) as e:
        plb.plb_solve_params(plb.pr_eos(1.05))
    assert e.value.code == plb.PLB_EINVAL


@pytest.mark.parametrize("gamma,tau_l", [(7.58e-3, 0.56), (0.758e-3, 0.68), (75.8e-3, 0.52)])
def test_si_converter_matches_oracle(L, gamma, tau_l):
    out = plb.plb_si_convert([37.5, 1187.0, 0.339e-6, 0.158e-6, gamma, 10e-6], [100, tau_l, 1.187], 1.5)
    ref = pp.si_converter(rho_v_phs=37.5, rho_l_phs=1187.0, nu_v_phs=0.339e-6, nu_l_phs=0.158e-6, gamma_phs=gamma,
                          L_phs=10e-6, L_lat=100, tau_l=tau_l, rho_l_lat=1.187, xi_lat=1.5)
    for k in ("C_L", "C_T", "C_M", "C_U", "C_VF", "C_gamma", "rho_v", "tau_v", "gamma_lat", "P", "kappa"):
        assert out[k] == pytest.approx(ref[k], rel=1e-12), k


def test_workspace_layout(L):
    o = plb.make_opts(precision=plb.PLB_FP32)
    n = plb.plb_workspace_bytes(plb.PLB_D3Q19, (512, 256, 256), o)
    pops = 19 * 512 * 256 * 256 * 4
    psi = (512 + 8 + 24) * 258 * 258 * 4
    assert pops + psi < n < pops + psi + 64 * 2 ** 20
    assert plb.plb_workspace_bytes(plb.PLB_D2Q9, (8, 8, 2), o) == 0      # D2Q9 needs nz = 1
    assert plb.plb_workspace_bytes(plb.PLB_D2Q9, (0, 8, 1), o) == 0
    o16 = plb.make_opts(precision=plb.PLB_FP16S)
    assert plb.plb_workspace_bytes(plb.PLB_D3Q19, (64, 64, 64), o16) < plb.plb_workspace_bytes(
        plb.PLB_D3Q19, (64, 64, 64), o)
    # single-pass stepping keeps a second population copy (planes padded to 128 cells)
    of = plb.make_opts(precision=plb.PLB_FP32, streaming=plb.PLB_STREAM_FUSED)
    assert plb.plb_workspace_bytes(plb.PLB_D3Q19, (512, 256, 256), of) == n + pops
    assert plb.plb_workspace_bytes(plb.PLB_D2Q9, (30, 7, 1), of) - plb.plb_workspace_bytes(
        plb.PLB_D2Q9, (30, 7, 1), o) == (9 * 256 * 4 + 255) // 256 * 256


def test_create_rejects_bad_arguments_without_touching_the_device(L):
    eos = plb.pr_eos(0.8)
    dims = (8, 8, 1)
    o = plb.plb_default_opts()
    nbytes = plb.plb_workspace_bytes(plb.PLB_D2Q9, dims, o)
    fake = 1 << 40          # never dereferenced: validation fails first
    cases = [
        dict(tau=0.5), dict(G=1.0), dict(G=0.0), dict(ws=nbytes - 1), dict(ptr=fake + 8),
    ]
    for c in cases:
        with pytest.raises(plb.PlbError) as e:
            plb.plb_create(plb.PLB_D2Q9, dims, eos, c.get("tau", 1.0), c.get("G", -1.0), 2.0, o,
                           c.get("ptr", fake), c.get("ws", nbytes), 0)
        assert e.value.code in (plb.PLB_EINVAL, plb.PLB_ENOMEM)
    with pytest.raises(plb.PlbError) as e:
        plb.plb_create(plb.PLB_D2Q9, dims, eos, 1.0, -1.0, 2.0, o, fake, nbytes - 1, 0)
    assert e.value.code == plb.PLB_ENOMEM


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of plb_eos_params, plb_opts and plb_instance have the size and the
    field offsets the C compiler gives the header's structs (a C program built with gcc
    against include/plb.h prints them)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"plb_eos_params": plb.plb_eos_params, "plb_opts": plb.plb_opts, "plb_instance": plb.plb_instance}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "plb.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ['    return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


NULL_HANDLE_CALLS = r"""
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_2504_15018_gb300 as plb
L = plb.lib()
buf = np.zeros(64)
dp = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
calls = {
    "plb_init": lambda: L.plb_init(None, dp, None),
    "plb_init_physical": lambda: L.plb_init_physical(None, dp, None),
    "plb_step": lambda: L.plb_step(None, 1),
    "plb_step_timed": lambda: L.plb_step_timed(None, 1, dp),
    "plb_status": lambda: L.plb_status(None),
    "plb_time": lambda: L.plb_time(None),
    "plb_moments": lambda: L.plb_moments(None, dp, None, None),
    "plb_reduce": lambda: L.plb_reduce(None, 0, None, None, dp),
    "plb_get_populations": lambda: L.plb_get_populations(None, dp),
    "plb_set_populations": lambda: L.plb_set_populations(None, dp),
    "plb_state_bytes": lambda: L.plb_state_bytes(None),
    "plb_get_state": lambda: L.plb_get_state(None, None, 0),
    "plb_set_state": lambda: L.plb_set_state(None, None, 0),
    "plb_destroy": lambda: L.plb_destroy(None),
    "plb_batch_instance": lambda: L.plb_batch_instance(None, 0),
    "plb_batch_init": lambda: L.plb_batch_init(None, 0, dp, None),
    "plb_batch_init_physical": lambda: L.plb_batch_init_physical(None, 0, dp, None),
    "plb_batch_step": lambda: L.plb_batch_step(None, 1),
    "plb_batch_status": lambda: L.plb_batch_status(None),
    "plb_batch_reset_error": lambda: L.plb_batch_reset_error(None),
    "plb_batch_configure": lambda: L.plb_batch_configure(None, 0, 0, 0),
    "plb_batch_autotune": lambda: L.plb_batch_autotune(None, 1, None, None, None),
    "plb_batch_withhold_arrivals": lambda: L.plb_batch_withhold_arrivals(None, 1),
    "plb_batch_time": lambda: L.plb_batch_time(None),
    "plb_batch_destroy": lambda: L.plb_batch_destroy(None),
}
print(json.dumps({k: f() for k, f in calls.items()}))
"""


def test_null_handles_are_refused_before_any_device_work(L, tmp_path):
    """Every entry point that takes a lattice or batch handle, given NULL, returns
    PLB_EINVAL (or its documented value: -1 steps, 0 bytes, a NULL view) without touching
    the device; run in a child process so that a crash fails this test only."""
    import json
    import subprocess
    import sys
    script = tmp_path / "null_calls.py"
    script.write_text(NULL_HANDLE_CALLS)
    r = subprocess.run([sys.executable, str(script), ROOT], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    value_returning = {"plb_time": -1, "plb_batch_time": -1, "plb_state_bytes": 0,
                       "plb_batch_instance": None, "plb_destroy": None, "plb_batch_destroy": None}
    handle_funcs = [n for n in declared_functions() if n in got]
    assert len(handle_funcs) == len(got)
    for name, v in got.items():
        assert v == value_returning.get(name, plb.PLB_EINVAL), (name, v)
