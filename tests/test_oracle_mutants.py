"""The oracle's pins are sharp: for each of ten plausible mistakes planted in the oracle
(a separate build of lbm.c with ORC_MUTANT = k; the oracle itself is ORC_MUTANT = 0), the pin
aimed at it fails, while the same pins pass on an unmutated build made the same way.  Each run
is a child pytest process that loads the variant through ORC_LIB_OVERRIDE."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# mutant -> (the planted mistake, the pins of tests/test_oracle_step.py that must catch it)
MUTANTS = {
    1: ("sign of the u^2 term of f^eq", "test_equilibrium_moments"),
    2: ("Guo term without its (c.u)(c.F) part", "test_guo_forcing_moments"),
    3: ("sign of the kappa term of the interaction force", "test_force_terms_follow_the_pressure_tensor"),
    4: ("M1 stencil without the 1/c_s^2 factor", "test_stencils_exact_on_quadratic_psi"),
    5: ("D3Q19 MRT rates s_q and s_m swapped", "test_mrt_modes_relax_at_their_own_rates"),
    6: ("MRT forcing factor 1 - s instead of 1 - s/2", "test_momentum_balance_and_third_law"),
    7: ("upper bounce-back wall off by one row", "test_poiseuille_between_bounce_back_walls"),
    8: ("psi without the factor 2 of Eq. Interaction_Potential",
        "test_planar_coexistence_follows_mechanical_stability"),
    9: ("tau(rho) not clamped above rho_l", "test_shear_wave_decay_follows_tau_of_rho"),
    10: ("D2Q9 Shan-Chen weight omega(2) = 1/6 instead of 1/12", "test_stencils_exact_on_quadratic_psi"),
}


def _run_pins(lib_path, expr):
    env = dict(os.environ, ORC_LIB_OVERRIDE=lib_path)
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_step.py"), "-k", expr],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_pins_pass_on_an_unmutated_variant_build(tmp_path):
    path = oracle.build_variant(str(tmp_path / "orc0.so"), 0)
    r = _run_pins(path, " or ".join(pin for _, pin in MUTANTS.values()))
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_each_planted_mistake_fails_its_pin(tmp_path, mutant):
    what, pin = MUTANTS[mutant]
    path = oracle.build_variant(str(tmp_path / f"orc{mutant}.so"), mutant)
    r = _run_pins(path, pin)
    assert r.returncode == 1 and " failed" in r.stdout, f"mutant {mutant} ({what}) passed {pin}:\n{r.stdout[-2000:]}"
