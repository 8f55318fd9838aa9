"""The parameter-solve pins are sharp: four plausible mistakes planted in oracle.params (in this
process, with monkeypatch, one at a time) each make the pin aimed at it fail, while the same
pins pass on the unmodified module."""
import numpy as np
import pytest

import test_oracle_params as pins
from oracle import params as pp


def _alpha_without_acentric_factor(orig):
    return lambda T, Tc, omega: orig(T, Tc, 0.0)


def _thickness_without_the_6(orig):
    # Eq. thickness with r xi^2 in place of 6 r xi^2
    return lambda xi, rho_v, rho_l, r=1.0: 6.0 * orig(xi, rho_v, rho_l, r)


def _kappa_with_the_ratio_inverted(orig):
    # sqrt(2 r P / 27) in place of sqrt(27 / (2 r P)): the two differ by the factor 2 r P / 27
    return lambda gamma, P, rho_v, rho_l, r=1.0: orig(gamma, P, rho_v, rho_l, r) * (2.0 * r * P / 27.0)


def _tau_without_clamp(orig):
    return lambda rho, tau_v, tau_l, rho_v, rho_l: tau_v + (np.asarray(rho, dtype=np.float64) - rho_v) / (
        rho_l - rho_v) * (tau_l - tau_v)


KAPPA_CASE = pins.GOLDEN["kappa"]["cases"][0]
MUTANTS = {
    "pr_alpha": (_alpha_without_acentric_factor,
                 lambda: pins.test_pr_maxwell_equal_chemical_potential(0.8, 0.201851, 7.182058)),
    "P_from_thickness": (_thickness_without_the_6, lambda: pins.test_kappa_matches_printed_values(KAPPA_CASE)),
    "kappa_from_gamma": (_kappa_with_the_ratio_inverted, lambda: pins.test_kappa_matches_printed_values(KAPPA_CASE)),
    "tau_of_rho": (_tau_without_clamp, pins.test_tau_interpolation_hits_both_phases_and_clamps),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_its_pin(name, monkeypatch):
    make, pin = MUTANTS[name]
    pin()                                               # passes on the unmodified module
    monkeypatch.setattr(pp, name, make(getattr(pp, name)))
    with pytest.raises(AssertionError):
        pin()
