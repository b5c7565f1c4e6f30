"""Entropy production of the two dissipators (the paper's validation of the secular master
equation, the supplement's entropy-production section, Eqs. 202-210): the conventional
equation matches its closed form and can produce entropy at a negative rate; the secular
equation never does."""

import math

import numpy as np
import pytest

from oracle import entropy as en

TWO_PI = 2.0 * math.pi
OMEGA, KAPPA, N = TWO_PI * 5.0, 0.01, 48


@pytest.mark.parametrize("eta", [-TWO_PI * 0.05, TWO_PI * 0.05])
@pytest.mark.parametrize("kT", [TWO_PI * 2.0, TWO_PI * 8.0])
@pytest.mark.parametrize("c", [0.4, 1.0, 2.5, 4.0])
def test_conventional_matches_closed_form(eta, kT, c):
    """The supplement's Eq. 204: T_E Pi(0) / kappa = (N_0 - nbar)[omega (1 - T_E/T_0) + 4 eta N_0]."""
    nbar = 1.0 / math.expm1(OMEGA / kT)
    N0, T0 = 1.0 / math.expm1(c), OMEGA / c
    closed = KAPPA / kT * (N0 - nbar) * (OMEGA * (1.0 - kT / T0) + 4.0 * eta * N0)
    num = en.entropy_production(en.oscillator(N, OMEGA, eta, KAPPA, kT, False), en.gaussian_state(N, c), kT)
    assert abs(num - closed) <= 1e-4 * abs(closed) + 1e-12


@pytest.mark.parametrize("eta,c", [(-TWO_PI * 0.05, 2.495), (TWO_PI * 0.05, 2.504)])
def test_conventional_can_be_negative_and_secular_is_not(eta, c):
    """The supplement's Eqs. 207-209: for either sign of eta there is an initial temperature
    T_0 close to T_E (c close to omega / T_E) with Pi(0) < 0 under the conventional equation;
    the secular equation gives Pi(0) > 0 for the same state."""
    kT = TWO_PI * 2.0
    T0 = OMEGA / c
    N0 = 1.0 / math.expm1(c)
    bound = kT / (4.0 * N0 * eta / OMEGA + 1.0)
    assert min(kT, bound) < T0 < max(kT, bound)  # the paper's window for a negative rate
    rho = en.gaussian_state(N, c)
    assert en.entropy_production(en.oscillator(N, OMEGA, eta, KAPPA, kT, False), rho, kT) < 0.0
    assert en.entropy_production(en.oscillator(N, OMEGA, eta, KAPPA, kT, True), rho, kT) > 0.0


def test_secular_never_negative():
    """The secular equation satisfies detailed balance with respect to the Gibbs state of H at
    every transition frequency, so Pi >= 0 for every state (diagonal Gaussian states on a
    grid of c and T_E, and random full-rank states)."""
    rng = np.random.default_rng(7)
    for eta in (-TWO_PI * 0.05, TWO_PI * 0.05):
        for kT in (TWO_PI * 1.0, TWO_PI * 2.0, TWO_PI * 8.0):
            osc = en.oscillator(N, OMEGA, eta, KAPPA, kT, True)
            for c in np.linspace(0.3, 6.0, 24):
                assert en.entropy_production(osc, en.gaussian_state(N, c), kT) >= -1e-12
            small = en.oscillator(12, OMEGA, eta, KAPPA, kT, True)
            for _ in range(5):
                X = rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12))
                rho = X @ X.conj().T
                rho /= np.trace(rho)
                assert en.entropy_production(small, rho, kT) >= -1e-12


@pytest.mark.parametrize("ratio", [0.7, 1.3])
def test_secular_low_temperature_form(ratio):
    """The supplement's Eq. 210 at hbar omega / k_B T >> 1: T_0 T_E Pi(0) / (kappa omega) ~
    (T_E - T_0)(exp(-omega/T_E) - exp(-omega/T_0))."""
    kT = OMEGA / 10.0
    T0 = kT * ratio
    num = en.entropy_production(en.oscillator(30, OMEGA, TWO_PI * 0.25, KAPPA, kT, True),
                                en.gaussian_state(30, OMEGA / T0), kT)
    approx = KAPPA * OMEGA * (kT - T0) * (math.exp(-OMEGA / kT) - math.exp(-OMEGA / T0)) / (T0 * kT)
    assert abs(num / approx - 1.0) < 5e-3
