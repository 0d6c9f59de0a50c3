"""Pins of the closed-form physics relations against the numbers printed in the
paper's tables (fixtures in tests/golden/, each with its citation)."""
import os

import numpy as np

from oracle import theory

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#", ndmin=2)


def test_harris_relations_reproduce_table_tearing():
    for theta, wce, GU, L in _table("tearing_table.txt"):
        w, l = theory.harris_from_theta_GU(theta, GU)
        assert abs(w - wce) <= 0.02 * wce + 0.005, (theta, w, wce)
        assert abs(l - L) <= 0.02 * L, (theta, l, L)


def test_filamentation_rate_reproduces_table_two_stream():
    for beta0, tau in _table("filamentation_table.txt"):
        t = theory.tau_filamentation_pair(beta0)
        assert abs(t - tau) <= 0.006, (beta0, t, tau)


def test_electron_beam_variant_is_sqrt2_slower():
    b = np.sqrt(1 - 1 / 9.0)   # Gamma0 = 3
    assert np.isclose(theory.tau_filamentation_electron_beams(b), np.sqrt(2) * theory.tau_filamentation_pair(b))
    assert abs(theory.tau_filamentation_electron_beams(b) - 0.2924) < 5e-4


def test_cold_mode_formulas_reproduce_table_cold_modes():
    """The paper's theory columns are the heavy-ion formulas; its measured
    peaks are the cut-offs with the ions' finite mass (m_i/m_e = 49), to the
    table's two printed digits (spectral resolution 0.01 omega_pe)."""
    for wce, w_par, w_l, w_r, th_p, th_l, th_r in _table("cold_modes_table.txt"):
        assert abs(theory.cold_plasma_frequency(49.0) - th_p) <= 5e-4
        hl, hr = theory.cold_cutoffs_heavy_ions(wce)
        assert abs(hl - th_l) <= 5e-3 and abs(hr - th_r) <= 5e-3, (wce, hl, hr)
        ml, mr = theory.cold_cutoffs_two_species(wce, 49.0)
        assert abs(ml - w_l) <= 0.011 and abs(mr - w_r) <= 0.021, (wce, ml, mr)
        assert abs(theory.cold_plasma_frequency(49.0) - w_par) <= 0.005


def test_two_species_cutoffs_tend_to_the_heavy_ion_formulas():
    for wce in (0.3, 1.0, 3.0):
        a = theory.cold_cutoffs_two_species(wce, 1e9)
        b = theory.cold_cutoffs_heavy_ions(wce)
        assert np.allclose(a, b, rtol=1e-7)
        # R(omega_R) = 0 and L(omega_L) = 0 with the ions' terms
        mu = 49.0
        wl, wr = theory.cold_cutoffs_two_species(wce, mu)
        R = 1 - 1 / (wr * (wr - wce)) - (1 / mu) / (wr * (wr + wce / mu))
        L = 1 - 1 / (wl * (wl + wce)) - (1 / mu) / (wl * (wl - wce / mu))
        assert abs(R) < 1e-10 and abs(L) < 1e-10


def test_thermal_mode_branches_meet_at_the_plasma_frequency():
    """Sect. 3.1.1: both unmagnetized branches start at omega_P (1.010 omega_pe for
    m_i/m_e = 49, as printed), the Langmuir branch rises as 3 k^2 lambda_D^2 / 2
    at small k, and the transverse branch tends to the light line k c."""
    assert abs(theory.transverse_wave(0.0, 49.0) - 1.010) < 5e-4
    assert abs(theory.langmuir_wave(0.0, 49.0) - 1.010) < 5e-4
    wp = theory.cold_plasma_frequency(49.0)
    assert abs(theory.langmuir_wave(1e-3, 49.0) / wp - 1 - 1.5e-6) < 1e-10
    assert abs(theory.transverse_wave(1e4, 49.0) / 1e4 - 1) < 1e-8
