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
