"""Pins of the Maxwell-Juttner loader oracle (Sect. 4, App. D, App. E).

Philox against its published known-answer vectors; the marginal and
conditional samples against their exact cumulative distributions (adaptive
quadrature, the closed-form conditional CDF); sample moments against the
closed forms of Table averages; and the naive particle-by-particle boost of
Sect. 4.2 against the same tests, which it must fail at T = mc^2, Gamma0
beta0 = sqrt(2) (the case of Fig. testJuttner).
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import mj


def test_philox_known_answer_vectors():
    """Philox-4x32-10 known-answer tests (Salmon et al. 2011, Random123)."""
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, exp in cases:
        out = mj.philox4x32([np.array([c], dtype=np.uint32) for c in ctr], key)
        assert tuple(int(o[0]) for o in out) == exp


def test_uniforms_are_open_unit_interval_and_uniform():
    w = mj.uniforms(12345, 1, np.arange(200000))
    assert w.shape == (6, 200000)
    assert w.min() > 0.0 and w.max() < 1.0
    for r in w:
        assert abs(r.mean() - 0.5) < 0.005
        assert abs(r.var() - 1.0 / 12.0) < 0.002


@pytest.mark.parametrize("theta,beta0", [(1.0, np.sqrt(2.0) / np.sqrt(3.0)), (0.1, 0.5), (0.01, 0.0),
                                         (10.0, 0.9)])
def test_marginal_pdf_normalised_and_inverse_exact(theta, beta0):
    tot, _ = integrate.quad(mj.marginal_pdf, -np.inf, np.inf, args=(theta, beta0), limit=400)
    assert abs(tot - 1.0) < 1e-9
    inv = mj.MarginalInverse(theta, beta0)
    w = np.array([1e-6, 0.01, 0.3, 0.5, 0.77, 0.99, 1 - 1e-6])
    y = inv(w)
    F = mj.marginal_cdf_quad(y, theta, beta0)
    assert np.allclose(F, w, rtol=1e-8, atol=1e-11), (F - w)


def _ks(sample_cdf_values):
    u = np.sort(sample_cdf_values)
    n = len(u)
    i = np.arange(1, n + 1)
    return max((i / n - u).max(), (u - (i - 1) / n).max())


def test_sampled_drift_component_passes_ks_and_naive_boost_fails():
    """T = mc^2, Gamma0 beta0 = sqrt(2) (Fig. testJuttner): the exact loader
    follows Eq. distr_y, the naive boost does not."""
    theta, b = 1.0, np.sqrt(2.0 / 3.0)   # Gamma0 beta0 = sqrt(2)
    n = 20000
    w = mj.uniforms(7, 0, np.arange(n))
    p = mj.sample_momenta(w[3], w[4], w[5], theta, [0.0, b, 0.0])
    crit = 1.63 / np.sqrt(n)   # 1 % level
    # exact CDF at a sorted subsample via quadrature (independent of the tables)
    idx = np.linspace(0, n - 1, 400).astype(int)
    ys = np.sort(p[1])
    F = mj.marginal_cdf_quad(ys[idx], theta, b)
    d_exact = np.abs(F - (idx + 0.5) / n).max()
    assert d_exact < crit
    pn = mj.naive_boost(w[3], w[4], w[5], theta, [0.0, b, 0.0])
    ysn = np.sort(pn[1])
    Fn = mj.marginal_cdf_quad(ysn[idx], theta, b)
    d_naive = np.abs(Fn - (idx + 0.5) / n).max()
    assert d_naive > 5 * crit, d_naive


def test_conditional_is_exact():
    """Given y, w' = l(a u)/l(a) must be uniform (closed-form conditional CDF)."""
    theta, b = 0.5, 0.6
    n = 20000
    w = mj.uniforms(9, 0, np.arange(n))
    y = mj.MarginalInverse(theta, b)(w[3])
    u = mj.conditional_u(y, w[4], theta, b)
    mu, G0 = 1 / theta, 1 / np.sqrt(1 - b * b)
    a = mu * G0 * np.sqrt(1 + y * y)
    l = lambda x: np.log1p(x) - x
    back = np.exp(l(a * u) - l(a))
    assert np.allclose(back, w[4], rtol=1e-10, atol=1e-14)
    assert np.all(u >= 1.0)
    assert _ks(back) < 1.63 / np.sqrt(n)
    # closed form with the lower Lambert-W branch where it is finite
    assert np.allclose(mj.conditional_u_lambertw(y, w[4], theta, b), u, rtol=1e-12)
    # large a (cold, fast drift): still finite and exact
    uu = mj.conditional_u(np.array([0.0, 5.0]), np.array([0.3, 1e-9]), 0.01, np.sqrt(8 / 9.0))
    aa = 100 * 3 * np.sqrt(1 + np.array([0.0, 25.0]))
    assert np.all(np.isfinite(uu))
    assert np.allclose(np.exp(l(aa * uu) - l(aa)), [0.3, 1e-9], rtol=1e-9)


@pytest.mark.parametrize("theta,beta0", [(0.1, 0.0), (1.0, 0.5), (0.3, 0.9), (5.0, 0.3)])
def test_moments_match_table_averages(theta, beta0):
    n = 200000
    w = mj.uniforms(3, 2, np.arange(n))
    p = mj.sample_momenta(w[3], w[4], w[5], theta, [0.0, 0.0, beta0])
    g = np.sqrt(1 + (p ** 2).sum(0))
    v = p / g
    m = mj.moments(theta, beta0)
    est = {"gamma": g, "gamma_v_par": p[2], "pv_perp": p[0] * v[0], "pv_par": p[2] * v[2]}
    for k, x in est.items():
        se = x.std() / np.sqrt(n)
        assert abs(x.mean() - m[k]) < 4 * se + 1e-12, (k, x.mean(), m[k], se)
    # isotropy of the perpendicular plane and zero mean perpendicular momentum
    assert abs(p[0].mean()) < 4 * p[0].std() / np.sqrt(n)
    assert abs(p[1].mean()) < 4 * p[1].std() / np.sqrt(n)


def test_rest_frame_temperature_is_theta():
    """<u . v>/3 = Theta for the rest-frame distribution (Table averages, <gamma beta^2> = 3 Theta)."""
    theta = 0.4
    n = 200000
    w = mj.uniforms(5, 0, np.arange(n))
    p = mj.sample_momenta(w[3], w[4], w[5], theta, np.zeros(3))
    g = np.sqrt(1 + (p ** 2).sum(0))
    T = ((p ** 2).sum(0) / g).mean() / 3
    assert abs(T - theta) < 4 * ((p ** 2).sum(0) / g / 3).std() / np.sqrt(n)


def test_harris_positions_follow_sech2():
    nx, L, x0 = 64, 5.0, 32.0
    n = 100000
    w = mj.uniforms(11, 0, np.arange(n))
    pos = mj.positions_harris(w, nx, 8, 1, 2, L, x0)
    assert pos[0].min() >= 0 and pos[0].max() <= nx
    ta, tb = np.tanh(-x0 / L), np.tanh((nx - x0) / L)
    cdf = (np.tanh((pos[0] - x0) / L) - ta) / (tb - ta)
    assert _ks(cdf) < 1.63 / np.sqrt(n)
