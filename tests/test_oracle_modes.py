"""Oracle pins from the linear theory of three plasma modes, run by the FP64
CPU oracle itself on small boxes (no GPU):

- the cold filamentation instability of two counter-streaming electron beams
  on a positron background (Sect. 3.2.1), at a finite wavenumber, against the
  cold two-fluid growth rate whose k -> infinity limit is the paper's formula;
- the transverse electromagnetic branch omega^2 = omega_P^2 + k^2 c^2 of a
  cold pair plasma (Sect. 3.1.1);
- the thermal Langmuir branch omega^2 = omega_P^2 (1 + 3 k^2 lambda_D^2) of an
  electron-ion plasma with v_th = 0.1 c (Sect. 3.1.1).

Each run starts from a quiet state: particles on a regular lattice of points
per cell, cold, or thermal with every momentum paired with its opposite at the
same point, so that the seeded mode stands far above the particle noise.  The
seeds perturb b_y (filamentation), e_y (transverse) or u_x (Langmuir) with
cos(k x) for chosen box modes k.  These pins tie the oracle's current coupling
alpha, its Boris step, its deposit and its Yee update to the physics together:
a wrong alpha moves omega_P by sqrt(2) and the growth rate by 20 % or more.
"""
import numpy as np
from scipy.optimize import curve_fit

import oracle
from oracle import mj, theory


def _lattice(nx, ny, per_axis):
    """per_axis^2 points per cell at the centres of a regular sub-lattice, (3, n)."""
    off = (np.arange(per_axis) + 0.5) / per_axis
    i, j, a, b = np.meshgrid(np.arange(nx), np.arange(ny), off, off, indexing="ij")
    pos = np.zeros((3, i.size))
    pos[0] = (i + a).reshape(-1)
    pos[1] = (j + b).reshape(-1)
    return pos


def _frequency(sig, t, w_guess):
    """Angular frequency of a damped cosine a exp(-g t) cos(w t + ph) + c fitted
    to sig(t) by least squares (best of several starting phases); returns (w, g)."""
    f = lambda t, a, w, ph, g, c: a * np.exp(-g * t) * np.cos(w * t + ph) + c
    best = None
    for ph in np.linspace(0.0, 2 * np.pi, 8, endpoint=False):
        try:
            p, _ = curve_fit(f, t, sig, p0=[np.abs(sig).max(), w_guess, ph, 0.0, 0.0], maxfev=20000)
        except RuntimeError:
            continue
        r = ((f(t, *p) - sig) ** 2).sum()
        if best is None or r < best[0]:
            best = (r, p)
    return abs(best[1][1]), best[1][3]


def test_cold_rate_tends_to_the_papers_formula():
    """k -> infinity: delta = sqrt(sum omega_ps^2 beta_s^2 / gamma_s), i.e. the
    e-folding time tau = (1/2 pi) sqrt(Gamma0/2) / beta0 T_pe of the paper's
    formula for pair beams (pinned to Table two_stream in test_oracle_theory),
    and sqrt(2) slower for two electron beams on positrons at rest.  The rate
    grows with k and is below the limit at every finite k."""
    for G0 in (1.5, 3.0, 10.0):
        b0 = np.sqrt(1 - 1 / G0 ** 2)
        pair = [(0.5, b0, G0), (0.5, b0, G0), (0.5, b0, G0), (0.5, b0, G0)]   # e+ and e- in both beams
        ebeams = [(0.5, b0, G0), (0.5, b0, G0), (1.0, 0.0, 1.0)]
        assert np.isclose(theory.filamentation_rate_cold(1e6, pair), 1 / (2 * np.pi * theory.tau_filamentation_pair(b0)),
                          rtol=1e-8)
        assert np.isclose(theory.filamentation_rate_cold(1e6, ebeams),
                          1 / (2 * np.pi * theory.tau_filamentation_electron_beams(b0)), rtol=1e-8)
        ks = np.array([0.3, 1.0, 3.0, 10.0])
        r = np.array([theory.filamentation_rate_cold(k, ebeams) for k in ks])
        assert np.all(np.diff(r) > 0) and np.all(r < theory.filamentation_rate_cold(1e6, ebeams))
        # the root solves the quartic
        for k, d in zip(ks, r):
            A = sum(w / g ** 3 for w, b, g in ebeams)
            C = sum(w * b * b / g for w, b, g in ebeams)
            assert abs(d ** 4 + (k * k + A) * d * d - k * k * C) < 1e-12


def test_oracle_cold_filamentation_grows_at_the_cold_rate():
    """Two cold electron beams (Gamma0 = 3, along +-z, half the electron density
    each) on positrons at rest, 2D3V, 64 x 4 cells, 8 cells per c/omega_pe, 4
    particles per cell per beam on a lattice.  b_y is seeded at box modes 2 and
    4 (k c/omega_pe = 1.57, 3.14).  After the oscillating part of the seed has
    decayed relative to the growing part, ln |b_y(k)| grows at the rate of
    the cold dispersion relation (0.444 and 0.512 omega_pe) within 3 % (the
    oracle measures 0.444 and 0.502: at k dx = 0.39 the node averaging and
    the linear weights of gather and deposit lower the coupling by about 2 %)."""
    nx, ny, n_x, dt, G0 = 64, 4, 8.0, 0.5, 3.0
    b0 = np.sqrt(1 - 1 / G0 ** 2)
    pos = _lattice(nx, ny, 2)
    n = pos.shape[1]
    st = oracle.State.empty(2, nx, ny, 1, dt, n_x, rho_sp0=16.0)   # 4 + 4 electrons and 8 positrons per cell
    for sgn in (1.0, -1.0):
        u = np.zeros((3, n))
        u[2] = sgn * G0 * b0
        st.species.append(oracle.Species(pos.copy(), u, -1.0, 1.0))
    st.species.append(oracle.Species(np.ascontiguousarray(np.concatenate([pos, pos], axis=1)), np.zeros((3, 2 * n)),
                                     1.0, 1.0))
    modes = (2, 4)
    xb = np.arange(nx) + 0.5                      # b_y sits at (i+1/2, j, k+1/2)
    eps = 1e-7
    st.b[1][0] = eps * sum(np.cos(2 * np.pi * m * xb / nx) for m in modes)[None, :]
    nsteps = 300
    amp = np.zeros((len(modes), nsteps))
    for s in range(nsteps):
        by = st.b[1][0].mean(0)
        for q, m in enumerate(modes):
            amp[q, s] = abs((by * np.exp(-2j * np.pi * m * xb / nx)).sum()) * 2 / nx
        oracle.step(st)
    t = np.arange(nsteps) * dt / n_x                # in 1/omega_pe
    pops = [(0.5, b0, G0), (0.5, b0, G0), (1.0, 0.0, 1.0)]
    for q, m in enumerate(modes):
        la = np.log(amp[q] / eps)
        sel = (t > 6.0) & (la > np.log(20.0)) & (la < np.log(3e3))
        assert sel.sum() > 40, (m, sel.sum())
        rate = np.polyfit(t[sel], la[sel], 1)[0]
        delta = theory.filamentation_rate_cold(2 * np.pi * m / nx * n_x, pops)
        print("mode %d: oracle %.4f, cold theory %.4f omega_pe" % (m, rate, delta))
        assert abs(rate / delta - 1) < 0.03, (m, rate, delta)


def test_oracle_transverse_branch_of_a_cold_pair_plasma():
    """Cold pair plasma, 2D3V, 64 x 2 cells, 10 cells per c/omega_pe, 4
    particles per cell per species on a lattice.  e_y seeded uniform (k = 0)
    and at box modes 1 and 2 (k c/omega_pe = 0.98, 1.96).  The k = 0 field
    oscillates at omega_P = sqrt(2) omega_pe (within 0.5 %), and
    (omega_k^2 - omega_0^2) / (k c)^2 = 1 within 2 %."""
    nx, ny, n_x, dt = 64, 2, 10.0, 0.5
    pos = _lattice(nx, ny, 2)
    n = pos.shape[1]
    st = oracle.State.empty(2, nx, ny, 1, dt, n_x, rho_sp0=8.0)
    st.species.append(oracle.Species(pos.copy(), np.zeros((3, n)), -1.0, 1.0))
    st.species.append(oracle.Species(pos.copy(), np.zeros((3, n)), 1.0, 1.0))
    x = np.arange(nx)                               # e_y sits at (i, j+1/2)
    ks = [2 * np.pi * m / nx for m in (1, 2)]
    st.e[1][0] = 1e-3 * (1.0 + sum(np.cos(k * x) for k in ks))[None, :]
    nsteps = 700
    sig = np.zeros((3, nsteps))
    for s in range(nsteps):
        ey = st.e[1][0].mean(0)
        sig[0, s] = ey.mean()
        for q, k in enumerate(ks):
            sig[1 + q, s] = (ey * np.cos(k * x)).sum() * 2 / nx
        oracle.step(st)
    t = np.arange(nsteps) * dt / n_x
    wP = np.sqrt(2.0)
    w0, _ = _frequency(sig[0], t, wP)
    assert abs(w0 / wP - 1) < 0.005, w0
    for q, k in enumerate(ks):
        kc = k * n_x
        wk, _ = _frequency(sig[1 + q], t, np.sqrt(wP ** 2 + kc * kc))
        r = (wk ** 2 - w0 ** 2) / kc ** 2
        print("k c/omega_pe %.3f: omega %.4f, (omega^2 - omega_0^2)/k^2c^2 = %.4f" % (kc, wk, r))
        assert abs(r - 1) < 0.02, (kc, r)


def test_oracle_langmuir_branch_of_a_thermal_plasma():
    """Electron-ion plasma (m_i/m_e = 49, ions cold), electrons Maxwell-Juttner
    at theta = 0.01 (v_th = 0.1 c), 10 cells per c/omega_pe so lambda_D is one
    cell, 40 x 2 cells, 128 electrons per cell: 64 lattice points, each with a
    momentum from the oracle's exact loader and its opposite.  u_x is kicked
    by 0.02 (1 + cos k1 x + cos k2 x) at box modes 1 and 2 (k lambda_D = 0.155,
    0.31).  The thermal shift of each mode, omega_k^2 - omega_0^2 with omega_0
    the measured k = 0 frequency, equals 3 k^2 lambda_D^2 omega_0^2 within
    15 % (lambda_D from the loaded <v_x^2>); omega_0 lies within 2 % below
    omega_P = (1 + m_e/m_i)^1/2 omega_pe (the thermal plasma's cutoff is
    lowered by the relativistic mass increase)."""
    nx, ny, n_x, dt, theta, mu = 40, 2, 10.0, 0.5, 0.01, 49.0
    pos = _lattice(nx, ny, 8)
    nh = pos.shape[1]
    w = mj.uniforms(3, 0, np.arange(nh))
    u = mj.sample_momenta(w[3], w[4], w[5], theta, np.zeros(3))
    pos_e = np.ascontiguousarray(np.concatenate([pos, pos], axis=1))
    u_e = np.concatenate([u, -u], axis=1)
    gam = np.sqrt(1 + (u_e ** 2).sum(0))
    lam = np.sqrt(((u_e[0] / gam) ** 2).mean()) * n_x      # lambda_D in cells
    ks = [2 * np.pi * m / nx for m in (1, 2)]
    u_e[0] += 0.02 * (1.0 + sum(np.cos(k * pos_e[0]) for k in ks))
    ne = pos_e.shape[1]
    st = oracle.State.empty(2, nx, ny, 1, dt, n_x, rho_sp0=2.0 * ne / (nx * ny))
    st.species.append(oracle.Species(pos_e, np.ascontiguousarray(u_e), -1.0, 1.0))
    st.species.append(oracle.Species(pos_e.copy(), np.zeros((3, ne)), 1.0, mu))
    x = np.arange(nx) + 0.5                         # e_x sits at (i+1/2, j)
    nsteps = 600
    sig = np.zeros((3, nsteps))
    for s in range(nsteps):
        ex = st.e[0][0].mean(0)
        sig[0, s] = ex.mean()
        for q, k in enumerate(ks):
            sig[1 + q, s] = (ex * np.cos(k * x)).sum() * 2 / nx
        oracle.step(st)
    t = np.arange(nsteps) * dt / n_x
    wP = theory.cold_plasma_frequency(mu)
    w0, _ = _frequency(sig[0], t, wP)
    assert 0.98 * wP < w0 < wP, (w0, wP)
    for q, k in enumerate(ks):
        kl = k * lam
        wk, _ = _frequency(sig[1 + q], t, theory.langmuir_wave(kl, mu))
        r = (wk ** 2 - w0 ** 2) / (3 * kl * kl * w0 * w0)
        print("k lambda_D %.3f: omega %.4f omega_pe, thermal shift / 3 k^2 lambda_D^2 omega_0^2 = %.3f" % (kl, wk, r))
        assert abs(r - 1) < 0.15, (kl, r)
