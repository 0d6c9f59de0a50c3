"""Long-run physics on the GPU paths (Sect. 3.2.1, Sect. 5).

Filamentation of two counter-streaming electron beams (Gamma0 = 3, theta =
0.01) on a positron background at rest, 2D3V with the beams along the
ignorable z axis, as in the paper's filamentation study: the magnetic energy
grows as exp(2 delta t) in the linear phase, with the cold k_perp -> infinity
rate delta = beta0 omega_pe / sqrt(Gamma0) (oracle/theory.py).  The mixed path
must reproduce the FP64 path's measured rate within 5 %, the FP64 GPU path the
oracle's within 2 %, and all of them the cold rate within 20 % (the paper
finds 6-14 % at its resolution; finite temperature and grid lower the rate).
A thermal pair plasma checks the energy drift of both paths.
"""
import numpy as np
import pytest

import oracle
import oracle.theory as theory
import paper_1308_5892_gb300 as pic

pytestmark = pytest.mark.gpu

NX, NY, PPC, N_X, DT, STEPS = 64, 64, 8, 4.0, 0.5, 200
BETA0 = np.sqrt(8.0 / 9.0)   # Gamma0 = 3


def _desc():
    n = PPC * NX * NY
    return pic.run_desc(2, NX, NY, 1, N_X, 4.0 * PPC, DT, [(-1.0, 1.0, n), (1.0, 1.0, n), (-1.0, 1.0, n),
                                                           (1.0, 1.0, n)])


def _load(ctx):
    # each electron beam with its own positrons on top of it, so rho = 0 at t = 0
    ctx.load_maxwell_juttner(0, 0, PPC, 0.01, (0.0, 0.0, BETA0), seed=11)
    ctx.load_maxwell_juttner(0, 1, PPC, 0.01, (0.0, 0.0, 0.0), colocate_with=0, seed=12)
    ctx.load_maxwell_juttner(0, 2, PPC, 0.01, (0.0, 0.0, -BETA0), seed=13)
    ctx.load_maxwell_juttner(0, 3, PPC, 0.01, (0.0, 0.0, 0.0), colocate_with=2, seed=14)


def _growth_rate(eb, dt, window=24, skip=10):
    """Largest least-squares slope of log(E_B) over `window` consecutive
    samples, divided by 2: the field growth rate delta (per unit time).  The
    first `skip` samples (fields start at zero and fill up to the noise floor)
    are left out."""
    y = np.log(eb[skip:])
    t = (np.arange(len(y)) + skip) * dt
    best = -np.inf
    for i in range(len(y) - window):
        best = max(best, np.polyfit(t[i:i + window], y[i:i + window], 1)[0])
    return 0.5 * best


@pytest.fixture(scope="module")
def runs():
    out = {}
    for name, prec in (("fp64", pic.PIC_FP64), ("mixed", pic.PIC_MIXED)):
        with pic.Context([_desc()], precision=prec) as ctx:
            _load(ctx)
            if name == "fp64":
                f0, p0, _ = ctx.get_state(0)
                out["initial"] = (f0, p0)
            ctx.step(STEPS)
            out[name] = ctx.energy_history(0)
    return out


def test_filamentation_growth_rate_mixed_matches_fp64(runs):
    """The magnetic energy of the whole box grows at the same rate in both paths."""
    d64 = _growth_rate(runs["fp64"][:, 2], DT)
    dmx = _growth_rate(runs["mixed"][:, 2], DT)
    # the linear phase is resolved: e-folds of the magnetic energy above the noise floor
    assert np.log(runs["fp64"][:, 2].max() / runs["fp64"][10, 2]) > 4
    print("growth rates of E_B: fp64 %.5f mixed %.5f" % (d64, dmx))
    assert abs(dmx / d64 - 1) <= 0.05, (dmx, d64)


def _linear_phase_rate(e, dt, floor_at=(20, 40)):
    """Growth rate of one mode's energy over its linear phase: from the first
    time it exceeds 10x its noise floor (median of samples floor_at) to the
    first time it reaches 10 % of its maximum; None without 2 decades of growth."""
    floor, peak = np.median(e[floor_at[0]:floor_at[1]]), e.max()
    if peak < 100 * floor:
        return None
    i1 = int(np.argmax(e > 10 * floor))
    i2 = int(np.argmax(e > 0.1 * peak))
    if i2 - i1 < 8:
        return None
    t = np.arange(i1, i2) * dt
    return 0.5 * np.polyfit(t, np.log(e[i1:i2]), 1)[0]


def _shell_energy(b, nshell):
    """In-plane magnetic energy |b_x(k)|^2 + |b_y(k)|^2 summed over shells of |k| (2D)."""
    ny, nx = b.shape[-2:]
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    kk = np.sqrt(kx * kx + ky * ky) / 0.5           # 1 at the grid cutoff
    idx = np.minimum((kk * nshell).astype(int), nshell - 1)
    e = np.abs(np.fft.fft2(b[0, 0])) ** 2 + np.abs(np.fft.fft2(b[1, 0])) ** 2
    return np.bincount(idx.ravel(), weights=e.ravel(), minlength=nshell)


def test_filamentation_fastest_mode_grows_at_the_cold_rate():
    """Sect. 3.2.1: the fastest-growing Fourier modes grow at the cold
    k_perp -> infinity rate delta = beta0 omega_pe / sqrt(Gamma0) within 20 %
    (the paper measures 6-14 % at n_x = 20); finite temperature and grid
    lower it.  8 cells per c / omega_pe, 16 skin depths, both paths."""
    nx, n_x, ppc, steps, nshell = 128, 8.0, 8, 240, 16
    n = ppc * nx * nx
    d = pic.run_desc(2, nx, nx, 1, n_x, 4.0 * ppc, DT, [(-1.0, 1.0, n), (1.0, 1.0, n), (-1.0, 1.0, n),
                                                         (1.0, 1.0, n)])
    omega_pe = 1.0 / n_x          # all electrons; n_x cells per c / omega_pe
    d_th = 1.0 / (theory.tau_filamentation_electron_beams(BETA0) * 2 * np.pi / omega_pe)
    rates = {}
    for name, prec in (("fp64", pic.PIC_FP64), ("mixed", pic.PIC_MIXED)):
        with pic.Context([d], precision=prec) as ctx:
            ctx.load_maxwell_juttner(0, 0, ppc, 0.01, (0.0, 0.0, BETA0), seed=31)
            ctx.load_maxwell_juttner(0, 1, ppc, 0.01, (0.0, 0.0, 0.0), colocate_with=0, seed=32)
            ctx.load_maxwell_juttner(0, 2, ppc, 0.01, (0.0, 0.0, -BETA0), seed=33)
            ctx.load_maxwell_juttner(0, 3, ppc, 0.01, (0.0, 0.0, 0.0), colocate_with=2, seed=34)
            shells = np.zeros((steps, nshell))
            for k in range(steps):
                ctx.step(1)
                f, _, _ = ctx.get_state(0, fields_only=True)
                shells[k] = _shell_energy(f[3:5], nshell)
        rates[name] = max(r for r in (_linear_phase_rate(shells[:, q], DT) for q in range(1, nshell)) if r)
    print("fastest-shell growth rates: fp64 %.5f mixed %.5f cold theory %.5f" % (rates["fp64"], rates["mixed"], d_th))
    assert abs(rates["mixed"] / rates["fp64"] - 1) <= 0.05, rates
    for name in rates:
        assert abs(rates[name] / d_th - 1) <= 0.20, (name, rates[name], d_th)


def test_filamentation_at_the_configured_size_grows_at_the_cold_rate():
    """The filamentation workload as configured (Sect. 3.2.1, Table two_stream's
    resolution): 1024^2 cells, 20 cells per c/omega_pe (51.2 skin depths),
    electrons 25 + 25 per cell in the two beams (Gamma0 = 3, theta = 0.01),
    positrons 50 per cell at rest (theta = 0.01) on the electrons, 2000 steps
    of the mixed path (7.96 plasma periods).  The fastest-growing shell of
    in-plane magnetic modes grows within 15 % of the cold rate beta0 omega_pe /
    sqrt(Gamma0), i.e. its e-folding time is within 15 % of 0.292 T_pe (the
    paper measures 6-14 % at this resolution; measured here 0.86 of the rate,
    stable between 0.85 and 0.88 over reasonable fit windows: the thermal
    spread of the beams lowers the fastest rate below the cold limit).  The
    long-wavelength shells match the cold rate at their own k within 10 %
    (measured 0.91-0.93).  The box's magnetic energy saturates within the run
    and charge stays conserved to 1e-6 of max rho."""
    nx, n_x, ppc, steps, every, nshell = 1024, 20.0, 25, 2000, 4, 64
    n = ppc * nx * nx
    d = pic.run_desc(2, nx, nx, 1, n_x, 4.0 * ppc, DT, [(-1.0, 1.0, n), (1.0, 1.0, 2 * n), (-1.0, 1.0, n)])
    omega_pe = 1.0 / n_x          # all electrons (50 per cell = rho_sp0 / 2)
    d_th = BETA0 * omega_pe / np.sqrt(3.0)
    with pic.Context([d], precision=pic.PIC_MIXED) as ctx:
        ctx.load_maxwell_juttner(0, 0, ppc, 0.01, (0.0, 0.0, BETA0), seed=3)
        ctx.load_maxwell_juttner(0, 2, ppc, 0.01, (0.0, 0.0, -BETA0), seed=4)
        # positrons at rest on top of both beams (species 1 holds 2 ppc: loaded from beam 1, then its
        # second half re-seated on beam 2 through a state round trip)
        ctx.load_maxwell_juttner(0, 1, 2 * ppc, 0.01, (0.0, 0.0, 0.0), seed=5)
        f, p, _ = ctx.get_state(0)
        p[1][:3, :n] = p[0][:3]
        p[1][:3, n:] = p[2][:3]
        ctx.set_state(0, f, p)
        shells = []
        for k in range(0, 1400, every):
            ctx.step(every)
            fb, _, _ = ctx.get_state(0, fields_only=True)
            shells.append(_shell_energy(fb[3:5], nshell))
        ctx.step(steps - 1400)
        dg = ctx.diagnostics(0)
        hist = ctx.energy_history(0)
    shells = np.array(shells)
    rates = {q: _linear_phase_rate(shells[:, q], every * DT, floor_at=(5, 10)) for q in range(1, nshell)}
    best = max(r for r in rates.values() if r)
    print("configured filamentation: fastest-shell rate %.5f, cold rate %.5f (ratio %.3f); tau = %.3f T_pe" %
          (best, d_th, best / d_th, 1.0 / (2 * np.pi * best / omega_pe)))
    assert abs(best / d_th - 1) <= 0.15, (best, d_th)
    # the long-wavelength shells (k c/omega_pe < 3) follow the cold rate at their own k (finite-k
    # cold two-fluid relation) within 10 %: thermal spread matters only at larger k
    pops = [(0.5, BETA0, 3.0), (0.5, BETA0, 3.0), (1.0, 0.0, 1.0)]
    for q in (1, 2, 3):
        kc = (q + 0.5) / nshell * np.pi * n_x          # shell centre, k c / omega_pe
        d_k = theory.filamentation_rate_cold(kc, pops) * omega_pe
        print("shell %d (k c/omega_pe = %.2f): rate %.5f, finite-k cold rate %.5f (ratio %.3f)" %
              (q, kc, rates[q], d_k, rates[q] / d_k))
        assert abs(rates[q] / d_k - 1) <= 0.10, (q, rates[q], d_k)
    eb = hist[:, 2]
    assert eb.max() > 1e3 * eb[20]                                # grew by more than three decades
    late = np.log(eb[-1] / eb[-400]) / (2 * 400 * DT)             # field growth rate over the last 400 steps
    assert late < 0.3 * d_th, late                                # ... and saturated
    assert dg["gauss_max"] <= 1e-6 * dg["rho_max"], dg


def test_filamentation_growth_rate_fp64_matches_oracle(runs):
    f0, p0 = runs["initial"]
    d = _desc()
    st = oracle.State.empty(2, NX, NY, 1, DT, N_X, 4.0 * PPC)
    st.e[:] = f0[:3]
    st.b[:] = f0[3:]
    for s, p in enumerate(p0):
        st.species.append(oracle.Species(np.ascontiguousarray(p[:3]), np.ascontiguousarray(p[3:]),
                                         d.species[s].q_over_e, d.species[s].m_over_me))
    eb = np.zeros(STEPS)
    for n in range(STEPS):
        oracle.step(st)
        eb[n] = oracle.energies(st)["field_b"].sum()
    d_or = _growth_rate(eb, DT)
    d64 = _growth_rate(runs["fp64"][:, 2], DT)
    print("growth rates: fp64 %.5f oracle %.5f" % (d64, d_or))
    assert abs(d64 / d_or - 1) <= 0.02, (d64, d_or)


def _drift_rate(etot, dt):
    """Least-squares slope of E_tot(t) / E_tot(0) per unit time."""
    t = np.arange(len(etot)) * dt
    return np.polyfit(t, etot / etot[0], 1)[0]


def test_thermal_plasma_energy_drift_scales_as_one_over_rho_sp_in_both_paths():
    """Energy conservation of a thermal pair plasma (Sect. 2.4): the total
    energy drifts linearly in time at a rate proportional to 1 / rho_sp.  Both
    paths must show the same drift (within 15 %) and a drift rate that falls
    by 2.5x to 6x when the particles per cell grow 4x."""
    rates = {}
    for ppc in (8, 32):
        n = ppc * 48 * 48
        d = pic.run_desc(2, 48, 48, 1, 3.0, 2.0 * ppc, 0.5, [(-1.0, 1.0, n), (1.0, 1.0, n)])
        for name, prec in (("fp64", pic.PIC_FP64), ("mixed", pic.PIC_MIXED)):
            with pic.Context([d], precision=prec) as ctx:
                ctx.load_maxwell_juttner(0, 0, ppc, 0.1, seed=21)
                ctx.load_maxwell_juttner(0, 1, ppc, 0.1, colocate_with=0, seed=22)
                ctx.step(200)
                rates[name, ppc] = _drift_rate(ctx.energy_history(0)[:, 3], 0.5)
    print("energy drift rates per unit time:", rates)
    for ppc in (8, 32):
        assert abs(rates["mixed", ppc] / rates["fp64", ppc] - 1) <= 0.15, (ppc, rates)
    for name in ("fp64", "mixed"):
        ratio = rates[name, 8] / rates[name, 32]
        assert 2.5 <= ratio <= 6.0, (name, ratio)


def _mj_cutoff_factor(theta):
    """<gamma^-1 (1 - beta^2 / 3)> over a Maxwell-Juttner distribution at rest,
    by quadrature in u = gamma beta: weight u^2 exp(-gamma / theta)."""
    from scipy import integrate
    w = lambda u: u * u * np.exp(-(np.sqrt(1 + u * u) - 1) / theta)
    f = lambda u: w(u) / np.sqrt(1 + u * u) * (1 - (u * u / (1 + u * u)) / 3)
    top = integrate.quad(f, 0, np.inf, limit=400)[0]
    bot = integrate.quad(w, 0, np.inf, limit=400)[0]
    return top / bot


def test_thermal_plasma_k0_spectrum_peaks_at_the_relativistic_cutoff():
    """Sect. 3.1: the k = 0 electric field of a thermal pair plasma oscillates
    at the plasma cutoff, omega_cut^2 = omega_P^2 <gamma^-1 (1 - beta^2/3)> with
    omega_P^2 = 2 omega_pe^2 for pairs (relativistic correction of the paper's
    omega_P).  Configuration 1: 64^2, theta = 0.1, n_x = theta^-1/2 (dx = Debye
    length), 16 ppc per species, dt = 0.5, run over 60 plasma periods; the peak
    of |FFT_t <e_x>|^2 must fall within 2 % of omega_cut in both paths, and the
    two paths within two frequency bins of each other (the peak of a noise-driven
    spectrum moves by a bin between realisations)."""
    theta, ppc, nsteps, dt = 0.1, 16, 2400, 0.5
    n_x = theta ** -0.5
    n = ppc * 64 * 64
    d = pic.run_desc(2, 64, 64, 1, n_x, 2.0 * ppc, dt, [(-1.0, 1.0, n), (1.0, 1.0, n)])
    omega_cut = np.sqrt(2.0) / n_x * np.sqrt(_mj_cutoff_factor(theta))
    peaks = {}
    for name, prec in (("fp64", pic.PIC_FP64), ("mixed", pic.PIC_MIXED)):
        with pic.Context([d], precision=prec) as ctx:
            ctx.load_maxwell_juttner(0, 0, ppc, theta, seed=1)
            ctx.load_maxwell_juttner(0, 1, ppc, theta, colocate_with=0, seed=2)
            ex = np.zeros(nsteps)
            for k in range(nsteps):
                ctx.step(1)
                f, _, _ = ctx.get_state(0, fields_only=True)
                ex[k] = f[0].mean()
        spec = np.abs(np.fft.rfft((ex - ex.mean()) * np.hanning(nsteps))) ** 2
        omega = 2 * np.pi * np.fft.rfftfreq(nsteps, dt)
        peaks[name] = omega[1 + np.argmax(spec[1:])]
    dw = 2 * np.pi / (nsteps * dt)
    print("k=0 peak: fp64 %.4f mixed %.4f theory %.4f (bin %.4f)" % (peaks["fp64"], peaks["mixed"], omega_cut, dw))
    for name, w in peaks.items():
        assert abs(w / omega_cut - 1) <= 0.02, (name, w, omega_cut)
    assert abs(peaks["mixed"] - peaks["fp64"]) <= 2 * dw + 1e-12


def test_harris_sheet_tearing_grows_at_the_same_rate_in_both_paths():
    """Config 5 (Sect. 3.4, App. C): a relativistic pair Harris sheet between
    conducting walls, Theta = 1 with the Table tearing relations (omega_ce /
    omega_pe = 1.82, Gamma U = 0.68, L = 1.62 d_e), loaded by the library's
    Harris profile with drifting Maxwell-Juttner beams; the current is along the
    ignorable z, B_y(x) = B0 tanh((x - x0)/L).  The tearing mode (k along y)
    makes b_x grow; its energy must grow at the same rate in the FP64 and the
    mixed path (within 10 %), over a linear phase of at least two decades."""
    theta, GU, wce, l_over_de = 1.0, 0.68, 1.82, 1.62
    n_x, ppc, nx, ny, dt, nsteps = 4.0, 16, 128, 256, 0.5, 1600
    L, x0 = l_over_de * n_x, nx / 2.0
    beta = GU / np.sqrt(1.0 + GU * GU)
    b0 = wce / n_x                                    # omega_ce in units of c / X0 with X0 = d_e / n_x
    cap = int(ppc * 2.2 * L * ny) + 1024
    d = pic.run_desc(2, nx, ny, 1, n_x, 2.0 * ppc, dt, [(-1.0, 1.0, cap), (1.0, 1.0, cap)], bc=(1, 0, 0))
    rates = {}
    for name, prec in (("fp64", pic.PIC_FP64), ("mixed", pic.PIC_MIXED)):
        with pic.Context([d], precision=prec) as ctx:
            # electrons drift along -z, positrons along +z: J_z > 0 at the centre, dB_y/dx = J_z
            ctx.load_maxwell_juttner(0, 0, ppc, theta, (0.0, 0.0, -beta), profile=pic.PIC_PROFILE_HARRIS,
                                     profile_params=(L, x0), seed=41)
            ctx.load_maxwell_juttner(0, 1, ppc, theta, (0.0, 0.0, beta), profile=pic.PIC_PROFILE_HARRIS,
                                     profile_params=(L, x0), colocate_with=0, seed=42)
            f, p, _ = ctx.get_state(0)
            i = np.arange(nx)
            f[4, 0, :, :] = b0 * np.tanh((i[None, :] + 0.5 - x0) / L)    # b_y at (i + 1/2, j)
            ctx.set_state(0, f, p)
            ebx = np.zeros(nsteps)
            for k in range(nsteps):
                ctx.step(1)
                g, _, _ = ctx.get_state(0, fields_only=True)
                ebx[k] = (g[3] ** 2).sum()
        rates[name] = _linear_phase_rate(ebx, dt)
        print("tearing %s: E_bx from %.3e to %.3e, growth rate %s" % (name, ebx[30], ebx.max(), rates[name]))
    T_pe = 2 * np.pi * n_x
    for name, r in rates.items():
        if r:
            print("tearing %s: tau = %.2f T_pe (paper: 2.5 T_pe at n_x = 15)" % (name, 1.0 / r / T_pe))
    assert rates["fp64"] and rates["mixed"], rates
    assert abs(rates["mixed"] / rates["fp64"] - 1) <= 0.10, rates


HARRIS = dict(theta=1.0, GU=0.68, wce=1.82, l_over_de=1.62, n_x=4.0, ppc=16, nx=64, ny=128)


def _harris_desc(mu):
    h = HARRIS
    L = h["l_over_de"] * h["n_x"]
    cap = int(h["ppc"] * 2.2 * L * h["ny"]) + 1024
    return pic.run_desc(2, h["nx"], h["ny"], 1, h["n_x"], 2.0 * h["ppc"], DT, [(-1.0, 1.0, cap), (1.0, mu, cap)],
                        bc=(1, 0, 0))


def _harris_load(ctx, mu, method, seeds):
    """Electrons drifting along -z and ions (or positrons) along +z with Gamma U
    = 0.68 and equal temperatures (App. C: Theta_i = Theta_e m_e/m_i, Gamma_i U_i
    = -Gamma_e U_e), sech^2 profile, B_y = B0 tanh((x - x0)/L) with the Table
    tearing relations for Theta = 1 (omega_ce/omega_pe = 1.82, L = 1.62 d_e)."""
    h = HARRIS
    L, x0 = h["l_over_de"] * h["n_x"], h["nx"] / 2.0
    beta = h["GU"] / np.sqrt(1.0 + h["GU"] ** 2)
    ctx.load_maxwell_juttner(0, 0, h["ppc"], h["theta"], (0.0, 0.0, -beta), profile=pic.PIC_PROFILE_HARRIS,
                             profile_params=(L, x0), method=method, seed=seeds[0])
    ctx.load_maxwell_juttner(0, 1, h["ppc"], h["theta"] / mu, (0.0, 0.0, beta), profile=pic.PIC_PROFILE_HARRIS,
                             profile_params=(L, x0), colocate_with=0, method=method, seed=seeds[1])
    f, p, _ = ctx.get_state(0)
    i = np.arange(h["nx"])
    f[4, 0, :, :] = h["wce"] / h["n_x"] * np.tanh((i[None, :] + 0.5 - x0) / L)    # b_y at (i + 1/2, j)
    ctx.set_state(0, f, p)
    return f, p


def _run_ebx(ctx, nsteps):
    e = np.zeros(nsteps)
    for k in range(nsteps):
        ctx.step(1)
        g, _, _ = ctx.get_state(0, fields_only=True)
        e[k] = (g[3] ** 2).sum()
    return e


@pytest.mark.parametrize("mu,nsteps", [(1.0, 1000), (25.0, 1400)])
def test_harris_tearing_matches_oracle_from_the_same_state(mu, nsteps):
    """Config 5 (Sect. 3.4, App. C) at reduced size: a relativistic Harris sheet
    of pairs (mu = m_i/m_e = 1) or of ions and electrons at equal temperature
    (mu = 25) between conducting walls, 64 x 128 cells, 4 cells per d_e, 16
    particles per cell per species at the sheet centre.  From one loaded state,
    the oracle, the FP64 path and the mixed path run side by side; the tearing
    mode grows out of the particle noise (b_x energy up by more than 1.5
    decades in the linear phase).  The FP64 path's E_bx equals the oracle's at
    every step to 1e-6 relative through step 800 (measured 2e-8 and 1e-7; the
    runs separate only once the sheet has torn), and the growth rates of both
    GPU paths equal the oracle's, FP64 to 1e-6 and mixed to 1 % (measured 1e-10
    and 8e-4).  The oracle runs as its OpenMP build (the same arithmetic; only
    the order of the FP64 current sums differs, as it does on the GPU)."""
    d = _harris_desc(mu)
    with pic.Context([d], precision=pic.PIC_FP64) as ctx:
        f, p = _harris_load(ctx, mu, pic.PIC_MJ_EXACT, (41, 42))
    st = oracle.State.empty(2, d.nx, d.ny, 1, DT, d.n_x, d.rho_sp0, bc_x=oracle.BC_CONDUCTOR)
    st.e[:] = f[:3]
    st.b[:] = f[3:]
    st.species.append(oracle.Species(p[0][:3].copy(), p[0][3:].copy(), -1.0, 1.0))
    st.species.append(oracle.Species(p[1][:3].copy(), p[1][3:].copy(), 1.0, mu))
    e_orc = np.zeros(nsteps)
    for k in range(nsteps):
        oracle.step_parallel(st, 1)
        e_orc[k] = (st.b[0] ** 2).sum()
    runs = {}
    for name, prec in (("fp64", pic.PIC_FP64), ("mixed", pic.PIC_MIXED)):
        with pic.Context([d], precision=prec) as ctx:
            ctx.set_state(0, f, p)
            runs[name] = _run_ebx(ctx, nsteps)
    ok = e_orc[:800] > 0
    rel = np.abs(runs["fp64"][:800] - e_orc[:800])[ok] / e_orc[:800][ok]
    r_orc = _linear_phase_rate(e_orc, DT)
    r64, rmx = _linear_phase_rate(runs["fp64"], DT), _linear_phase_rate(runs["mixed"], DT)
    print("tearing mu=%g: max |E_bx fp64 - oracle|/oracle over 800 steps %.2e; rates oracle %.6f fp64 %.6f mixed %.6f"
          % (mu, rel.max(), r_orc, r64, rmx))
    assert rel.max() <= 1e-6, rel.max()
    assert r_orc and r64 and rmx
    assert abs(r64 / r_orc - 1) <= 1e-6 and abs(rmx / r_orc - 1) <= 0.01, (r_orc, r64, rmx)


@pytest.mark.parametrize("mu,nsteps", [(1.0, 1000), (25.0, 1400)])
def test_harris_sheet_loaded_by_the_learned_sampler_tears_like_the_exact_loader(mu, nsteps):
    """Config 5 with the learned loader (the brief's pattern 4): the same Harris
    sheet (pairs, and ions of m_i/m_e = 25 at Theta_i = 0.04) loaded on the GPU
    by the trained network (FP16 inference) and by the exact inversion, with
    the same random streams, then advanced by the mixed path.  The tearing
    growth rates agree within 5 % (measured 1 %); sheets loaded with other
    seeds differ by about 18 %, so the learned sampler reproduces the exact
    loader's realisation, not only its statistics."""
    d = _harris_desc(mu)
    rates = {}
    for tag, method in (("exact", pic.PIC_MJ_EXACT), ("mlp", pic.PIC_MJ_MLP)):
        with pic.Context([d], precision=pic.PIC_MIXED) as ctx:
            if method == pic.PIC_MJ_MLP:
                ctx.mlp_train(steps=12000, batch=8192, lr=3e-3, seed=1)
            _harris_load(ctx, mu, method, (51, 52))
            rates[tag] = _linear_phase_rate(_run_ebx(ctx, nsteps), DT)
    print("tearing mu=%g by loader: exact %s mlp %s" % (mu, rates["exact"], rates["mlp"]))
    assert rates["exact"] and rates["mlp"]
    assert abs(rates["mlp"] / rates["exact"] - 1) <= 0.05, rates


def test_ensemble_field_fluctuation_level_scales_as_one_over_ppc():
    """Config 4 (Sect. 5.3): in thermal equilibrium each field mode holds an
    energy of order the temperature, so the field-fluctuation level, the field
    energy over the kinetic energy, falls as 1 / (particles per cell).  Five
    runs of one batched ensemble (64^2, theta = 0.1, n_x = theta^-1/2, 4 to 64
    ppc per species), levels averaged over steps 100-300; the log-log slope
    against ppc must be -1 within 0.25 (the paper pins the scaling, not the
    constant)."""
    theta, n_x = 0.1, 0.1 ** -0.5
    ppcs = [4, 8, 16, 32, 64]
    descs = [pic.run_desc(2, 64, 64, 1, n_x, 2.0 * ppc, 0.5,
                          [(-1.0, 1.0, ppc * 4096), (1.0, 1.0, ppc * 4096)]) for ppc in ppcs]
    with pic.Context(descs, precision=pic.PIC_MIXED) as ctx:
        for r, ppc in enumerate(ppcs):
            ctx.load_maxwell_juttner(r, 0, ppc, theta, seed=50 + 2 * r)
            ctx.load_maxwell_juttner(r, 1, ppc, theta, colocate_with=0, seed=51 + 2 * r)
        ctx.step(300)
        level = []
        for r in range(len(ppcs)):
            h = ctx.energy_history(r)
            level.append(((h[100:, 1] + h[100:, 2]) / h[100:, 0]).mean())
    slope = np.polyfit(np.log(ppcs), np.log(level), 1)[0]
    print("fluctuation level by ppc:", dict(zip(ppcs, np.round(level, 6))), "slope %.3f" % slope)
    assert abs(slope + 1.0) <= 0.25, slope


# ---------------------------------------------------------------- magnetized cold modes (Sect. 3.1.2)

def _cold_table():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "cold_modes_table.txt")
    return {row[0]: row for row in np.loadtxt(path, comments="#", ndmin=2)}


def _peak(omega, spec, mask):
    idx = np.where(mask)[0]
    i = idx[np.argmax(spec[idx])]
    a, b, c = np.log(spec[i - 1]), np.log(spec[i]), np.log(spec[(i + 1) % len(spec)])
    return omega[i] + 0.5 * (a - c) / (a - 2 * b + c) * (omega[1] - omega[0])


def _cold_modes(precision, wce, mu=49.0, theta_e=0.0016, ppc=16, nx=32, n_x=16.0, dt=0.5, periods=100, every=2):
    """Peaks of the electrons' k = 0 momentum spectra: (+omega_R, -omega_L) of
    sum (u_x + i u_y) and omega_P of sum u_z, in units of omega_pe."""
    nsamp = int(round(periods * 2 * np.pi * n_x / dt)) // every
    n = ppc * nx * nx
    d = pic.run_desc(2, nx, nx, 1, n_x, 2.0 * ppc, dt, [(-1.0, 1.0, n), (1.0, mu, n)])
    Z = np.zeros(nsamp, complex)
    Uz = np.zeros(nsamp)
    with pic.Context([d], precision=precision) as ctx:
        ctx.set_uniform_field(0, (0.0, 0.0, 0.0), (0.0, 0.0, wce / n_x))   # b = omega_ce X0 / c along z
        ctx.load_maxwell_juttner(0, 0, ppc, theta_e, (0.0, 0.0, 0.0), seed=31)
        ctx.load_maxwell_juttner(0, 1, ppc, theta_e / mu, (0.0, 0.0, 0.0), colocate_with=0, seed=32)
        for k in range(nsamp):
            ctx.step(every)
            su = ctx.diagnostics(0)["sum_u"][0]
            Z[k] = su[0] + 1j * su[1]
            Uz[k] = su[2]
    win = np.hanning(nsamp)
    omega = 2 * np.pi * np.fft.fftfreq(nsamp, every * dt) * n_x
    S = np.abs(np.fft.fft((Z - Z.mean()) * win)) ** 2
    Sz = np.abs(np.fft.fft((Uz - Uz.mean()) * win)) ** 2
    return (_peak(omega, S, omega > 0.2), -_peak(omega, S, omega < -0.2), _peak(omega, Sz, omega > 0.2))


@pytest.mark.parametrize("precision,wce", [(pic.PIC_MIXED, 1.0), (pic.PIC_MIXED, 2.0), (pic.PIC_FP64, 1.0)])
def test_magnetized_cold_modes_match_theory_and_table(precision, wce):
    """Table cold_modes (Sect. 3.1.2): a thermal electron-ion plasma (m_i/m_e =
    49, v_th = 0.04 c) in a uniform b0 along z, 32^2 cells, 16 cells per
    c/omega_pe (Debye length 0.64 cells), 16 ppc per species, 100 plasma periods
    (bins of 0.01 omega_pe), as in the table.  The electrons' total momentum
    peaks at omega_P along b0 and at the cut-offs across it, R at +omega_R and L
    at -omega_L in the spectrum of sum (u_x + i u_y) (the sense of gyration).
    Bars: 0.015 omega_pe against the cold two-species theory, and 0.025
    against the peaks the paper measured."""
    wr_m, wl_m, wp_m = _cold_modes(precision, wce)
    wl, wr = theory.cold_cutoffs_two_species(wce, 49.0)
    wp = theory.cold_plasma_frequency(49.0)
    assert abs(wr_m - wr) <= 0.015, (wr_m, wr)
    assert abs(wl_m - wl) <= 0.015, (wl_m, wl)
    assert abs(wp_m - wp) <= 0.015, (wp_m, wp)
    row = _cold_table()[wce]
    assert abs(wp_m - row[1]) <= 0.025 and abs(wl_m - row[2]) <= 0.025 and abs(wr_m - row[3]) <= 0.025, row


# ---------------------------------------------------------------- 3D filamentation and filament merging (Sect. 3.2, 3.3)

def filamentation_3d(precision=pic.PIC_MIXED, n_x=20.0, box_de=(4.5, 4.5, 15.0), rho_sp=80, beta0=0.995,
                     theta=0.01, n_t=250, periods=7.0, snap_every=0.5):
    """The paper's 3D counter-streaming setup: two electron-positron beams along
    +-z (co-located pairs, so rho = 0), thermal spread theta = 0.01 (v_th = 0.1 c)
    in each beam's frame, n_x cells per c/omega_pe, rho_sp superparticles per
    cell in all, n_t steps per plasma period.  Returns (t / T_pe per step, total
    magnetic energy per step, [(t / T_pe, filament scale in cells)])."""
    from oracle import filaments
    nx, ny, nz = (int(round(b * n_x)) for b in box_de)
    ppc = rho_sp // 4
    n = ppc * nx * ny * nz
    dt = 2 * np.pi * n_x / n_t
    d = pic.run_desc(3, nx, ny, nz, n_x, float(rho_sp), dt, [(-1.0, 1.0, n), (1.0, 1.0, n), (-1.0, 1.0, n),
                                                              (1.0, 1.0, n)])
    nsteps = int(round(periods * n_t))
    snap = int(round(snap_every * n_t))
    scales = []
    with pic.Context([d], precision=precision) as ctx:
        ctx.load_maxwell_juttner(0, 0, ppc, theta, (0.0, 0.0, beta0), seed=41)
        ctx.load_maxwell_juttner(0, 1, ppc, theta, (0.0, 0.0, beta0), colocate_with=0, seed=42)
        ctx.load_maxwell_juttner(0, 2, ppc, theta, (0.0, 0.0, -beta0), seed=43)
        ctx.load_maxwell_juttner(0, 3, ppc, theta, (0.0, 0.0, -beta0), colocate_with=2, seed=44)
        done = 0
        while done + snap + 1 <= nsteps:
            ctx.step(snap - 1)
            f0 = ctx.get_state(0, fields_only=True)[0]
            ctx.step(1)
            f1 = ctx.get_state(0, fields_only=True)[0]
            done += snap
            J = filaments.step_current(f0[:3], f1[:3], f1[3:], dt)
            scales.append((done / n_t, filaments.filament_scale(J)))
        h = ctx.energy_history(0)
    return np.arange(1, len(h) + 1) / n_t, h[:, 2], scales


def _tau_total_energy(t, eb, window=0.5):
    """e-folding time of the field amplitude, in T_pe, from the steepest fit of
    ln E_B over a window of `window` T_pe: E_B ~ exp(2 t / tau)."""
    dt = t[1] - t[0]
    w = int(round(window / dt))
    le = np.log(eb)
    best = 0.0
    for a in range(0, len(le) - w, max(1, w // 8)):
        slope = np.polyfit(t[a:a + w], le[a:a + w], 1)[0]
        best = max(best, slope)
    return 2.0 / best


def test_3d_relativistic_filamentation_matches_oracle_step_by_step():
    """3D counter-streaming pair beams (beta0 = 0.995, Gamma0 = 10, theta =
    0.01) in a 10 x 10 x 30 cell box (10 cells per c/omega_pe, 16 particles per
    cell, 125 steps per plasma period), from the oracle loader's state, over 4
    plasma periods: the magnetic energy grows by decades through the linear
    phase.  The GPU's per-step magnetic energy at time t must match the
    oracle's b^t (its b^{t-dt/2} advanced by the half step) to 1e-6 relative in
    the FP64 path, and the mixed path's growth to 2 %."""
    from oracle import mj
    nx, ny, nz, n_x, n_t, ppc, beta0, theta = 10, 10, 30, 10.0, 125, 4, 0.995, 0.01
    dt = 2 * np.pi * n_x / n_t
    steps = 4 * n_t
    n = ppc * nx * ny * nz
    parts, sp = [], []
    for s, (q, drift, seed) in enumerate([(-1.0, beta0, 51), (1.0, beta0, 52), (-1.0, -beta0, 53), (1.0, -beta0, 54)]):
        pos, u = mj.load(seed, s, n, theta, (0.0, 0.0, drift), 3, nx, ny, nz)
        if s % 2 == 1:
            pos = parts[-1][:3].copy()          # co-located with the electrons of the same beam
        parts.append(np.concatenate([pos, u]))
        sp.append(q)
    d = pic.run_desc(3, nx, ny, nz, n_x, 4.0 * ppc, dt, [(q, 1.0, n) for q in sp])
    fields = np.zeros((6, nz, ny, nx))
    st = oracle.State.empty(3, nx, ny, nz, dt, n_x, 4.0 * ppc)
    for q, p in zip(sp, parts):   # copies: the oracle advances its particles in place
        st.species.append(oracle.Species(p[:3].copy(), p[3:].copy(), q, 1.0))
    eb_or = np.zeros(steps)
    for k in range(steps):
        b_save = st.b.copy()
        oracle.b_advance(st, 0.5 * dt)                  # b^t of the step about to run
        eb_or[k] = 0.5 * (st.b ** 2).sum() * st.inv_alpha_abs
        st.b[:] = b_save
        oracle.step(st)
    hist = {}
    for name, prec in (("fp64", pic.PIC_FP64), ("mixed", pic.PIC_MIXED)):
        with pic.Context([d], precision=prec) as ctx:
            ctx.set_state(0, fields, parts)
            ctx.step(steps)
            hist[name] = ctx.energy_history(0)[:, 2]
    growth = eb_or[-1] / eb_or[n_t // 2]
    assert growth > 1e3, growth
    live = eb_or > 0
    assert np.abs(hist["fp64"][live] / eb_or[live] - 1).max() <= 1e-6
    t = np.arange(steps) / n_t
    lin = (t > 1.0) & (t < 3.5)
    s_or = np.polyfit(t[lin], np.log(eb_or[lin]), 1)[0]
    s_mx = np.polyfit(t[lin], np.log(hist["mixed"][lin]), 1)[0]
    assert abs(s_mx / s_or - 1) <= 0.02, (s_mx, s_or)


def test_3d_filamentation_at_the_paper_scale_grows_and_its_filaments_merge():
    """The 4.5 x 4.5 x 15 d_e setup of Table two_stream (beta0 = 0.995, 20 cells
    per d_e, rho_sp = 80, 250 steps per plasma period; 90 x 90 x 300 cells, 194M
    particles, ragged 8^3 tiles).  The magnetic energy grows exponentially and
    saturates; its growth time lies between the cold maximum rate and 1.75
    times it.  The filament scale (Sect. 3.3) grows through the non-linear
    phase: at saturation it is more than three times its value at the middle of
    the linear phase."""
    t, eb, scales = filamentation_3d()
    tau = _tau_total_energy(t[t > 0.5], eb[t > 0.5])
    tau_th = theory.tau_filamentation_pair(0.995)
    isat = int(np.argmax(eb))
    print("3D filamentation: tau_tot %.3f T_pe (cold maximum %.3f), saturation at %.2f T_pe" % (tau, tau_th, t[isat]))
    print("filament scale (T_pe, cells):", [(round(a, 2), round(b, 2)) for a, b in scales])
    assert eb[isat] / eb[int(0.5 * 250)] > 1e3
    assert tau_th <= tau <= 1.75 * tau_th, tau
    # middle of the linear phase: halfway (in log E_B) between 0.5 T_pe and saturation
    le = np.log(np.maximum(eb, 1e-300))
    lo = le[int(0.5 * 250)]
    tmid = t[int(np.argmax(le > 0.5 * (lo + le[isat])))]
    s_mid = np.interp(tmid, [a for a, _ in scales], [b for _, b in scales])
    s_sat = np.interp(t[isat], [a for a, _ in scales], [b for _, b in scales])
    print("scale at %.2f T_pe: %.2f cells, at saturation: %.2f cells" % (tmid, s_mid, s_sat))
    assert s_sat > 3.0 * s_mid


# ---------------------------------------------------------------- thermalization time against rho_sp (Sect. 5.2)

def _half_thermalization_time(rho_sp, precision=pic.PIC_MIXED, n=25, n_x=25.0, n_t=500, mu=25.0, t_cold=1.6e-3,
                              t_hot=1.8e-2, sample=0.5, progress=0.25, max_periods=120.0):
    """Two ion-electron plasmas, cold (T = 1.6e-3 m_e c^2) and hot (1.8e-2), m_i/m_e
    = 25, in a 25^3 box with 25 cells per c/omega_pe and 500 steps per plasma
    period (the paper's setup), rho_sp superparticles per cell over the four
    species.  Each plasma's ions sit on its electrons (rho = 0).  The cold
    electrons' temperature T1 relaxes as T_inf - (T_inf - T1(0)) exp(-2 t / t_th),
    T_inf = (T1 + T2) / 2 measured; t_th is taken from the slope of
    ln(T_inf - T1) over the start of the relaxation (until T1 has covered
    `progress` of the way), in plasma periods."""
    ppc = rho_sp // 4
    npart = ppc * n ** 3
    dt = 2 * np.pi * n_x / n_t
    d = pic.run_desc(3, n, n, n, n_x, float(rho_sp), dt, [(-1.0, 1.0, npart), (1.0, mu, npart),
                                                          (-1.0, 1.0, npart), (1.0, mu, npart)])
    ts, gap = [], []
    every = int(round(sample * n_t))
    with pic.Context([d], precision=precision) as ctx:
        ctx.load_maxwell_juttner(0, 0, ppc, t_cold, seed=71)
        ctx.load_maxwell_juttner(0, 1, ppc, t_cold / mu, colocate_with=0, seed=72)
        ctx.load_maxwell_juttner(0, 2, ppc, t_hot, seed=73)
        ctx.load_maxwell_juttner(0, 3, ppc, t_hot / mu, colocate_with=2, seed=74)
        t = 0.0
        while t < max_periods:
            dg = ctx.diagnostics(0)
            t1, t2 = dg["temperature"][0], dg["temperature"][2]
            ts.append(t)
            gap.append(0.5 * (t2 - t1))          # T_inf - T1
            if gap[-1] <= (1.0 - progress) * gap[0]:
                break
            ctx.step(every)
            t += sample
    ts, gap = np.array(ts), np.array(gap)
    slope = np.polyfit(ts, np.log(gap), 1)[0]
    return -2.0 / slope, ts[-1]


def test_thermalization_time_grows_as_rho_sp():
    """Sect. 5.2: the collision- and fluctuation-induced thermalization time of
    a PIC plasma scales as the PIC plasma parameter, t_th ~ rho_sp at fixed
    resolution (the paper disclaims the constant).  rho_sp = 4, 16, 64, 128:
    the log-log slope of t_th against rho_sp must lie in [0.7, 1.3]."""
    res = {r: _half_thermalization_time(r) for r in (4, 16, 64, 128)}
    print("thermalization time t_th / T_pe (window):", {r: (round(v[0], 1), v[1]) for r, v in res.items()})
    r = np.array(sorted(res))
    tth = np.array([res[k][0] for k in r])
    slope = np.polyfit(np.log(r), np.log(tth), 1)[0]
    print("log-log slope %.3f" % slope)
    assert np.all(np.diff(tth) > 0)
    assert 0.7 <= slope <= 1.3, slope
    # the FP64 path relaxes at the same rate: the mixed arithmetic does not change the collisionality
    t64 = _half_thermalization_time(4, precision=pic.PIC_FP64)[0]
    print("rho_sp = 4: t_th %.1f (mixed) %.1f (FP64)" % (res[4][0], t64))
    assert abs(t64 / res[4][0] - 1) <= 0.2


# ---------------------------------------------------------------- thermal-mode branches (Sect. 3.1.1)

def test_thermal_plasma_mode_branches_follow_the_dispersion_relations():
    """Sect. 3.1.1: in an unmagnetized thermal electron-ion plasma (m_i/m_e = 49,
    v_th = 0.1 c, Debye length = 1 cell, 10 cells per c/omega_pe) the Fourier modes
    k_x of the fields oscillate on two branches that meet at k = 0: the Langmuir
    wave (longitudinal e_x), omega^2 - omega_0^2 = 3 k^2 lambda_D^2 omega_pe^2,
    and the transverse wave (e_y), omega^2 - omega_0^2 = k^2 c^2.  omega_0 is the
    measured k = 0 oscillation (the relativistic shift of omega_P at this
    temperature, 1.3 %, cancels).  A 256 x 8 box, 32 ppc per species, 100
    plasma periods (bins of 0.01 omega_pe).  Bars: the Langmuir increments within
    15 %, the transverse ones within 3 %."""
    mu, theta, ppc, nx, ny, n_x, dt, every = 49.0, 0.01, 32, 256, 8, 10.0, 0.5, 2
    n = ppc * nx * ny
    d = pic.run_desc(2, nx, ny, 1, n_x, 2.0 * ppc, dt, [(-1.0, 1.0, n), (1.0, mu, n)])
    nsamp = int(round(100 * 2 * np.pi * n_x / dt)) // every
    ex = np.zeros((nsamp, nx // 2 + 1), complex)
    ey = np.zeros((nsamp, nx // 2 + 1), complex)
    with pic.Context([d], precision=pic.PIC_MIXED) as ctx:
        ctx.load_maxwell_juttner(0, 0, ppc, theta, (0.0, 0.0, 0.0), seed=81)
        ctx.load_maxwell_juttner(0, 1, ppc, theta / mu, (0.0, 0.0, 0.0), colocate_with=0, seed=82)
        for q in range(nsamp):
            ctx.step(every)
            f = ctx.get_state(0, fields_only=True)[0]
            ex[q] = np.fft.rfft(f[0, 0].mean(axis=0))
            ey[q] = np.fft.rfft(f[1, 0].mean(axis=0))
    win = np.hanning(nsamp)[:, None]
    omega = 2 * np.pi * np.fft.fftfreq(nsamp, every * dt) * n_x          # units of omega_pe

    def peak(series):
        spec = np.abs(np.fft.fft((series - series.mean()) * win[:, 0])) ** 2
        return abs(_peak(omega, spec, np.abs(omega) > 0.5))

    w0 = peak(ex[:, 0])
    kx = 2 * np.pi * np.arange(nx // 2 + 1) / nx                        # per cell
    for m in (6, 8, 10):
        k_lambda = kx[m] * (np.sqrt(theta) * n_x)                         # lambda_D = v_th / omega_pe in cells
        inc = (peak(ex[:, m]) ** 2 - w0 ** 2) / (3 * k_lambda ** 2)
        print("Langmuir m=%d k lambda_D=%.3f: increment ratio %.3f" % (m, k_lambda, inc))
        assert abs(inc - 1) <= 0.15, (m, inc)
    for m in (4, 8):
        kc = kx[m] * n_x
        inc = (peak(ey[:, m]) ** 2 - w0 ** 2) / kc ** 2
        print("transverse m=%d kc/omega_pe=%.3f: increment ratio %.4f" % (m, kc, inc))
        assert abs(inc - 1) <= 0.03, (m, inc)
    print("omega_0 = %.4f omega_pe (cold omega_P %.4f)" % (w0, theory.cold_plasma_frequency(mu)))
    assert abs(w0 / theory.cold_plasma_frequency(mu) - 1) <= 0.03


def _shell_spectrum_3d(e, nshell):
    """Shell sums of |E_k|^2 (all components) over |k| / |k|_max in nshell bins."""
    n = e.shape[-1]
    k = np.fft.fftfreq(n)
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2) / (0.5 * np.sqrt(3.0))
    idx = np.minimum((kk * nshell).astype(int), nshell - 1)
    p = sum(np.abs(np.fft.fftn(e[c])) ** 2 for c in range(3))
    return np.bincount(idx.ravel(), weights=p.ravel(), minlength=nshell)


def test_thermal_3d_long_run_tracks_oracle_energy_history_and_spectrum():
    """The 128^3 thermal pair plasma's parameters (theta = 1, 32 ppc per
    species, n_x = 1, rho_sp0 = 64, dt = 0.5 c/omega_pe) on a 32^3 copy, 1000
    steps of the mixed path and of the FP64 oracle (its OpenMP build, all host
    cores) from the same loaded state.
    - Energy history, compared quantity by quantity at every step: the kinetic
      energy at t_n (mean over u^{n-1/2} and u^{n+1/2}), the electric energy of
      e^n and the magnetic energy of b^n = (b^{n-1/2} + b^{n+1/2}) / 2, the
      time-centred field the step records.  Over the first 100 steps the paths
      agree to 1e-5 at every step (measured 1e-8 kinetic, 6e-7 electric: the
      FP32 and FP64 trajectories separate about tenfold every 50 steps); over
      steps 500-1000, where they have decorrelated, the means agree to 1%
      (measured 1e-4 kinetic, 1e-3 electric, 2e-3 magnetic) and the
      total-energy drift rates to 5% (measured 2.58e-4 per step in both, within
      0.2%; numerical heating, the paper's Sect. 3.1.3 quantity).
    - Electric-field spectrum: shell sums of |E_k|^2 averaged over the
      snapshots at steps 500, 600, ..., 1000 agree within [0.8, 1.25] in every
      shell but the corner one (measured 0.95-1.09; one snapshot scatters by
      10-20% per shell)."""
    N, ppc, theta, n_x, rho0, dt, steps, nshell = 32, 32, 1.0, 1.0, 64.0, 0.5, 1000, 16
    snaps = list(range(500, 1001, 100))
    n = ppc * N ** 3
    d = pic.run_desc(3, N, N, N, n_x, rho0, dt, [(-1.0, 1.0, n), (1.0, 1.0, n)])
    with pic.Context([d], precision=pic.PIC_MIXED) as ctx:
        ctx.load_maxwell_juttner(0, 0, ppc, theta, (0.0, 0.0, 0.0), seed=21)
        ctx.load_maxwell_juttner(0, 1, ppc, theta, (0.0, 0.0, 0.0), colocate_with=0, seed=22)
        f0, p0, _ = ctx.get_state(0)
        spec_g, done = [], 0
        for s in snaps:
            ctx.step(s - done)
            done = s
            f, _, _ = ctx.get_state(0, fields_only=True)
            spec_g.append(_shell_spectrum_3d(f[:3], nshell))
        hist = ctx.energy_history(0)
    st = oracle.State.empty(3, N, N, N, dt, n_x, rho0)
    st.e[:] = f0[:3]
    st.b[:] = f0[3:]
    for s, q in ((0, -1.0), (1, 1.0)):
        st.species.append(oracle.Species(np.ascontiguousarray(p0[s][:3]), np.ascontiguousarray(p0[s][3:]), q, 1.0))
    half_alpha = 0.5 * st.inv_alpha_abs
    kin = np.zeros(steps + 1)
    ele = np.zeros(steps)
    mag = np.zeros(steps)
    spec_o = []
    kin[0] = oracle.energies(st)["kinetic"].sum()
    for k in range(steps):
        ele[k] = half_alpha * (st.e ** 2).sum()
        b_before = st.b.copy()
        oracle.step_parallel(st, 1)
        mag[k] = half_alpha * (((b_before + st.b) * 0.5) ** 2).sum()
        kin[k + 1] = oracle.energies(st)["kinetic"].sum()
        if k + 1 in snaps:
            spec_o.append(_shell_spectrum_3d(st.e, nshell))
    ref = np.stack([0.5 * (kin[:-1] + kin[1:]), ele, mag], axis=1)
    got = hist[:steps, :3]
    early = np.abs(got[1:100] / ref[1:100] - 1).max(axis=0)
    late = got[500:].mean(axis=0) / ref[500:].mean(axis=0) - 1
    print("3D long run: early max rel diff (kin, E, B)", early, "late mean rel diff", late)
    assert np.all(early <= 1e-5), early
    assert np.all(np.abs(late) <= 1e-2), late
    tot_g, tot_o = got.sum(axis=1), ref.sum(axis=1)
    x = np.arange(100, steps)
    rate_g = np.polyfit(x, tot_g[100:] / tot_g[0], 1)[0]
    rate_o = np.polyfit(x, tot_o[100:] / tot_o[0], 1)[0]
    print("total-energy drift per step: mixed %.3e, oracle %.3e" % (rate_g, rate_o))
    assert abs(rate_g / rate_o - 1) <= 0.05, (rate_g, rate_o)
    ratio = np.mean(spec_g, axis=0) / np.mean(spec_o, axis=0)
    print("E spectrum ratio per shell:", np.round(ratio, 3))
    assert np.all((ratio[:-1] >= 0.8) & (ratio[:-1] <= 1.25)), ratio
