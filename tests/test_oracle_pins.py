"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an invariant of the scheme, or a brute-force geometric computation.
"""
import numpy as np
import pytest

import oracle
import synth


def _state(ndim, n, dt=0.5, n_x=1.0, rho_sp0=1e30, bc_x=oracle.BC_PERIODIC):
    nx, ny, nz = n
    return oracle.State.empty(ndim, nx, ny, nz, dt, n_x, rho_sp0, bc_x)


def _cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


# ---------------------------------------------------------------- Boris (App. A.3.3)

def test_boris_solves_implicit_rotation_equation():
    """u+ and u- satisfy (u+ - u-)/dt = h/(2 gamma) (u+ + u-) x b, Eq. mover1."""
    rng = np.random.default_rng(11)
    n = 2000
    u0 = rng.normal(0, 3.0, (3, n))
    EB = rng.normal(0, 2.0, (6, n))
    for h, dt in [(-1.0, 0.5), (1.0 / 25.0, 0.5), (1.0, 0.1)]:
        u1 = oracle.boris(u0, EB, h, dt)
        um = u0 + h * EB[:3] * dt / 2
        up = u1 - h * EB[:3] * dt / 2
        gam = np.sqrt(1 + (um ** 2).sum(0))
        lhs = (up - um) / dt
        rhs = h / (2 * gam) * _cross(up + um, EB[3:])
        scale = np.abs(h) * np.linalg.norm(um, axis=0) * np.linalg.norm(EB[3:], axis=0) / gam + 1e-300
        assert np.max(np.abs(lhs - rhs).max(0) / scale) < 1e-13
        # the rotation conserves |u|: gamma^t is the same from u- and u+
        assert np.allclose((up ** 2).sum(0), (um ** 2).sum(0), rtol=1e-14, atol=0)


def test_boris_pure_magnetic_conserves_energy_and_gyrates_in_closed_form():
    """Uniform b, e = 0: the discrete orbit advances by the constant angle
    2 atan(h b dt / (2 gamma)) per step (clockwise for h b > 0)."""
    B = 0.7
    h = -1.0
    dt = 0.5
    u = np.array([[2.0], [0.0], [0.3]])
    EB = np.zeros((6, 1))
    EB[5] = B
    gam = np.sqrt(1 + (u ** 2).sum())
    phi = 2 * np.arctan(h * B * dt / (2 * gam))
    for n in range(1, 501):
        u = oracle.boris(u, EB, h, dt)
        ang = -n * phi
        exp = np.array([2.0 * np.cos(ang), 2.0 * np.sin(ang), 0.3])
        assert np.allclose(u[:, 0], exp, rtol=0, atol=1e-12 * n)


def test_full_step_gyration_orbit_is_the_discrete_circle():
    """Through the whole oracle step (gather of a uniform b_z from the Yee grid,
    push, move): positions lie on the circle of the discrete orbit and advance
    by the closed-form angle per step (gyration test, Sect. 3.1.2)."""
    st = _state(2, (32, 32, 1), dt=0.5, rho_sp0=1e30)  # negligible self-field
    B = 0.2
    st.b[2][:] = B
    h = -1.0
    u_perp, uz = 0.5, 0.1
    # staggered start: u^{-1/2} rotated back by half the step angle is not needed;
    # we only check the orbit geometry produced by the scheme.
    pos = np.array([[16.0], [16.0], [0.0]])
    u = np.array([[u_perp], [0.0], [uz]])
    st.species.append(oracle.Species(pos, u, -1.0, 1.0))
    gam = np.sqrt(1 + u_perp ** 2 + uz ** 2)
    phi = 2 * np.arctan(h * B * st.dt / (2 * gam))
    xs = []
    for n in range(200):
        oracle.step(st)
        xs.append(st.species[0].pos[:2, 0].copy())
    xs = np.array(xs)
    step_len = st.dt * u_perp / gam
    R = step_len / (2 * abs(np.sin(phi / 2)))
    # centre from three consecutive points
    a, b, c = xs[0], xs[1], xs[2]
    d = 2 * (a[0] * (b[1] - c[1]) + b[0] * (c[1] - a[1]) + c[0] * (a[1] - b[1]))
    ux_ = ((a ** 2).sum() * (b[1] - c[1]) + (b ** 2).sum() * (c[1] - a[1]) + (c ** 2).sum() * (a[1] - b[1])) / d
    uy_ = ((a ** 2).sum() * (c[0] - b[0]) + (b ** 2).sum() * (a[0] - c[0]) + (c ** 2).sum() * (b[0] - a[0])) / d
    r = np.hypot(xs[:, 0] - ux_, xs[:, 1] - uy_)
    assert np.allclose(r, R, rtol=1e-10)
    ang = np.unwrap(np.arctan2(xs[:, 1] - uy_, xs[:, 0] - ux_))
    assert np.allclose(np.diff(ang), -phi, atol=1e-10)


def test_uniform_e_momentum_exact_and_position_second_order():
    """b = 0, uniform e: u^{n+1/2} = u^{-1/2} + h e n dt exactly; positions
    converge to relativistic hyperbolic motion x(t) = (sqrt(1+(h e t)^2)-1)/(h e)
    at second order in dt."""
    E = 0.05
    h = 1.0
    T = 40.0
    errs = []
    for dt in (0.5, 0.25, 0.125):
        st = _state(2, (256, 8, 1), dt=dt, rho_sp0=1e30)
        st.e[0][:] = E
        x0 = 100.0
        st.species.append(oracle.Species(np.array([[x0], [4.0], [0.0]]), np.zeros((3, 1)), 1.0, 1.0))
        oracle.stagger_back(st)
        u_half = st.species[0].u[0, 0]
        assert abs(u_half - (-h * E * dt / 2)) < 1e-15
        nsteps = int(round(T / dt))
        for n in range(nsteps):
            oracle.step(st)
        assert abs(st.species[0].u[0, 0] - (u_half + h * E * nsteps * dt)) < 1e-12
        x = st.species[0].pos[0, 0] - x0
        exact = (np.sqrt(1 + (h * E * T) ** 2) - 1) / (h * E)
        errs.append(abs(x - exact))
    order = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 1.8 < order[0] < 2.2 and 1.8 < order[1] < 2.2, (errs, order)


# ---------------------------------------------------------------- gather (App. A.3.3)

@pytest.mark.parametrize("ndim", [2, 3])
def test_gather_constant_fields_exact(ndim):
    """Constant fields interpolate exactly (Sect. 3.1.2, no self-force/bias)."""
    st = _state(ndim, (8, 6, 5))
    vals = [0.3, -1.1, 2.5, 0.7, -0.4, 1.9]
    for c in range(3):
        st.e[c][:] = vals[c]
        st.b[c][:] = vals[3 + c]
    rng = np.random.default_rng(3)
    pos = synth.positions(rng, ndim, st.nx, st.ny, st.nz, 500)
    EB = oracle.gather(st, pos)
    for c in range(6):
        assert np.allclose(EB[c], vals[c], rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("ndim", [2, 3])
def test_gather_linear_fields_exact(ndim):
    """Each component linear in space, sampled at its own staggered location,
    is reproduced exactly at the particle: node averaging and trilinear
    weighting are both exact on linear functions."""
    nx, ny, nz = 12, 10, 9
    st = _state(ndim, (nx, ny, nz))
    rng = np.random.default_rng(5)
    coef = rng.normal(0, 1, (6, 4))
    # staggering offsets of (e_x, e_y, e_z, b_x, b_y, b_z)
    off = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    K, J, I = np.meshgrid(np.arange(st.nz), np.arange(ny), np.arange(nx), indexing="ij")
    for c in range(6):
        ox, oy, oz = off[c]
        zz = (K + oz) if ndim == 3 else 0.0 * K
        if ndim == 2:
            coef[c, 3] = 0.0
        f = coef[c, 0] + coef[c, 1] * (I + ox) + coef[c, 2] * (J + oy) + coef[c, 3] * zz
        (st.e if c < 3 else st.b)[c % 3][:] = f
    n = 400
    pos = np.zeros((3, n))
    pos[0] = rng.uniform(2, nx - 3, n)
    pos[1] = rng.uniform(2, ny - 3, n)
    if ndim == 3:
        pos[2] = rng.uniform(2, nz - 3, n)
    EB = oracle.gather(st, pos)
    for c in range(6):
        exp = coef[c, 0] + coef[c, 1] * pos[0] + coef[c, 2] * pos[1] + coef[c, 3] * pos[2]
        assert np.allclose(EB[c], exp, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- deposit (App. A.1, A.3.4)

def _overlap(center, lo, hi):
    """Length of [center-1/2, center+1/2] intersected with [lo, hi]."""
    return np.clip(np.minimum(center + 0.5, hi) - np.maximum(center - 0.5, lo), 0.0, None)


def _geometric_currents(ndim, shape, x0, disp, alpha):
    """Brute force: the current of a uniformly charged unit cube moving along a
    straight line, integrated over the step as the geometric flux through each
    face of the grid-B cells (cells centred on the nodes).  The flux through the
    x face at x = i+1/2, |y - j| < 1/2, |z - k| < 1/2 is D_x times the time
    integral of the area of the cube's cross-section with that face patch
    (App. A.1).  Between the instants where a coordinate of the centre crosses
    an integer the integrand is a polynomial of degree <= 2, so 3-point
    Gauss-Legendre on each such piece integrates it exactly.
    Returns J = -alpha * flux, shape (3, nz, ny, nx)."""
    nz, ny, nx = shape
    brk = [0.0, 1.0]
    for a in range(ndim):
        for m in range(-20, 40):
            if disp[a] != 0.0:
                t = (m - x0[a]) / disp[a]
                if 0.0 < t < 1.0:
                    brk.append(t)
    brk = np.unique(brk)
    gx, gw = np.polynomial.legendre.leggauss(3)
    t = np.concatenate([lo + (hi - lo) * (gx + 1) / 2 for lo, hi in zip(brk[:-1], brk[1:])])
    w = np.concatenate([(hi - lo) * gw / 2 for lo, hi in zip(brk[:-1], brk[1:])])
    P = x0[:, None] + disp[:, None] * t[None, :]
    J = np.zeros((3, nz, ny, nx))
    axes = range(3) if ndim == 3 else range(2)
    rng_ = [range(int(np.floor(min(x0[a], x0[a] + disp[a]))) - 2, int(np.floor(max(x0[a], x0[a] + disp[a]))) + 3)
            for a in range(3)]
    if ndim == 2:
        rng_[2] = range(0, 1)
    for a in axes:
        b_, c_ = [x for x in range(3) if x != a]
        flat = ndim == 2 and c_ == 2
        for fa in rng_[a]:
            straddle = (np.abs(P[a] - (fa + 0.5)) < 0.5).astype(float)
            for fb in rng_[b_]:
                ob = _overlap(P[b_], fb - 0.5, fb + 0.5)
                for fc in ([0] if flat else rng_[c_]):
                    oc = np.ones_like(ob) if flat else _overlap(P[c_], fc - 0.5, fc + 0.5)
                    flux = disp[a] * np.sum(w * straddle * ob * oc)
                    idx = [0, 0, 0]
                    idx[a], idx[b_], idx[c_] = fa, fb, fc
                    i, j, k = idx[0] % nx, idx[1] % ny, idx[2] % nz
                    J[a, k, j, i] += -alpha * flux
    if ndim == 2:
        # out-of-plane current: D_z times the time-averaged overlap with each grid-B cell
        for fa in rng_[0]:
            ox = _overlap(P[0], fa - 0.5, fa + 0.5)
            for fb in rng_[1]:
                oy = _overlap(P[1], fb - 0.5, fb + 0.5)
                J[2, 0, fb % ny, fa % nx] += -alpha * disp[2] * np.sum(w * ox * oy)
    return J


@pytest.mark.parametrize("ndim", [2, 3])
def test_deposit_equals_geometric_flux_of_moving_cube(ndim):
    """Single paths with and without node-plane crossings (up to one per axis),
    compared with the brute-force geometric flux."""
    rng = np.random.default_rng(17 + ndim)
    shape = (1 if ndim == 2 else 8, 8, 8)
    st = _state(ndim, (8, 8, shape[0]))
    cases = []
    for _ in range(12):
        x0 = rng.uniform(2.0, 6.0, 3)
        d = rng.uniform(-0.45, 0.45, 3)
        if ndim == 2:
            x0[2] = 0.0
        cases.append((x0, d))
    # forced crossings in every axis and a corner
    cases.append((np.array([3.9, 4.05, 2.95 if ndim == 3 else 0.0]), np.array([0.3, -0.2, 0.4])))
    cases.append((np.array([4.0, 4.0, 4.0 if ndim == 3 else 0.0]), np.array([-0.3, 0.25, -0.1])))
    for x0, d in cases:
        alpha = 0.37
        Jo = oracle.deposit(st, x0[:, None], d[:, None], alpha)
        Jg = _geometric_currents(ndim, st.e.shape[1:], x0, d, alpha)
        assert np.allclose(Jo, Jg, rtol=0, atol=1e-14), (x0, d, np.abs(Jo - Jg).max())


@pytest.mark.parametrize("ndim,bc", [(2, oracle.BC_PERIODIC), (3, oracle.BC_PERIODIC)])
def test_step_conserves_gauss_law_to_roundoff(ndim, bc):
    """Discrete charge conservation (Sect. 2.1, App. A.1): the change of
    div e - rho~ over a step vanishes to round-off, from an arbitrary
    non-neutral state with fast particles crossing planes in every axis."""
    shape = (10, 9, 8)
    arr = synth.random_state_arrays(23 + ndim, ndim, *shape, ppc=6, spread=2.0,
                                    amp_e=0.01, amp_b=0.01, colocate=False)
    st = oracle.State.empty(ndim, *shape, dt=0.5, n_x=2.0, rho_sp0=8.0, bc_x=bc)
    st.e[:] = arr["e"]
    st.b[:] = arr["b"]
    for s in arr["species"]:
        st.species.append(oracle.Species(s["pos"], s["u"], s["q_over_e"], s["m_over_me"]))
    r0 = oracle.div_e(st) - oracle.rho(st)
    rmax = max(np.abs(oracle.rho(st, s)).max() for s in range(2))
    for _ in range(5):
        oracle.step(st)
        r1 = oracle.div_e(st) - oracle.rho(st)
        assert np.abs(r1 - r0).max() <= 1e-12 * rmax


@pytest.mark.parametrize("ndim", [2, 3])
def test_conductor_walls_reflect_and_conserve_charge_off_the_wall(ndim):
    """Conducting walls at x = 0 and x = n_x (App. A.4): particles stay in
    [0, n_x] with u_x reversed on reflection; the tangential e and the normal
    b vanish on the wall; the path to the wall and the mirrored remainder are
    each charge-conserving, so div e - rho~ is unchanged at every node off the
    wall plane (on it, the zeroed e_y, e_z change div e)."""
    shape = (10, 9, 8)
    arr = synth.random_state_arrays(31 + ndim, ndim, *shape, ppc=8, spread=2.0,
                                    amp_e=0.01, amp_b=0.01, colocate=False)
    st = oracle.State.empty(ndim, *shape, dt=0.5, n_x=2.0, rho_sp0=8.0, bc_x=oracle.BC_CONDUCTOR)
    st.e[:] = arr["e"]
    st.b[:] = arr["b"]
    for s in arr["species"]:
        st.species.append(oracle.Species(s["pos"], s["u"], s["q_over_e"], s["m_over_me"]))
    r0 = oracle.div_e(st) - oracle.rho(st)
    rmax = max(np.abs(oracle.rho(st, s)).max() for s in range(2))
    x_before = [sp.pos[0].copy() for sp in st.species]
    ux_before = [sp.u[0].copy() for sp in st.species]
    oracle.step(st)
    reflected = 0
    for s, sp in enumerate(st.species):
        assert sp.pos[0].min() >= 0.0 and sp.pos[0].max() <= shape[0]
        # a particle reflected at a wall comes back with u_x of the other sign
        flip = np.sign(sp.u[0]) == -np.sign(ux_before[s])
        reflected += int(flip.sum())
    assert reflected > 0
    for c in (1, 2):
        assert np.all(st.e[c][:, :, 0] == 0.0)
    assert np.all(st.b[0][:, :, 0] == 0.0)
    r1 = oracle.div_e(st) - oracle.rho(st)
    assert np.abs((r1 - r0)[:, :, 1:]).max() <= 1e-12 * rmax


def test_colocated_pairs_start_neutral_and_stay_neutral():
    """Pairs loaded on top of each other give rho~ = 0 with e = 0 (Sect. 2.1);
    Gauss's law then holds to round-off for all later steps."""
    arr = synth.random_state_arrays(29, 2, 16, 16, 1, ppc=8, spread=0.5)
    st = oracle.State.empty(2, 16, 16, 1, dt=0.5, n_x=3.0, rho_sp0=16.0)
    for s in arr["species"]:
        st.species.append(oracle.Species(s["pos"], s["u"], s["q_over_e"], s["m_over_me"]))
    g, rmax = oracle.gauss_residual(st)
    assert g < 1e-14
    for _ in range(20):
        oracle.step(st)
    g, rmax = oracle.gauss_residual(st)
    assert g <= 1e-12 * rmax


# ---------------------------------------------------------------- Yee solver (App. A.3.2)

def _yee_plane_wave_2d(nx, ny, mx, my, dt, n_t):
    """TE-like discrete eigenmode with e_z, b_x, b_y on a periodic 2D Yee grid,
    obeying sin^2(w dt/2)/dt^2 = sin^2(kx/2) + sin^2(ky/2)."""
    kx, ky = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
    s = np.sqrt(np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2)
    w = 2 * np.arcsin(s * dt) / dt
    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")

    def fields(t_e, t_b):
        # e_z at (i, j) time t_e; b_x at (i, j+1/2) and b_y at (i+1/2, j), time t_b
        ez = np.cos(kx * I + ky * J - w * t_e)
        # Faraday: db_x/dt = -d e_z/dy, db_y/dt = +d e_z/dx (discrete); amplitude from it
        ax = 2 * np.sin(ky / 2) / (2 * np.sin(w * dt / 2) / dt)
        ay = -2 * np.sin(kx / 2) / (2 * np.sin(w * dt / 2) / dt)
        bx = ax * np.cos(kx * I + ky * (J + 0.5) - w * t_b)
        by = ay * np.cos(kx * (I + 0.5) + ky * J - w * t_b)
        return ez, bx, by
    return fields


def test_yee_vacuum_wave_follows_discrete_dispersion():
    """A vacuum plane wave on the periodic Yee grid keeps the discrete
    dispersion relation sin^2(w dt/2)/dt^2 = sum_i sin^2(k_i/2) to round-off."""
    nx, ny, dt = 32, 24, 0.5
    fields = _yee_plane_wave_2d(nx, ny, 3, 2, dt, 0)
    st = _state(2, (nx, ny, 1), dt=dt, rho_sp0=1.0)
    ez, bx, by = fields(0.0, -0.5 * dt)
    st.e[2][0] = ez
    st.b[0][0] = bx
    st.b[1][0] = by
    nsteps = 60
    for _ in range(nsteps):
        oracle.step(st)  # no particles: pure field update
    ez, bx, by = fields(nsteps * dt, (nsteps - 0.5) * dt)
    assert np.abs(st.e[2][0] - ez).max() < 1e-11
    assert np.abs(st.b[0][0] - bx).max() < 1e-11
    assert np.abs(st.b[1][0] - by).max() < 1e-11
    assert np.abs(st.e[:2]).max() == 0.0 and np.abs(st.b[2]).max() == 0.0


def test_yee_3d_wave_and_div_b_preserved():
    """3D: an oblique TE wave in the (x, y) plane copied along z stays exact,
    and div b of an arbitrary random field is preserved by the field update."""
    nx, ny, nz, dt = 16, 12, 6, 0.5
    fields = _yee_plane_wave_2d(nx, ny, 2, 1, dt, 0)
    st = _state(3, (nx, ny, nz), dt=dt, rho_sp0=1.0)
    ez, bx, by = fields(0.0, -0.5 * dt)
    st.e[2][:] = ez[None]
    st.b[0][:] = bx[None]
    st.b[1][:] = by[None]
    for _ in range(30):
        oracle.step(st)
    ez, bx, by = fields(30 * dt, 29.5 * dt)
    assert np.abs(st.e[2] - ez[None]).max() < 1e-11
    rng = np.random.default_rng(2)
    st2 = _state(3, (nx, ny, nz), dt=dt, rho_sp0=1.0)
    st2.e[:] = rng.normal(0, 1, st2.e.shape)
    st2.b[:] = rng.normal(0, 1, st2.b.shape)

    def div_b(b):  # at cell centres (i+1/2, j+1/2, k+1/2)
        return ((np.roll(b[0], -1, axis=2) - b[0]) + (np.roll(b[1], -1, axis=1) - b[1]) +
                (np.roll(b[2], -1, axis=0) - b[2]))
    d0 = div_b(st2.b)
    for _ in range(10):
        oracle.step(st2)
    assert np.abs(div_b(st2.b) - d0).max() < 1e-12


def test_field_energy_units():
    """Field energy is |alpha|^-1 sum c^2/2 with |alpha| = 2/(n_x^2 rho_sp0), Eq. alpha."""
    st = _state(2, (4, 4, 1), n_x=3.0, rho_sp0=10.0)
    st.e[0][:] = 2.0
    en = oracle.energies(st)
    assert np.isclose(en["field_e"][0], 16 * 0.5 * 4.0 / (2.0 / (9.0 * 10.0)))


def _two_species_exact_gammas():
    """A heavy species (m/m_e = 25) and an electron species whose momenta have
    exact Lorentz factors: |u|^2 = 3, 8, 0.5625 give gamma = 2, 3, 1.25, and
    |u|^2 = 24, 0.5625 give gamma = 5, 1.25."""
    st = _state(3, (4, 4, 4))
    u_ion = np.array([[0.0, 2.0, 0.75], [0.0, 2.0, 0.0], [np.sqrt(3.0), 0.0, 0.0]])
    u_el = np.array([[2.0, -0.75], [2.0, 0.0], [4.0, 0.0]])
    st.species.append(oracle.Species(np.zeros((3, 3)), np.ascontiguousarray(u_ion), 1.0, 25.0))
    st.species.append(oracle.Species(np.zeros((3, 2)), np.ascontiguousarray(u_el), -1.0, 1.0))
    return st


def test_kinetic_energy_counts_the_species_mass():
    """App. A.2 energy units: the kinetic energy is sum (m_s/m_e)(gamma - 1).
    Worked by hand: ions 25 (1 + 2 + 0.25) = 81.25, electrons 4 + 0.25 = 4.25.
    Dropping the mass factor would give 3.25 for the ions."""
    en = oracle.energies(_two_species_exact_gammas())
    assert abs(en["kinetic"][0] - 81.25) < 1e-12
    assert abs(en["kinetic"][1] - 4.25) < 1e-12


def test_temperature_is_mass_times_mean_u_dot_v_over_3():
    """Sect. 3.1.3: T = m <v^2>/3, relativistically (m_s/m_e) <u . v>/3 in
    units of m_e c^2 (u . v = |u|^2/gamma).  Worked by hand: ions 25 (3/2 +
    8/3 + 0.45)/9 = 1385/108, electrons (24/5 + 0.45)/6 = 7/8."""
    T = oracle.temperature(_two_species_exact_gammas())
    assert abs(T[0] - 1385.0 / 108.0) < 1e-12
    assert abs(T[1] - 0.875) < 1e-14


def test_temperature_of_maxwell_juttner_ions_is_mass_times_theta():
    """A Maxwell-Juttner population of Theta = T/(m c^2) has <u . v> = 3 Theta
    (Table averages of Sect. 4), so ions of m_i/m_e = 25 loaded at Theta =
    0.04 report T = 1 m_e c^2, and electrons at Theta = 1 report 1: the two
    species of a plasma in equilibrium share T (within 4 sigma of the sample)."""
    from oracle import mj
    n = 100000
    st = _state(3, (8, 8, 8))
    for seed, theta, m in ((21, 0.04, 25.0), (22, 1.0, 1.0)):
        w = mj.uniforms(seed, 0, np.arange(n))
        u = mj.sample_momenta(w[3], w[4], w[5], theta, np.zeros(3))
        st.species.append(oracle.Species(np.zeros((3, n)), np.ascontiguousarray(u), 1.0, m))
        uv = (u ** 2).sum(0) / np.sqrt(1 + (u ** 2).sum(0))
        sigma = m * uv.std() / 3 / np.sqrt(n)
        T = oracle.temperature(st)[-1]
        assert abs(T - 1.0) < 4 * sigma, (theta, m, T, sigma)


def test_thermal_plasma_k0_oscillation_is_at_the_relativistic_cutoff():
    """Sect. 3.1: the k = 0 electric field of a thermal pair plasma oscillates
    at omega_cut = omega_P <gamma^-1 (1 - beta^2/3)>^(1/2), omega_P^2 = 2/n_x^2
    for pairs (n_x cells per c/omega_pe).  A small box (16^2, theta = 0.1,
    dx = lambda_D, 16 ppc per species) over 60 plasma periods: the peak of the
    power spectrum of the box-mean e_x lies within 3 % of the cutoff (the
    frequency bins are 1.3 % of it)."""
    from scipy import integrate
    from oracle import mj
    theta, ppc, nsteps, dt, nx = 0.1, 16, 2400, 0.5, 16
    n_x = theta ** -0.5
    n = ppc * nx * nx
    st = oracle.State.empty(2, nx, nx, 1, dt, n_x, 2.0 * ppc)
    pos, u0 = mj.load(5, 0, n, theta, (0.0, 0.0, 0.0), 2, nx, nx, 1)
    _, u1 = mj.load(6, 1, n, theta, (0.0, 0.0, 0.0), 2, nx, nx, 1)
    st.species.append(oracle.Species(pos, u0, -1.0, 1.0))
    st.species.append(oracle.Species(pos.copy(), u1, 1.0, 1.0))
    ex = np.zeros(nsteps)
    for k in range(nsteps):
        oracle.step(st)
        ex[k] = st.e[0].mean()
    spec = np.abs(np.fft.rfft((ex - ex.mean()) * np.hanning(nsteps))) ** 2
    omega = 2 * np.pi * np.fft.rfftfreq(nsteps, dt)
    peak = omega[1 + np.argmax(spec[1:])]
    w = lambda uu: uu * uu * np.exp(-(np.sqrt(1 + uu * uu) - 1) / theta)
    f = lambda uu: w(uu) / np.sqrt(1 + uu * uu) * (1 - (uu * uu / (1 + uu * uu)) / 3)
    factor = integrate.quad(f, 0, np.inf, limit=400)[0] / integrate.quad(w, 0, np.inf, limit=400)[0]
    omega_cut = np.sqrt(2.0) / n_x * np.sqrt(factor)
    assert abs(peak / omega_cut - 1) <= 0.03, (peak, omega_cut)


# ---------------------------------------------------------------- current smoothing (App. A.3.4)

def _printed_smoothing_weights():
    """Weight by number of shifted indices, as printed in App. A.3.4 (golden fixture)."""
    import os
    w = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "current_smoothing_weights.txt")
    for line in open(path):
        f = line.split("#")[0].split()
        if f:
            w[int(f[0])] = float(f[1])
    return w


@pytest.mark.parametrize("ndim", [2, 3])
def test_smoothing_impulse_response_is_the_printed_weights(ndim):
    """A unit value spread by one pass: every neighbour receives its printed
    weight divided by the sum of the 27 weights.  In 2D3V the z neighbours are
    the cell itself (z ignorable), so their weights land on the same plane."""
    w = _printed_smoothing_weights()
    st = _state(ndim, (7, 6, 5))
    nz, ny, nx = st.e.shape[1:]
    c = (2, 3, 4) if ndim == 3 else (0, 3, 4)            # (k, j, i), the second near the edge
    a = np.zeros((nz, ny, nx))
    a[c] = 1.0
    expect = np.zeros_like(a)
    total = sum(w[(di != 0) + (dj != 0) + (dk != 0)]
                for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1))
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                q = ((c[0] + dk) % nz, (c[1] + dj) % ny, (c[2] + di) % nx)
                expect[q] += w[(di != 0) + (dj != 0) + (dk != 0)] / total
    out = oracle.smooth(st, a)
    assert np.abs(out - expect).max() <= 1e-16
    assert abs(out.sum() - 1.0) <= 1e-15


@pytest.mark.parametrize("ndim,passes", [(2, 1), (3, 1), (3, 2)])
def test_smoothing_transfer_function_is_a_product_of_cos_squared(ndim, passes):
    """A Fourier mode of wavenumbers (m_x, m_y, m_z) is an eigenvector of one
    pass with eigenvalue prod_a cos^2(pi m_a / n_a) (the 1-2-1 stencil per
    axis); the Nyquist mode m_x = n_x/2 is removed."""
    st = _state(ndim, (12, 10, 8))
    nz, ny, nx = st.e.shape[1:]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for m in [(0, 0, 0), (1, 0, 0), (2, 3, 1), (5, 4, 3), (6, 5, 4)]:
        mz = m[2] if ndim == 3 else 0
        a = np.cos(2 * np.pi * (m[0] * i / nx + m[1] * j / ny + mz * k / nz) + 0.3)
        H = np.cos(np.pi * m[0] / nx) ** 2 * np.cos(np.pi * m[1] / ny) ** 2 * np.cos(np.pi * mz / nz) ** 2
        out = oracle.smooth(st, a, passes)
        assert np.abs(out - H ** passes * a).max() <= 1e-14, m


@pytest.mark.parametrize("ndim,passes", [(2, 1), (3, 1), (2, 2)])
def test_smoothed_step_conserves_the_smoothed_gauss_law(ndim, passes):
    """With the current smoothed by S before it is added to e (main-loop step
    10), a step conserves div e - S rho~ to round-off: S is a translation-
    invariant stencil, so it commutes with the discrete divergence.  The
    unsmoothed residual div e - rho~ then changes at the level of the charge."""
    shape = (10, 9, 8)
    arr = synth.random_state_arrays(31 + ndim + passes, ndim, *shape, ppc=6, spread=2.0,
                                    amp_e=0.01, amp_b=0.01, colocate=False)
    st = oracle.State.empty(ndim, *shape, dt=0.5, n_x=2.0, rho_sp0=8.0, smooth_passes=passes)
    st.e[:] = arr["e"]
    st.b[:] = arr["b"]
    for s in arr["species"]:
        st.species.append(oracle.Species(s["pos"], s["u"], s["q_over_e"], s["m_over_me"]))
    rmax = max(np.abs(oracle.rho(st, s)).max() for s in range(2))
    smoothed0 = oracle.div_e(st) - oracle.smooth(st, oracle.rho(st), passes)
    raw0 = oracle.div_e(st) - oracle.rho(st)
    for _ in range(4):
        oracle.step(st)
        smoothed1 = oracle.div_e(st) - oracle.smooth(st, oracle.rho(st), passes)
        assert np.abs(smoothed1 - smoothed0).max() <= 1e-12 * rmax
    raw1 = oracle.div_e(st) - oracle.rho(st)
    assert np.abs(raw1 - raw0).max() > 1e-3 * rmax
    assert oracle.gauss_residual(st)[0] == pytest.approx(np.abs(smoothed1).max(), rel=0, abs=0)


def test_smoothing_off_leaves_the_step_unchanged():
    """smooth_passes = 0 is the unsmoothed scheme, bit for bit."""
    shape = (8, 6, 1)
    arr = synth.random_state_arrays(41, 2, *shape, ppc=4, spread=1.0, amp_e=0.01, amp_b=0.01, colocate=False)
    out = []
    for passes in (0, 1):
        st = oracle.State.empty(2, *shape, dt=0.5, n_x=2.0, rho_sp0=8.0, smooth_passes=passes)
        st.e[:] = arr["e"]
        st.b[:] = arr["b"]
        for s in arr["species"]:
            st.species.append(oracle.Species(s["pos"].copy(), s["u"].copy(), s["q_over_e"], s["m_over_me"]))
        J = oracle.step(st)
        out.append((st.e.copy(), J))
    st0 = oracle.State.empty(2, *shape, dt=0.5, n_x=2.0, rho_sp0=8.0)
    assert np.array_equal(out[1][1], oracle.smooth(st0, out[0][1], 1))
    assert not np.array_equal(out[0][0], out[1][0])


# ---------------------------------------------------------------- magnetized cold modes (Sect. 3.1.2)

def _spectral_peak(omega, spec, mask):
    """Frequency of the largest value of spec inside mask, refined by a parabola
    through the logarithms of the three bins around it."""
    idx = np.where(mask)[0]
    i = idx[np.argmax(spec[idx])]
    a, b, c = np.log(spec[i - 1]), np.log(spec[i]), np.log(spec[(i + 1) % len(spec)])
    return omega[i] + 0.5 * (a - c) / (a - 2 * b + c) * (omega[1] - omega[0])


def test_magnetized_plasma_k0_modes_are_the_cold_cutoffs():
    """Sect. 3.1.2: in a thermal electron-ion plasma (m_i/m_e = 49, v_th = 0.04 c)
    with a uniform b0 along z, the electrons' total momentum oscillates at
    omega_P along b0 and at the cut-offs omega_L, omega_R across it.  The
    transverse spectrum is taken of sum (u_x + i u_y): electrons gyrate in the
    positive sense about +z, so the R cut-off (same sense) appears at +omega_R and
    the L cut-off (opposite sense) at -omega_L, which pins the sense of the
    magnetic rotation.  omega_ce = 2 omega_pe, 8^2 cells, 16 cells per c/omega_pe,
    60 plasma periods (bins of 0.017 omega_pe); the ions' finite mass moves
    omega_L by 0.04 omega_pe from the heavy-ion formula, 3 bins."""
    from oracle import mj, theory
    wce, mu, theta_e, ppc, nx, n_x, dt = 2.0, 49.0, 0.0016, 8, 8, 16.0, 0.5
    nsteps = int(round(60 * 2 * np.pi * n_x / dt))
    n = ppc * nx * nx
    st = oracle.State.empty(2, nx, nx, 1, dt, n_x, 2.0 * ppc)
    pos, ue = mj.load(21, 0, n, theta_e, (0.0, 0.0, 0.0), 2, nx, nx, 1)
    _, ui = mj.load(22, 1, n, theta_e / mu, (0.0, 0.0, 0.0), 2, nx, nx, 1)
    st.species.append(oracle.Species(pos, ue, -1.0, 1.0))
    st.species.append(oracle.Species(pos.copy(), ui, 1.0, mu))
    st.b[2][:] = wce / n_x                  # b = omega_ce X0 / c
    oracle.stagger_back(st)
    Z = np.zeros(nsteps, complex)
    Uz = np.zeros(nsteps)
    for k in range(nsteps):
        oracle.step(st)
        u = st.species[0].u
        Z[k] = u[0].sum() + 1j * u[1].sum()
        Uz[k] = u[2].sum()
    win = np.hanning(nsteps)
    omega = 2 * np.pi * np.fft.fftfreq(nsteps, dt) * n_x      # units of omega_pe
    S = np.abs(np.fft.fft((Z - Z.mean()) * win)) ** 2
    Sz = np.abs(np.fft.fft((Uz - Uz.mean()) * win)) ** 2
    wl, wr = theory.cold_cutoffs_two_species(wce, mu)
    wp = theory.cold_plasma_frequency(mu)
    assert abs(_spectral_peak(omega, S, omega > 0.2) - wr) <= 0.015
    assert abs(_spectral_peak(omega, S, omega < -0.2) + wl) <= 0.015
    assert abs(_spectral_peak(omega, Sz, omega > 0.2) - wp) <= 0.015


# ---------------------------------------------------------------- filament-merging diagnostic (Sect. 3.3)

def test_step_current_is_recovered_from_two_field_states():
    """J = e^{t+dt} - e^t - dt curl b^{t+dt/2} returns exactly what the oracle's
    step added to e (the identity of main-loop steps 6 and 12)."""
    from oracle import filaments
    shape = (10, 9, 8)
    arr = synth.random_state_arrays(61, 3, *shape, ppc=4, spread=1.5, amp_e=0.02, amp_b=0.02, colocate=False)
    st = oracle.State.empty(3, *shape, dt=0.5, n_x=2.0, rho_sp0=8.0)
    st.e[:] = arr["e"]
    st.b[:] = arr["b"]
    for s in arr["species"]:
        st.species.append(oracle.Species(s["pos"], s["u"], s["q_over_e"], s["m_over_me"]))
    e0 = st.e.copy()
    J = oracle.step(st)
    rec = filaments.step_current(e0, st.e, st.b, st.dt)
    assert np.abs(rec - J).max() <= 1e-14 * max(1.0, np.abs(st.e).max())
    assert np.abs(J).max() > 1e-4


def test_filament_scale_of_gaussian_filaments_is_the_closed_form():
    """Randomly placed Gaussian filaments exp(-r^2 / 2 s^2): the autocorrelation
    of the field is exp(-r^2 / 4 s^2), so corr = 0.8 at r = 2 s sqrt(ln 1.25)
    and the scale is 5 times that."""
    from oracle import filaments
    rng = np.random.default_rng(7)
    n, s = 256, 3.0
    y, x = np.mgrid[0:n, 0:n]
    amp = np.zeros((n, n))
    for cx, cy in rng.uniform(0, n, size=(600, 2)):
        dx = np.minimum(np.abs(x - cx), n - np.abs(x - cx))
        dy = np.minimum(np.abs(y - cy), n - np.abs(y - cy))
        amp += np.exp(-(dx * dx + dy * dy) / (2 * s * s))
    cur = np.zeros((3, 4, n, n))
    cur[2] = amp[None]                         # J_z filaments, constant along z
    expect = 5.0 * 2.0 * s * np.sqrt(np.log(1.25))
    assert abs(filaments.filament_scale(cur) / expect - 1) <= 0.05


def test_openmp_build_of_the_oracle_equals_the_plain_build():
    """The all-cores timing build (particle loop shared between threads, one
    current grid per thread) gives the plain oracle's step up to the order of
    the FP64 current sums."""
    import synth
    arr = synth.random_state_arrays(3, 3, 12, 10, 8, ppc=6, spread=0.5, amp_e=0.02, amp_b=0.02, colocate=False)

    def make():
        st = oracle.State.empty(3, 12, 10, 8, 0.5, 2.0, 12.0)
        st.e[:] = arr["e"]
        st.b[:] = arr["b"]
        for sp in arr["species"]:
            st.species.append(oracle.Species(sp["pos"].copy(), sp["u"].copy(), sp["q_over_e"], sp["m_over_me"]))
        return st
    a, b = make(), make()
    oracle.step(a, 3)
    threads = oracle.step_parallel(b, 3, 4)
    assert threads >= 1
    assert np.abs(a.e - b.e).max() <= 1e-13 * np.abs(a.e).max()
    for sa, sb in zip(a.species, b.species):
        assert np.abs(sa.pos - sb.pos).max() <= 1e-12
        assert np.abs(sa.u - sb.u).max() <= 1e-13 * np.abs(sa.u).max()

