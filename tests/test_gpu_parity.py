"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

FP64 path: one step (and several) from an identical state, norm-wise relative
difference <= 1e-12 per field component and per particle array.
Mixed path: one step from the same FP32-rounded state, fields <= 1e-5
relative (norm-wise), positions <= 2e-6 cells, momenta <= 1e-5 relative, and
the Gauss residual of a neutral start <= 1e-6 of max |rho~_s|.
"""
import numpy as np
import pytest

import oracle
import paper_1308_5892_gb300 as pic
import synth

pytestmark = pytest.mark.gpu


def _make(ndim, shape, ppc, seed, spread, amp, colocate, n_x=2.0, rho_sp0=8.0, dt=0.5, species=synth.PAIR,
          bc=(0, 0, 0)):
    nx, ny, nz = shape
    arr = synth.random_state_arrays(seed, ndim, nx, ny, nz, ppc=ppc, spread=spread, amp_e=amp, amp_b=amp,
                                    colocate=colocate, species=species)
    n = arr["species"][0]["pos"].shape[1]
    desc = pic.run_desc(ndim, nx, ny, nz if ndim == 3 else 1, n_x, rho_sp0, dt,
                        [(s["q_over_e"], s["m_over_me"], n) for s in arr["species"]], bc=bc)
    fields = np.concatenate([arr["e"], arr["b"]])
    parts = [np.concatenate([s["pos"], s["u"]]) for s in arr["species"]]
    return desc, fields, parts, arr


def _oracle_state(desc, fields, parts, arr):
    st = oracle.State.empty(desc.ndim, desc.nx, desc.ny, desc.nz, desc.dt, desc.n_x, desc.rho_sp0,
                            bc_x=desc.bc[0])
    st.e[:] = fields[:3]
    st.b[:] = fields[3:]
    for s, p in zip(arr["species"], parts):
        st.species.append(oracle.Species(np.ascontiguousarray(p[:3]), np.ascontiguousarray(p[3:]),
                                         s["q_over_e"], s["m_over_me"]))
    return st


def _rel(a, b):
    if a.size == 0:
        return 0.0
    den = np.abs(b).max()
    return np.abs(a - b).max() / den if den > 0 else np.abs(a - b).max()


def _pos_diff(a, b, L):
    if a.size == 0:
        return 0.0
    d = a - b
    return np.abs(d - L * np.round(d / L)).max()


def _compare(desc, f_gpu, p_gpu, st, tol_field, tol_pos, tol_u):
    ref_f = np.concatenate([st.e, st.b])
    for c in range(6):
        r = _rel(f_gpu[c], ref_f[c])
        assert r <= tol_field, ("field component", c, r)
    L = [desc.nx, desc.ny, desc.nz]
    for s, sp in enumerate(st.species):
        for a in range(desc.ndim):
            d = _pos_diff(p_gpu[s][a], sp.pos[a], L[a])
            assert d <= tol_pos, ("position", s, a, d)
        for a in range(3):
            r = _rel(p_gpu[s][3 + a], sp.u[a])
            assert r <= tol_u, ("momentum", s, a, r)


# ----------------------------------------------------------------- FP64 path

@pytest.mark.parametrize("ndim,shape,ppc", [(2, (33, 20, 1), 4), (3, (12, 10, 9), 3)])
def test_fp64_steps_match_oracle_to_1e12(ndim, shape, ppc):
    desc, fields, parts, arr = _make(ndim, shape, ppc, seed=100 + ndim, spread=2.0, amp=0.05, colocate=False)
    with pic.Context([desc], precision=pic.PIC_FP64) as ctx:
        ctx.set_state(0, fields, parts)
        st = _oracle_state(desc, fields, parts, arr)
        for nsteps in (1, 4):
            ctx.step(nsteps)
            oracle.step(st, nsteps)
            f, p, step = ctx.get_state(0)
            _compare(desc, f, p, st, 1e-12, 1e-12 * max(shape), 1e-12)


def test_fp64_diagnostics_match_oracle():
    desc, fields, parts, arr = _make(2, (24, 16, 1), 6, seed=7, spread=1.0, amp=0.05, colocate=False)
    with pic.Context([desc], precision=pic.PIC_FP64) as ctx:
        ctx.set_state(0, fields, parts)
        ctx.step(3)
        d = ctx.diagnostics(0)
        f, p, _ = ctx.get_state(0)
    st = _oracle_state(desc, f, p, arr)
    en = oracle.energies(st)
    assert np.allclose(d["kinetic"], en["kinetic"], rtol=1e-12)
    assert np.allclose(d["field_e"], en["field_e"], rtol=1e-12)
    assert np.allclose(d["field_b"], en["field_b"], rtol=1e-12)
    g, rmax = oracle.gauss_residual(st)
    assert abs(d["gauss_max"] - g) <= 1e-12 * rmax
    assert np.isclose(d["rho_max"], rmax, rtol=1e-12)
    for s in range(2):
        assert np.allclose(d["sum_u"][s], st.species[s].u.sum(1), rtol=1e-12, atol=1e-9)


ION_ELECTRON = (synth.SpeciesSpec(-1.0, 1.0), synth.SpeciesSpec(+1.0, 25.0))


@pytest.mark.parametrize("precision,tol", [(pic.PIC_FP64, 1e-12), (pic.PIC_MIXED, 1e-6)])
def test_diagnostics_with_a_heavy_species_match_oracle(precision, tol):
    """Temperature (m_s/m_e) <u . v>/3 and kinetic energy sum (m_s/m_e)(gamma - 1)
    of an electron-ion state (m_i/m_e = 25, Sect. 3.1.3, App. A.2) against the
    oracle's pinned functions, on the uploaded state and after 3 steps: FP64
    to 1e-12, mixed to 1e-6 (its FP32 momenta differ from the oracle's FP64
    trajectories at about 1e-7 per step)."""
    desc, fields, parts, arr = _make(3, (12, 10, 8), 6, seed=17, spread=0.8, amp=0.05, colocate=False,
                                     species=ION_ELECTRON)
    with pic.Context([desc], precision=precision) as ctx:
        ctx.set_state(0, fields, parts)
        f0, p0, _ = ctx.get_state(0)
        d0 = ctx.diagnostics(0)
        ctx.step(3)
        d3 = ctx.diagnostics(0)
    st = _oracle_state(desc, f0, p0, arr)
    for d, label in ((d0, "uploaded"), (None, "after 3 steps")):
        if d is None:
            oracle.step(st, 3)
            d = d3
        T = oracle.temperature(st)
        en = oracle.energies(st)
        assert np.allclose(d["temperature"], T, rtol=tol), (label, d["temperature"], T)
        assert np.allclose(d["kinetic"], en["kinetic"], rtol=tol), (label, d["kinetic"], en["kinetic"])
    # the heavy species' temperature carries its mass: u.v/3 alone would be 25x smaller
    assert d0["temperature"][1] > 5 * d0["temperature"][0]


def test_fp64_neutral_start_keeps_gauss_to_roundoff():
    desc, fields, parts, arr = _make(3, (10, 12, 8), 4, seed=9, spread=1.5, amp=0.0, colocate=True)
    fields[3:] = np.random.default_rng(1).normal(0, 0.05, fields[3:].shape)
    with pic.Context([desc], precision=pic.PIC_FP64) as ctx:
        ctx.set_state(0, fields, parts)
        ctx.step(20)
        d = ctx.diagnostics(0)
    assert d["gauss_max"] <= 1e-12 * d["rho_max"]


def _walls(parts, nx):
    """Put particles on and next to both walls, moving into them (App. A.4)."""
    for p in parts:
        k = min(8, p.shape[1])
        p[0, :k] = [0.0, nx, 0.05, nx - 0.05, 0.3, nx - 0.3, 0.0, nx][:k]
        p[3, :k] = [-1.5, 1.5, -2.0, 2.0, -3.0, 3.0, 0.7, -0.7][:k]


@pytest.mark.parametrize("ndim,shape,ppc", [(2, (33, 20, 1), 6), (3, (12, 10, 9), 4)])
def test_fp64_conductor_walls_match_oracle(ndim, shape, ppc):
    desc, fields, parts, arr = _make(ndim, shape, ppc, seed=120 + ndim, spread=2.0, amp=0.05, colocate=False,
                                     bc=(1, 0, 0))
    _walls(parts, shape[0])
    with pic.Context([desc], precision=pic.PIC_FP64) as ctx:
        ctx.set_state(0, fields, parts)
        st = _oracle_state(desc, fields, parts, arr)
        for nsteps in (1, 4):
            ctx.step(nsteps)
            oracle.step(st, nsteps)
            f, p, step = ctx.get_state(0)
            _compare(desc, f, p, st, 1e-12, 1e-12 * max(shape), 1e-12)
            assert all(q[0].min() >= 0.0 and q[0].max() <= shape[0] for q in p)


# ----------------------------------------------------------------- mixed path

def _mixed_roundtrip(desc, fields, parts, arr, **kw):
    ctx = pic.Context([desc], precision=pic.PIC_MIXED, **kw)
    ctx.set_state(0, fields, parts)
    f0, p0, _ = ctx.get_state(0)
    return ctx, _oracle_state(desc, f0, p0, arr)


@pytest.mark.parametrize("ndim,shape,ppc", [(2, (64, 40, 1), 8), (3, (20, 16, 12), 4), (2, (7, 5, 1), 5)])
def test_mixed_one_step_matches_oracle(ndim, shape, ppc):
    desc, fields, parts, arr = _make(ndim, shape, ppc, seed=200 + ndim, spread=1.0, amp=0.05, colocate=False)
    ctx, st = _mixed_roundtrip(desc, fields, parts, arr)
    with ctx:
        ctx.step(1)
        f, p, _ = ctx.get_state(0)
    oracle.step(st)
    _compare(desc, f, p, st, 1e-5, 2e-6, 1e-5)


@pytest.mark.parametrize("ndim,shape", [(2, (48, 32, 1)), (3, (16, 16, 16))])
def test_mixed_neutral_start_gauss_residual(ndim, shape):
    desc, fields, parts, arr = _make(ndim, shape, 8, seed=300 + ndim, spread=1.0, amp=0.0, colocate=True)
    fields[3:] = np.random.default_rng(2).normal(0, 0.05, fields[3:].shape)
    with pic.Context([desc], precision=pic.PIC_MIXED) as ctx:
        ctx.set_state(0, fields, parts)
        ctx.step(1)
        d1 = ctx.diagnostics(0)
        ctx.step(19)
        d20 = ctx.diagnostics(0)
    assert d1["gauss_max"] <= 1e-6 * d1["rho_max"], d1
    # 20 steps, with re-sorts: still within the same bound
    assert d20["gauss_max"] <= 1e-6 * d20["rho_max"], d20


@pytest.mark.parametrize("ndim,shape,ppc,theta,n_x,rho_sp0,nsteps", [
    (3, (32, 32, 32), 32, 1.0, 1.0, 64.0, 1000),      # the 128^3 thermal plasma's parameters on a 32^3 box
    (2, (256, 256, 1), 50, 0.01, 20.0, 100.0, 2000),  # the 1024^2 filamentation box's parameters on 256^2
])
def test_mixed_gauss_residual_stays_below_1e6_over_a_long_run(ndim, shape, ppc, theta, n_x, rho_sp0, nsteps):
    """Charge conservation of the mixed path over the configured run lengths
    (1000 steps in 3D, 2000 in 2D), with the default sort interval: the Gauss
    residual max |div e - rho~| stays below 1e-6 of max |rho~_s|.  The fluxes
    are rounded once each (FP32 arithmetic, then 2^-26 fixed point), so the
    residual random-walks like sqrt(steps); e carries its FP32 rounding in a
    second FP32 word, which would otherwise add a drift growing linearly (it
    reached 5e-6 after 1000 steps before the pair was introduced)."""
    nx, ny, nz = shape
    n = ppc * nx * ny * nz
    desc = pic.run_desc(ndim, nx, ny, nz, n_x, rho_sp0, 0.5, [(-1.0, 1.0, n), (1.0, 1.0, n)])
    with pic.Context([desc], precision=pic.PIC_MIXED) as ctx:
        ctx.load_maxwell_juttner(0, 0, ppc, theta, (0.0, 0.0, 0.0), seed=11)
        ctx.load_maxwell_juttner(0, 1, ppc, theta, (0.0, 0.0, 0.0), colocate_with=0, seed=12)
        ratios = []
        for _ in range(4):
            ctx.step(nsteps // 4)
            d = ctx.diagnostics(0)
            ratios.append(d["gauss_max"] / d["rho_max"])
    print("gauss_max / rho_max at quarter points:", ["%.3e" % r for r in ratios])
    assert max(ratios) <= 1e-6, ratios


@pytest.mark.parametrize("sort_interval", [1, 4, 1000])
def test_mixed_multistep_with_sorting_and_halo_escape(sort_interval):
    """12 steps; with sort_interval = 1000 particles drift out of the staged
    halo of their tile and take the global slow path."""
    desc, fields, parts, arr = _make(2, (48, 40, 1), 6, seed=400, spread=3.0, amp=0.02, colocate=False)
    ctx, st = _mixed_roundtrip(desc, fields, parts, arr, sort_interval=sort_interval)
    with ctx:
        ctx.step(12)
        f, p, _ = ctx.get_state(0)
    oracle.step(st, 12)
    # FP32 vs FP64 over 12 steps: differences grow from 1e-7 per step
    _compare(desc, f, p, st, 2e-4, 1e-4, 2e-4)


@pytest.mark.parametrize("ndim,shape,ppc", [(2, (40, 24, 1), 8), (3, (16, 12, 10), 4)])
def test_mixed_conductor_walls_match_oracle(ndim, shape, ppc):
    """Conducting walls in x in the mixed path: reflected particles take the
    two-leg slow path; fields and particles after 1 and after 6 steps."""
    desc, fields, parts, arr = _make(ndim, shape, ppc, seed=220 + ndim, spread=2.0, amp=0.05, colocate=False,
                                     bc=(1, 0, 0))
    _walls(parts, shape[0])
    ctx, st = _mixed_roundtrip(desc, fields, parts, arr)
    with ctx:
        ctx.step(1)
        f, p, _ = ctx.get_state(0)
        oracle.step(st)
        _compare(desc, f, p, st, 1e-5, 2e-6, 1e-5)
        ctx.step(5)
        f, p, _ = ctx.get_state(0)
        oracle.step(st, 5)
        _compare(desc, f, p, st, 2e-4, 1e-4, 2e-4)
        assert all(q[0].min() >= 0.0 and q[0].max() <= shape[0] for q in p)


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED])
def test_set_state_rejects_bad_values_then_accepts_a_good_state(precision):
    """Values are validated on the device as they are converted: a non-finite
    momentum or field gives PIC_ENUMERIC, a position outside the domain
    PIC_EINVAL; the next valid state is accepted and steps normally."""
    desc, fields, parts, arr = _make(2, (16, 12, 1), 2, seed=51, spread=0.5, amp=0.01, colocate=False)
    with pic.Context([desc], precision=precision) as ctx:
        bad = [p.copy() for p in parts]
        bad[1][4, 3] = np.nan
        with pytest.raises(pic.PicError) as e:
            ctx.set_state(0, fields, bad)
        assert e.value.status == pic.PIC_ENUMERIC
        bad = [p.copy() for p in parts]
        bad[0][1, 5] = 12.0          # y = ny is outside [0, ny)
        with pytest.raises(pic.PicError) as e:
            ctx.set_state(0, fields, bad)
        assert e.value.status == pic.PIC_EINVAL
        badf = fields.copy()
        badf[4, 0, 2, 3] = np.inf
        with pytest.raises(pic.PicError) as e:
            ctx.set_state(0, badf, parts)
        assert e.value.status == pic.PIC_ENUMERIC
        ctx.set_state(0, fields, parts)
        ctx.step(2)
        d = ctx.diagnostics(0)
        assert d["nonfinite"] == 0


def test_mixed_empty_species_and_boundary_positions():
    desc, fields, parts, arr = _make(2, (32, 32, 1), 2, seed=5, spread=0.7, amp=0.03, colocate=False)
    n = parts[0].shape[1]
    # positions on node planes, on the periodic seam and just below a cell edge
    parts[0][0, :8] = [0.0, 1.0, 31.0, 31.999999999, 16.0, 0.5, 15.9999999999, 2.0]
    parts[0][1, :8] = [0.0, 31.99999999999, 5.0, 7.0, 16.0, 0.0, 3.0, 31.0]
    parts[1] = np.zeros((6, 0))
    desc.species[1].capacity = 0
    ctx, st = _mixed_roundtrip(desc, fields, parts, arr)
    st.species[1] = oracle.Species(np.zeros((3, 0)), np.zeros((3, 0)), 1.0, 1.0)
    with ctx:
        ctx.step(1)
        f, p, _ = ctx.get_state(0)
    oracle.step(st)
    assert p[1].shape == (6, 0)
    _compare(desc, f, p[:1] + [np.zeros((6, 0))], st, 1e-5, 2e-6, 1e-5)


def test_mixed_energy_history_tracks_oracle():
    desc, fields, parts, arr = _make(2, (32, 32, 1), 8, seed=11, spread=0.5, amp=0.0, colocate=True,
                                     species=ION_ELECTRON)
    ctx, st = _mixed_roundtrip(desc, fields, parts, arr)
    with ctx:
        ctx.step(10)
        hist = ctx.energy_history(0)
    assert hist.shape == (10, 4)
    # step 0 kinetic at t_0 is the average of the oracle's kinetic energy (pinned,
    # with the species masses) over u^{-1/2} and u^{1/2}
    ek_minus = oracle.energies(st)["kinetic"].sum()
    oracle.step(st)
    ek_plus = oracle.energies(st)["kinetic"].sum()
    assert np.isclose(hist[0, 0], 0.5 * (ek_minus + ek_plus), rtol=1e-5)
    assert np.all(np.isfinite(hist))


@pytest.mark.parametrize("precision", [pic.PIC_MIXED, pic.PIC_FP64])
def test_state_transfer_through_page_locked_buffers_equals_pageable(precision):
    """Page-locked host buffers are read and written by the conversion kernels
    directly; the transfers are bitwise those of the staged transfer of
    pageable buffers, and a bad value is still rejected.  After steps the mixed
    path stays bitwise equal (exact current); the FP64 path's global FP64
    atomics sum in a varying order, so two contexts agree to round-off."""
    torch = pytest.importorskip("torch")
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    desc, fields, parts, arr = _make(3, (20, 16, 12), 4, seed=77, spread=1.0, amp=0.05, colocate=False)
    with pic.Context([desc], precision=precision) as a, pic.Context([desc], precision=precision) as b:
        a.set_state(0, fields, parts)
        b.set_state(0, pin(fields), [pin(p) for p in parts])
        for nsteps in (0, 3):
            a.step(nsteps)
            b.step(nsteps)
            fa, pa, _ = a.get_state(0)
            out_f = pin(np.zeros_like(fa))
            out_p = [pin(np.zeros_like(p)) for p in pa]
            fb, pb, _ = b.get_state(0, out=(out_f, out_p))
            exact = nsteps == 0 or precision == pic.PIC_MIXED
            for x, y in [(fa, fb)] + list(zip(pa, pb)):
                if exact:
                    assert np.array_equal(x, y)
                else:
                    assert np.abs(x - y).max() <= 1e-12 * max(1.0, np.abs(y).max())
        bad = [pin(p) for p in parts]
        bad[0][4, 5] = np.inf
        with pytest.raises(pic.PicError) as e:
            b.set_state(0, pin(fields), bad)
        assert e.value.status == pic.PIC_ENUMERIC
