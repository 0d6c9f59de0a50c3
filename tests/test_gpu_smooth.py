"""Current smoothing (App. A.3.4, main-loop step 10) on the GPU.

The smoothed step of both paths is compared with the oracle's smoothed step on
the same seeded inputs, at the bars of the unsmoothed step: FP64 1e-12
norm-wise; mixed 1e-5 after one step.  With smoothing the conserved residual is
div e - S rho~ (S the smoothing), which the diagnostics report; it must stay at
round-off from a neutral start.  The mixed current is an exact fixed-point sum
folded before the smoothing, so graph replays and ensemble members stay
bitwise equal to direct launches and single runs.
"""
import numpy as np
import pytest

import oracle
import paper_1308_5892_gb300 as pic
import synth

pytestmark = pytest.mark.gpu


def _make(ndim, shape, ppc, seed, passes, spread=2.0, amp=0.05, colocate=False, n_x=2.0, rho_sp0=8.0):
    nx, ny, nz = shape
    arr = synth.random_state_arrays(seed, ndim, nx, ny, nz, ppc=ppc, spread=spread, amp_e=amp, amp_b=amp,
                                    colocate=colocate)
    n = arr["species"][0]["pos"].shape[1]
    desc = pic.run_desc(ndim, nx, ny, nz if ndim == 3 else 1, n_x, rho_sp0, 0.5,
                        [(s["q_over_e"], s["m_over_me"], n) for s in arr["species"]], smooth_passes=passes)
    fields = np.concatenate([arr["e"], arr["b"]])
    parts = [np.concatenate([s["pos"], s["u"]]) for s in arr["species"]]
    return desc, fields, parts, arr


def _oracle_state(desc, fields, parts, arr):
    st = oracle.State.empty(desc.ndim, desc.nx, desc.ny, desc.nz, desc.dt, desc.n_x, desc.rho_sp0,
                            smooth_passes=desc.smooth_passes)
    st.e[:] = fields[:3]
    st.b[:] = fields[3:]
    for s, p in zip(arr["species"], parts):
        st.species.append(oracle.Species(np.ascontiguousarray(p[:3]), np.ascontiguousarray(p[3:]),
                                         s["q_over_e"], s["m_over_me"]))
    return st


def _rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / den if den > 0 else np.abs(a - b).max()


def _compare(desc, f_gpu, p_gpu, st, tol_field, tol_pos, tol_u):
    ref_f = np.concatenate([st.e, st.b])
    for c in range(6):
        assert _rel(f_gpu[c], ref_f[c]) <= tol_field, ("field component", c, _rel(f_gpu[c], ref_f[c]))
    L = [desc.nx, desc.ny, desc.nz]
    for s, sp in enumerate(st.species):
        for a in range(desc.ndim):
            d = p_gpu[s][a] - sp.pos[a]
            assert np.abs(d - L[a] * np.round(d / L[a])).max() <= tol_pos, ("position", s, a)
        for a in range(3):
            assert _rel(p_gpu[s][3 + a], sp.u[a]) <= tol_u, ("momentum", s, a)


@pytest.mark.parametrize("ndim,shape,ppc,passes",
                         [(2, (33, 20, 1), 4, 1), (3, (12, 10, 9), 3, 1), (2, (24, 18, 1), 4, 2), (3, (10, 9, 8), 3, 4)])
def test_fp64_smoothed_steps_match_oracle_to_1e12(ndim, shape, ppc, passes):
    desc, fields, parts, arr = _make(ndim, shape, ppc, 900 + 10 * ndim + passes, passes)
    with pic.Context([desc], precision=pic.PIC_FP64) as ctx:
        ctx.set_state(0, fields, parts)
        st = _oracle_state(desc, fields, parts, arr)
        for nsteps in (1, 3):
            ctx.step(nsteps)
            oracle.step(st, nsteps)
            f, p, _ = ctx.get_state(0)
            _compare(desc, f, p, st, 1e-12, 1e-12 * max(shape), 1e-12)
        d = ctx.diagnostics(0)
    # the diagnostics' residual is div e - S^P rho~, as in the oracle
    g, rmax = oracle.gauss_residual(_oracle_state(desc, f, p, arr))
    assert abs(d["gauss_max"] - g) <= 1e-12 * rmax


@pytest.mark.parametrize("ndim,shape,ppc,passes",
                         [(2, (64, 40, 1), 8, 1), (3, (20, 16, 12), 4, 1), (2, (37, 29, 1), 5, 2)])
def test_mixed_smoothed_steps_match_oracle(ndim, shape, ppc, passes):
    desc, fields, parts, arr = _make(ndim, shape, ppc, 950 + 10 * ndim + passes, passes, spread=1.0)
    with pic.Context([desc], precision=pic.PIC_MIXED) as ctx:
        ctx.set_state(0, fields, parts)
        f0, p0, _ = ctx.get_state(0)
        st = _oracle_state(desc, f0, p0, arr)
        ctx.step(1)
        f, p, _ = ctx.get_state(0)
        oracle.step(st)
        _compare(desc, f, p, st, 1e-5, 2e-6, 1e-5)
        ctx.step(5)
        f, p, _ = ctx.get_state(0)
        oracle.step(st, 5)
        _compare(desc, f, p, st, 2e-4, 1e-4, 2e-4)


@pytest.mark.parametrize("precision,bound", [(pic.PIC_FP64, 1e-12), (pic.PIC_MIXED, 1e-6)])
@pytest.mark.parametrize("ndim,shape", [(2, (48, 32, 1)), (3, (16, 16, 16))])
def test_smoothed_neutral_start_keeps_the_smoothed_gauss_law(precision, bound, ndim, shape):
    desc, fields, parts, arr = _make(ndim, shape, 8, 980 + ndim, 2, spread=1.0, amp=0.0, colocate=True)
    fields[3:] = np.random.default_rng(3).normal(0, 0.05, fields[3:].shape)
    with pic.Context([desc], precision=precision) as ctx:
        ctx.set_state(0, fields, parts)
        ctx.step(20)
        d = ctx.diagnostics(0)
    assert d["gauss_max"] <= bound * d["rho_max"], d


def test_smoothed_graph_replay_and_ensemble_are_bitwise_equal():
    runs = [((40, 24), 6, 0), ((32, 32), 8, 1), ((24, 40), 4, 2)]
    made = [_make(2, (nx, ny, 1), ppc, 990 + i, passes, spread=1.0, amp=0.03)
            for i, ((nx, ny), ppc, passes) in enumerate(runs)]
    # one run, graph replay against direct launches
    out = {}
    for name, flags in (("graph", 0), ("direct", pic.PIC_FLAG_NO_GRAPH)):
        desc, fields, parts, _ = made[2]
        with pic.Context([desc], precision=pic.PIC_MIXED, sort_interval=2, flags=flags) as ctx:
            ctx.set_state(0, fields, parts)
            ctx.step(13)
            out[name] = ctx.get_state(0)
    for a, b in zip(out["graph"][1], out["direct"][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(out["graph"][0], out["direct"][0])
    # an ensemble of runs with 0, 1 and 2 passes against the runs advanced alone
    with pic.Context([m[0] for m in made], precision=pic.PIC_MIXED, sort_interval=2) as ens:
        for r, (desc, fields, parts, _) in enumerate(made):
            ens.set_state(r, fields, parts)
        ens.step(9)
        got = [ens.get_state(r) for r in range(len(made))]
    for r, (desc, fields, parts, _) in enumerate(made):
        with pic.Context([desc], precision=pic.PIC_MIXED, sort_interval=2) as one:
            one.set_state(0, fields, parts)
            one.step(9)
            f, p, _ = one.get_state(0)
        assert np.array_equal(f, got[r][0]), r
        for s in range(2):
            assert np.array_equal(p[s], got[r][1][s]), (r, s)


def test_smoothing_lowers_the_thermal_field_fluctuations():
    """The smoothing damps the short-wavelength part of the current (App.
    A.3.4): the electric fluctuation energy of a thermal plasma drops."""
    nx = ny = 64
    ppc, theta = 16, 0.1
    n = ppc * nx * ny
    level = {}
    for passes in (0, 1):
        d = pic.run_desc(2, nx, ny, 1, theta ** -0.5, 2.0 * ppc, 0.5, [(-1.0, 1.0, n), (1.0, 1.0, n)],
                         smooth_passes=passes)
        with pic.Context([d], precision=pic.PIC_MIXED) as ctx:
            ctx.load_maxwell_juttner(0, 0, ppc, theta, (0.0, 0.0, 0.0), seed=11)
            ctx.load_maxwell_juttner(0, 1, ppc, theta, (0.0, 0.0, 0.0), colocate_with=0, seed=12)
            ctx.step(200)
            h = ctx.energy_history(0)
        level[passes] = h[100:, 1].mean()
    assert level[1] < 0.7 * level[0], level
