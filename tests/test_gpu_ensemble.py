"""Batched ensemble (many independent runs in one context, one persistent
launch per step: the step walker) and the autotuner.  Both are checked for exactness: an
ensemble member must be bitwise identical to the same run advanced alone, and
a run advanced under the autotuner's trials must be bitwise identical to the
same run advanced with the default tuning (each particle's arithmetic is the
same and the current is an exact fixed-point sum).  Each member of an
ensemble is also compared with the FP64 oracle stepped from its own uploaded
(FP32-rounded) state, at the mixed path's parity bars."""
import time

import numpy as np
import pytest

import oracle
import paper_1308_5892_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

RUNS = [  # nx, ny, ppc per species, theta
    (32, 48, 4, 0.01), (40, 40, 16, 0.1), (64, 32, 8, 1.0), (48, 80, 32, 0.3), (33, 35, 6, 0.05)]


def _desc(nx, ny, ppc):
    n = ppc * nx * ny
    return pic.run_desc(2, nx, ny, 1, 3.0, 2.0 * ppc, 0.5, [(-1.0, 1.0, n), (1.0, 1.0, n)])


def _load(ctx, run, ppc, theta, seed):
    ctx.load_maxwell_juttner(run, 0, ppc, theta, (0.0, 0.0, 0.0), seed=seed)
    ctx.load_maxwell_juttner(run, 1, ppc, theta, (0.0, 0.0, 0.0), colocate_with=0, seed=seed + 1)


def test_ensemble_members_equal_single_runs_bitwise():
    descs = [_desc(nx, ny, ppc) for nx, ny, ppc, th in RUNS]
    with pic.Context(descs, precision=pic.PIC_MIXED) as ens:
        for r, (nx, ny, ppc, th) in enumerate(RUNS):
            _load(ens, r, ppc, th, 100 + 2 * r)
        ens.step(12)
        got = [ens.get_state(r) for r in range(len(RUNS))]
        dg = [ens.diagnostics(r) for r in range(len(RUNS))]
    for r, (nx, ny, ppc, th) in enumerate(RUNS):
        with pic.Context([descs[r]], precision=pic.PIC_MIXED) as one:
            _load(one, 0, ppc, th, 100 + 2 * r)
            one.step(12)
            f, p, step = one.get_state(0)
        assert step == got[r][2] == 12
        assert np.array_equal(f, got[r][0]), r
        for s in range(2):
            assert np.array_equal(p[s], got[r][1][s]), (r, s)
        assert dg[r]["gauss_max"] <= 1e-6 * dg[r]["rho_max"]


def test_autotuned_run_is_bitwise_equal_to_default_run():
    nx, ny, ppc, th = 96, 64, 24, 0.2
    d = _desc(nx, ny, ppc)
    with pic.Context([d], precision=pic.PIC_MIXED) as a:
        _load(a, 0, ppc, th, 7)
        choice = a.autotune(max_steps=120)
        n = choice["steps_taken"]
        assert n > 0
        a.step(10)
        fa, pa, sa = a.get_state(0)
        tuning = a.tuning()
    assert tuning["tile"] == choice["tile"] and tuning["sort_interval"] == choice["sort_interval"]
    with pic.Context([d], precision=pic.PIC_MIXED) as b:
        _load(b, 0, ppc, th, 7)
        b.step(n + 10)
        fb, pb, sb = b.get_state(0)
    assert sa == sb == n + 10
    assert np.array_equal(fa, fb)
    for s in range(2):
        assert np.array_equal(pa[s], pb[s])


# (nx, ny, particles per cell per species, field amplitude, smoothing passes)
ORACLE_RUNS = [(32, 48, 4, 0.05, 0), (41, 37, 7, 0.02, 1), (64, 32, 3, 0.05, 0), (24, 56, 9, 0.03, 2),
               (35, 33, 5, 0.05, 0)]
WALL_RUNS = [(40, 32, 4, 0.03, 0), (29, 47, 6, 0.05, 0), (48, 24, 3, 0.02, 0)]


def _rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / den if den > 0 else np.abs(a - b).max()


def _member_vs_oracle(f, p, st, tol_field, tol_pos, tol_u, label):
    ref = np.concatenate([st.e, st.b])
    for c in range(6):
        assert _rel(f[c], ref[c]) <= tol_field, (label, "field", c, _rel(f[c], ref[c]))
    L = (st.nx, st.ny)
    for s, sp in enumerate(st.species):
        for a in range(2):
            d = p[s][a] - sp.pos[a]
            if not (a == 0 and st.bc_x == oracle.BC_CONDUCTOR):
                d = d - L[a] * np.round(d / L[a])
            assert np.abs(d).max() <= tol_pos, (label, "position", s, a, np.abs(d).max())
        for a in range(3):
            assert _rel(p[s][3 + a], sp.u[a]) <= tol_u, (label, "momentum", s, a)


@pytest.mark.parametrize("walls", [False, True])
def test_ensemble_members_match_oracle(walls):
    """Uneven members (grids 24..64 cells per side, 3..9 particles per cell per
    species, random fields and momenta, two members with current smoothing of
    1 and 2 passes in the periodic ensemble; an ensemble between conducting
    x-walls, App. A.4) advanced together by the batched kernels.  Every member
    matches the oracle stepped from its own uploaded state: after 1 step at
    the mixed bars (fields 1e-5 relative, positions 2e-6 cells, momenta 1e-5
    relative), after 12 steps with re-sorts at 2e-4 (FP32 and FP64
    trajectories separate by about 1e-7 per step)."""
    runs = WALL_RUNS if walls else ORACLE_RUNS
    bc = (1, 0, 0) if walls else (0, 0, 0)
    descs, states = [], []
    for r, (nx, ny, ppc, amp, sm) in enumerate(runs):
        arr = synth.random_state_arrays(500 + r, 2, nx, ny, 1, ppc=ppc, spread=0.6, amp_e=amp, amp_b=amp,
                                        colocate=False)
        n = arr["species"][0]["pos"].shape[1]
        descs.append(pic.run_desc(2, nx, ny, 1, 2.0, 8.0, 0.5, [(-1.0, 1.0, n), (1.0, 1.0, n)], bc=bc,
                                  smooth_passes=sm))
        states.append((np.concatenate([arr["e"], arr["b"]]), [np.concatenate([sp["pos"], sp["u"]])
                                                              for sp in arr["species"]]))
    with pic.Context(descs, precision=pic.PIC_MIXED, sort_interval=4) as ens:
        for r, (fields, parts) in enumerate(states):
            ens.set_state(r, fields, parts)
        refs = []
        for r, d in enumerate(descs):
            f0, p0, _ = ens.get_state(r)
            st = oracle.State.empty(2, d.nx, d.ny, 1, d.dt, d.n_x, d.rho_sp0, bc_x=d.bc[0],
                                    smooth_passes=d.smooth_passes)
            st.e[:] = f0[:3]
            st.b[:] = f0[3:]
            for s, q in zip(range(2), (-1.0, 1.0)):
                st.species.append(oracle.Species(np.ascontiguousarray(p0[s][:3]), np.ascontiguousarray(p0[s][3:]),
                                                 q, 1.0))
            refs.append(st)
        ens.step(1)
        for r, st in enumerate(refs):
            oracle.step(st)
            f, p, step = ens.get_state(r)
            assert step == 1
            _member_vs_oracle(f, p, st, 1e-5, 2e-6, 1e-5, (walls, r, 1))
        ens.step(11)
        for r, st in enumerate(refs):
            oracle.step(st, 11)
            f, p, step = ens.get_state(r)
            assert step == 12
            _member_vs_oracle(f, p, st, 2e-4, 2e-4, 2e-4, (walls, r, 12))



def _random_ensemble(runs, bc, seed0):
    """runs: (nx, ny, ppc, amp, smoothing passes) for 2D3V members, (nx, ny, nz, ppc, amp,
    smoothing passes) for 3D3V members."""
    descs, states = [], []
    for r, run in enumerate(runs):
        if len(run) == 5:
            (nx, ny, ppc, amp, sm), nz, ndim = run, 1, 2
        else:
            (nx, ny, nz, ppc, amp, sm), ndim = run, 3
        arr = synth.random_state_arrays(seed0 + r, ndim, nx, ny, nz, ppc=ppc, spread=0.6, amp_e=amp, amp_b=amp,
                                        colocate=False)
        n = arr["species"][0]["pos"].shape[1]
        descs.append(pic.run_desc(ndim, nx, ny, nz, 2.0, 8.0, 0.5, [(-1.0, 1.0, n), (1.0, 1.0, n)], bc=bc,
                                  smooth_passes=sm))
        states.append((np.concatenate([arr["e"], arr["b"]]), [np.concatenate([sp["pos"], sp["u"]])
                                                              for sp in arr["species"]]))
    return descs, states


# members of similar size: no run holds a quarter of the particles, so the walker also runs the re-sorts
BALANCED_RUNS = [(40, 40, 6, 0.03, 0), (44, 36, 6, 0.05, 1), (36, 44, 6, 0.04, 0), (48, 32, 6, 0.05, 2),
                 (32, 48, 6, 0.02, 0), (40, 38, 6, 0.04, 0)]
BALANCED_WALL_RUNS = [(40, 32, 5, 0.03, 0), (36, 36, 5, 0.05, 0), (32, 40, 5, 0.02, 0), (38, 34, 5, 0.04, 0),
                      (34, 38, 5, 0.03, 0)]
BALANCED_3D_RUNS = [(16, 16, 12, 3, 0.03, 0), (12, 16, 16, 3, 0.05, 1), (16, 12, 16, 3, 0.04, 0),
                    (14, 14, 14, 3, 0.05, 0), (16, 16, 10, 3, 0.02, 0)]


@pytest.mark.parametrize("case", ["balanced", "balanced_walls", "balanced_3d", "dominated"])
def test_step_walker_equals_phase_launches_bitwise(case):
    """The step walker (every phase of every run in one persistent launch,
    with per-run dependencies) and one batched launch per phase advance the
    same uneven ensemble to bitwise the same fields and particles: 14 steps
    with re-sorts every 4 steps, graph replay on.  In the balanced ensembles
    (periodic, with members of 1 and 2 smoothing passes; conducting x-walls;
    3D3V members, one of which also matches its single-run context bitwise)
    the walker runs the re-sorts too and queues one kernel launch per step; in
    the ensemble where one run holds over a quarter of the particles the
    sorts run as launches per phase and the walker does the rest.  The phase
    launches queue five or more per step.  The energy histories agree to 1e-6
    (the kinetic energy is summed in FP32 per block of particles, whose order
    inside a cell the sort's atomics set)."""
    runs, walls = {"balanced": (BALANCED_RUNS, False), "balanced_walls": (BALANCED_WALL_RUNS, True),
                   "balanced_3d": (BALANCED_3D_RUNS, False), "dominated": (ORACLE_RUNS, False)}[case]
    descs, states = _random_ensemble(runs, (1, 0, 0) if walls else (0, 0, 0), 700)
    out = []
    for flags in (0, pic.PIC_FLAG_PHASE_LAUNCHES):
        with pic.Context(descs, precision=pic.PIC_MIXED, sort_interval=4, flags=flags) as ens:
            for r, (fields, parts) in enumerate(states):
                ens.set_state(r, fields, parts)
            ens.step(14)
            launches = ens.counters()["launches_per_step"]
            out.append(([ens.get_state(r) for r in range(len(runs))],
                        [ens.energy_history(r) for r in range(len(runs))], launches))
    (walk, hw, lw), (phase, hp, lp) = out
    for r in range(len(runs)):
        assert walk[r][2] == phase[r][2] == 14
        assert np.array_equal(walk[r][0], phase[r][0]), r
        for s in range(2):
            assert np.array_equal(walk[r][1][s], phase[r][1][s]), (r, s)
        # the order of the particles inside a cell (set by the sort's atomics) changes
        # the FP32 partial sums of the kinetic energy at the 1e-8 level
        np.testing.assert_allclose(hw[r], hp[r], rtol=1e-6, atol=0)
    assert lp >= 5 and (lw == 1 if case != "dominated" else 1 <= lw < lp), (lw, lp)
    if case == "balanced_3d":
        # a 3D member advanced alone (one CTA per tile, separate kernels) gives the same bits
        with pic.Context([descs[1]], precision=pic.PIC_MIXED, sort_interval=4) as one:
            one.set_state(0, *states[1])
            one.step(14)
            f, p, _ = one.get_state(0)
        assert np.array_equal(f, walk[1][0])
        for s in range(2):
            assert np.array_equal(p[s], walk[1][1][s])


def test_step_walker_bounded_wait_reports_timeout():
    """A dependency that never completes (PIC_FLAG_INJECT_STALL: the push of run
    0 waits for one item more than exist) makes the walker's bounded wait run
    out after 20 ms: pic_step returns PIC_ETIMEOUT within seconds, nothing
    faults, and the context stays usable: the states set again afterwards step
    to bitwise the result of a fresh context."""
    descs, states = _random_ensemble(ORACLE_RUNS[:3], (0, 0, 0), 900)
    with pic.Context(descs, precision=pic.PIC_MIXED, sort_interval=4,
                     flags=pic.PIC_FLAG_INJECT_STALL | pic.PIC_FLAG_NO_GRAPH) as ens:
        for r, (fields, parts) in enumerate(states):
            ens.set_state(r, fields, parts)
        t0 = time.time()
        with pytest.raises(pic.PicError) as ei:
            ens.step(1)
        assert ei.value.status == pic.PIC_ETIMEOUT
        assert time.time() - t0 < 10.0
        ens.set_flags(0)
        for r, (fields, parts) in enumerate(states):
            ens.set_state(r, fields, parts)
        ens.step(5)
        got = [ens.get_state(r) for r in range(len(descs))]
    with pic.Context(descs, precision=pic.PIC_MIXED, sort_interval=4) as ref:
        for r, (fields, parts) in enumerate(states):
            ref.set_state(r, fields, parts)
        ref.step(5)
        want = [ref.get_state(r) for r in range(len(descs))]
    for r in range(len(descs)):
        assert np.array_equal(got[r][0], want[r][0]), r
        for s in range(2):
            assert np.array_equal(got[r][1][s], want[r][1][s]), (r, s)


def test_step_walker_with_empty_species_and_runs():
    """Degenerate members in a walker ensemble: one run's positron species is
    empty (capacity 0) and another run holds no particles at all.  Over 9
    steps with re-sorts every 2 steps the walker and the launches per phase
    give bitwise the same fields and particles, and the empty species stay
    empty.  No run holds a quarter of the particles, so the walker sorts too."""
    runs = BALANCED_RUNS
    descs, states = _random_ensemble(runs, (0, 0, 0), 800)
    descs[1].species[1].capacity = 0
    states[1] = (states[1][0], [states[1][1][0], np.zeros((6, 0))])
    for q in range(2):
        descs[3].species[q].capacity = 0
    states[3] = (states[3][0], [np.zeros((6, 0)), np.zeros((6, 0))])
    out = []
    for flags in (0, pic.PIC_FLAG_PHASE_LAUNCHES):
        with pic.Context(descs, precision=pic.PIC_MIXED, sort_interval=2, flags=flags) as ens:
            for r, (fields, parts) in enumerate(states):
                ens.set_state(r, fields, parts)
            ens.step(9)
            out.append([ens.get_state(r) for r in range(len(runs))])
    walk, phase = out
    for r in range(len(runs)):
        assert np.array_equal(walk[r][0], phase[r][0]), r
        for s in range(2):
            assert np.array_equal(walk[r][1][s], phase[r][1][s]), (r, s)
    assert walk[1][1][1].shape == (6, 0) and walk[3][1][0].shape == (6, 0) and walk[3][1][1].shape == (6, 0)
    assert np.all(np.isfinite(walk[3][0]))
