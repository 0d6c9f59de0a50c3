"""Batched ensemble (many independent runs in one context, one persistent push
launch per step) and the autotuner.  Both are checked for exactness: an
ensemble member must be bitwise identical to the same run advanced alone, and
a run advanced under the autotuner's trials must be bitwise identical to the
same run advanced with the default tuning (each particle's arithmetic is the
same and the current is an exact fixed-point sum)."""
import numpy as np
import pytest

import paper_1308_5892_gb300 as pic

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
