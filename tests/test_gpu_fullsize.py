"""Parity at the benchmark's full size (3D3V, 128^3 cells, 32 particles per cell
per species, theta = 1, default tuning as timed by bench.py), on outputs the
oracle computes one by one: sampled loaded particles, sampled particles after
one step (gather from the downloaded fields, Boris, move), and the Gauss
residual, a property that holds at any size."""
import numpy as np
import pytest

import oracle
from oracle import mj
import paper_1308_5892_gb300 as pic

pytestmark = pytest.mark.gpu

N = 128
PPC = 32


@pytest.fixture(scope="module")
def loaded():
    n = PPC * N ** 3
    d = pic.run_desc(3, N, N, N, 1.0, 64.0, 0.5, [(-1.0, 1.0, n), (1.0, 1.0, n)])
    ctx = pic.Context([d], precision=pic.PIC_MIXED)
    ctx.load_maxwell_juttner(0, 0, PPC, 1.0, (0.0, 0.0, 0.0), seed=2)
    ctx.load_maxwell_juttner(0, 1, PPC, 1.0, (0.0, 0.0, 0.0), colocate_with=0, seed=3)
    yield ctx, d, n
    ctx.close()


def test_full_size_loaded_sample_matches_oracle(loaded):
    ctx, d, n = loaded
    rng = np.random.default_rng(0)
    ids = np.sort(rng.choice(n, 3000, replace=False))
    for s, seed in ((0, 2), (1, 3)):
        got = ctx.get_particles(0, s, ids)
        w = mj.uniforms(seed, s, ids)
        u = mj.sample_momenta(w[3], w[4], w[5], 1.0, np.zeros(3))
        assert np.abs(got[3:] - u).max() <= 1e-6 * max(1.0, np.abs(u).max())
    w0 = mj.uniforms(2, 0, ids)
    p0 = ctx.get_particles(0, 0, ids)
    assert np.abs(p0[:3] - N * w0[:3]).max() < 4e-5


def test_full_size_step_sampled_particles_and_gauss(loaded):
    ctx, d, n = loaded
    ctx.step(3)                                   # let fields grow out of the noise
    fields, counts, _ = ctx.get_state(0, fields_only=True)
    rng = np.random.default_rng(1)
    ids = np.sort(rng.choice(n, 2000, replace=False))
    before = [ctx.get_particles(0, s, ids) for s in range(2)]
    ctx.step(1)
    after = [ctx.get_particles(0, s, ids) for s in range(2)]
    dg = ctx.diagnostics(0)
    assert dg["gauss_max"] <= 1e-6 * dg["rho_max"], dg
    st = oracle.State.empty(3, N, N, N, 0.5, 1.0, 64.0)
    st.e[:] = fields[:3]
    st.b[:] = fields[3:]
    oracle.b_advance(st, 0.25)                    # b^{t-dt/2} -> b^t for the gather
    for s, h in ((0, -1.0), (1, 1.0)):
        pos = before[s][:3].copy()
        EB = oracle.gather(st, pos)
        u = oracle.boris(before[s][3:], EB, h, 0.5)
        g = np.sqrt(1 + (u ** 2).sum(0))
        x = (pos + 0.5 * u / g) % N
        assert np.abs(after[s][3:] - u).max() <= 2e-5 * np.abs(u).max()
        dx = after[s][:3] - x
        dx -= N * np.round(dx / N)
        assert np.abs(dx).max() < 1e-5
