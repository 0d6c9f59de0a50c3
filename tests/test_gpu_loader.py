"""GPU parity of the Maxwell-Juttner loader (Sect. 4.3, App. D) with the oracle:
same Philox streams, so positions agree to rounding and momenta to the
accuracy of the two independent inversions of the cumulative marginal."""
import numpy as np
import pytest

import oracle
from oracle import mj
import paper_1308_5892_gb300 as pic

pytestmark = pytest.mark.gpu


def _ctx(ndim, shape, cap, precision, nsp=2):
    nx, ny, nz = shape
    d = pic.run_desc(ndim, nx, ny, nz if ndim == 3 else 1, 2.0, 16.0, 0.5, [(-1.0, 1.0, cap), (1.0, 1.0, cap)][:nsp])
    return pic.Context([d], precision=precision), d


@pytest.mark.parametrize("precision,ptol,utol", [(pic.PIC_FP64, 1e-12, 1e-9), (pic.PIC_MIXED, 4e-6, 1e-6)])
@pytest.mark.parametrize("theta,beta", [(1.0, (0.0, np.sqrt(2 / 3.0), 0.0)), (0.01, (0.0, 0.0, np.sqrt(8 / 9.0))),
                                        (0.1, (0.0, 0.0, 0.0)), (10.0, (0.5, 0.0, 0.6))])
def test_loader_matches_oracle(precision, ptol, utol, theta, beta):
    ndim, shape, ppc = 2, (24, 20, 1), 8
    n = ppc * 24 * 20
    ctx, d = _ctx(ndim, shape, n, precision)
    with ctx:
        ctx.load_maxwell_juttner(0, 0, ppc, theta, beta, seed=1234)
        ctx.load_maxwell_juttner(0, 1, ppc, theta, tuple(-b for b in beta), colocate_with=0, seed=99)
        f, p, _ = ctx.get_state(0)
    pos0, u0 = mj.load(1234, 0, n, theta, beta, ndim, *shape)
    _, u1 = mj.load(99, 1, n, theta, tuple(-b for b in beta), ndim, *shape)
    assert np.abs(p[0][:2] - pos0[:2]).max() <= ptol * 24
    assert np.array_equal(p[1][:3], p[0][:3])          # colocated pairs
    for got, ref in ((p[0][3:], u0), (p[1][3:], u1)):
        assert np.abs(got - ref).max() <= utol * max(1.0, np.abs(ref).max())


def test_naive_boost_and_harris_profile_match_oracle():
    ndim, shape = 2, (64, 16, 1)
    ctx, d = _ctx(ndim, shape, 200000, pic.PIC_FP64, nsp=1)
    L, x0 = 4.0, 32.0
    with ctx:
        ctx.load_maxwell_juttner(0, 0, 10.0, 1.0, (0.0, 0.8, 0.0), profile=pic.PIC_PROFILE_HARRIS,
                                 profile_params=(L, x0), method=pic.PIC_MJ_NAIVE_BOOST, seed=5)
        f, p, _ = ctx.get_state(0)
    n = mj.harris_count(10.0, 64, 16, 1, 2, L, x0)
    assert p[0].shape[1] == n
    pos, u = mj.load(5, 0, n, 1.0, (0.0, 0.8, 0.0), ndim, *shape, profile=1, L=L, x0=x0, method="naive")
    assert np.abs(p[0][:2] - pos[:2]).max() < 1e-10
    assert np.abs(p[0][3:] - u).max() < 1e-9 * np.abs(u).max()


def test_loader_staggers_momenta_back_half_a_step():
    """With a uniform b field the loaded momenta are u^{-dt/2}: one Boris step of -dt/2."""
    ndim, shape, ppc = 2, (16, 16, 1), 4
    n = ppc * 256
    ctx, d = _ctx(ndim, shape, n, pic.PIC_FP64, nsp=1)
    with ctx:
        ctx.set_uniform_field(0, (0.01, 0.0, 0.0), (0.0, 0.0, 0.3))
        ctx.load_maxwell_juttner(0, 0, ppc, 0.2, (0.0, 0.0, 0.0), seed=3)
        f, p, _ = ctx.get_state(0)
    pos, u = mj.load(3, 0, n, 0.2, (0.0, 0.0, 0.0), ndim, *shape)
    EB = np.zeros((6, n))
    EB[0] = 0.01
    EB[5] = 0.3
    ref = oracle.boris(u, EB, -1.0, -0.25)
    assert np.abs(p[0][3:] - ref).max() < 1e-9


def test_loader_moments_on_gpu_match_table_averages():
    theta, b0 = 1.0, 0.6
    ctx, d = _ctx(3, (32, 32, 32), 32 * 32768, pic.PIC_MIXED, nsp=1)
    with ctx:
        ctx.load_maxwell_juttner(0, 0, 32, theta, (0.0, 0.0, b0), seed=21)
        ids = np.arange(0, 32 * 32768, 7)
        p = ctx.get_particles(0, 0, ids)
    u = p[3:]
    g = np.sqrt(1 + (u ** 2).sum(0))
    m = mj.moments(theta, b0)
    n = u.shape[1]
    for k, x in {"gamma": g, "gamma_v_par": u[2], "pv_perp": u[0] * u[0] / g, "pv_par": u[2] * u[2] / g}.items():
        assert abs(x.mean() - m[k]) < 4 * x.std() / np.sqrt(n) + 1e-6, (k, x.mean(), m[k])


def test_invalid_loader_arguments():
    ctx, d = _ctx(2, (8, 8, 1), 100, pic.PIC_FP64)
    with ctx:
        for kw in (dict(theta=-1.0), dict(beta=(0.0, 1.0, 0.0)), dict(ppc=1000.0), dict(profile=7),
                   dict(method=9), dict(colocate_with=0)):
            args = dict(ppc=1.0, theta=0.1, beta=(0.0, 0.0, 0.0))
            args.update(kw)
            with pytest.raises(pic.PicError):
                ctx.load_maxwell_juttner(0, 0, **args)
