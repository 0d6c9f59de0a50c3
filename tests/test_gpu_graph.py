"""CUDA-graph replay of the mixed step.

pic_step captures one period of 2K steps (K = sort interval) as a CUDA graph
once the step sequence is in phase, and replays it while the host state
matches the capture.  Replayed steps must be bitwise identical to the same
steps launched directly (PIC_FLAG_NO_GRAPH): the graph holds the same kernels
with the same arguments, and the current is an exact fixed-point sum.  A state
change (pic_set_state) between replays must be honoured.
"""
import numpy as np
import pytest

import paper_1308_5892_gb300 as pic
import synth

pytestmark = pytest.mark.gpu


def _state(ndim, shape, ppc, seed):
    nx, ny, nz = shape
    arr = synth.random_state_arrays(seed, ndim, nx, ny, nz, ppc=ppc, spread=1.0, amp_e=0.03, amp_b=0.03,
                                    colocate=False)
    n = arr["species"][0]["pos"].shape[1]
    desc = pic.run_desc(ndim, nx, ny, nz if ndim == 3 else 1, 2.0, 8.0, 0.5,
                        [(s["q_over_e"], s["m_over_me"], n) for s in arr["species"]])
    fields = np.concatenate([arr["e"], arr["b"]])
    parts = [np.concatenate([s["pos"], s["u"]]) for s in arr["species"]]
    return desc, fields, parts


def _same(a, b):
    fa, pa, sa = a
    fb, pb, sb = b
    assert sa == sb
    assert np.array_equal(fa, fb)
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("ndim,shape,K", [(2, (48, 40, 1), 2), (3, (16, 16, 12), 1), (2, (33, 21, 1), 4)])
def test_graph_replay_is_bitwise_equal_to_direct_launches(ndim, shape, K):
    desc, fields, parts = _state(ndim, shape, 6, seed=600 + ndim + K)
    out = {}
    for name, flags in (("graph", 0), ("direct", pic.PIC_FLAG_NO_GRAPH)):
        with pic.Context([desc], precision=pic.PIC_MIXED, sort_interval=K, flags=flags) as ctx:
            ctx.set_state(0, fields, parts)
            ctx.step(3)
            ctx.step(4 * K + 3)          # capture, replays and a remainder
            s1 = ctx.get_state(0)
            h1 = ctx.energy_history(0)
            # a new state mid-run: later replays must start from it
            ctx.set_state(0, fields, parts)
            ctx.step(6 * K + 1)
            s2 = ctx.get_state(0)
            h2 = ctx.energy_history(0)
        out[name] = (s1, h1, s2, h2)
    g, d = out["graph"], out["direct"]
    _same(g[0], d[0])
    _same(g[2], d[2])
    for hg, hd in ((g[1], d[1]), (g[3], d[3])):
        assert hg.shape == hd.shape
        # the order of the particles inside a cell (set by the sort's atomics) changes
        # the FP32 partial sums of the kinetic energy at the 1e-8 level
        assert np.allclose(hg, hd, rtol=1e-6, atol=0)


def test_graph_replay_of_an_ensemble_is_bitwise_equal_to_direct_launches():
    runs = [(32, 24, 4), (40, 40, 8), (24, 56, 6)]
    descs, states = [], []
    for i, (nx, ny, ppc) in enumerate(runs):
        d, f, p = _state(2, (nx, ny, 1), ppc, seed=700 + i)
        descs.append(d)
        states.append((f, p))
    res = {}
    for name, flags in (("graph", 0), ("direct", pic.PIC_FLAG_NO_GRAPH)):
        with pic.Context(descs, precision=pic.PIC_MIXED, sort_interval=2, flags=flags) as ctx:
            for r, (f, p) in enumerate(states):
                ctx.set_state(r, f, p)
            ctx.step(17)
            res[name] = [ctx.get_state(r) for r in range(len(runs))]
    for a, b in zip(res["graph"], res["direct"]):
        _same(a, b)
