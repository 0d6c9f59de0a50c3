"""The FP64 oracle network: gradients against central finite differences."""
import numpy as np

from oracle import mlp


def test_oracle_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    p = rng.normal(0, 0.3, mlp.NP)
    x = rng.normal(0, 1, (3, 37))
    t = rng.normal(0, 1, 37)
    loss, g = mlp.loss_and_grad(p, x, t)
    idx = rng.choice(mlp.NP, 120, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, x, t)[0] - mlp.loss_and_grad(pm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_oracle_forward_shapes_and_linear_output_layer():
    p = np.zeros(mlp.NP)
    p[-1] = 0.25                        # b4
    o, _ = mlp.forward(p, np.zeros((3, 5)))
    assert np.allclose(o, 0.25)
