"""FP64 oracle of the sampler network (TEST INFRASTRUCTURE, see oracle/__init__).

The network of the learned loader: 3 -> 64 -> 64 -> 64 -> 1, tanh hidden
layers, linear output, loss = mean (o - target)^2.  Parameters flat in the
order W1[64][3] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4.  Plain
numpy forward and reverse-mode gradient, checked against central finite
differences in the tests.
"""
import numpy as np
from scipy import special

H = 64
NP = H * 3 + H + H * H + H + H * H + H + H + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = []
    for shape in ((H, 3), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)):
        n = int(np.prod(shape))
        out.append(p[o:o + n].reshape(shape))
        o += n
    return out


def forward(p, x):
    """x: (3, n) -> outputs (n,) and the activations."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    a1 = np.tanh(W1 @ x + b1[:, None])
    a2 = np.tanh(W2 @ a1 + b2[:, None])
    a3 = np.tanh(W3 @ a2 + b3[:, None])
    o = W4 @ a3 + b4[0]
    return o, (a1, a2, a3)


def loss_and_grad(p, x, t):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    n = x.shape[1]
    o, (a1, a2, a3) = forward(p, x)
    e = o - t
    loss = np.mean(e * e)
    d4 = 2.0 * e / n
    gW4 = a3 @ d4
    gb4 = np.array([d4.sum()])
    d3 = (W4[:, None] * d4[None, :]) * (1 - a3 * a3)
    gW3 = d3 @ a2.T
    gb3 = d3.sum(1)
    d2 = (W3.T @ d3) * (1 - a2 * a2)
    gW2 = d2 @ a1.T
    gb2 = d2.sum(1)
    d1 = (W2.T @ d2) * (1 - a1 * a1)
    gW1 = d1 @ x.T
    gb1 = d1.sum(1)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3, gW4, gb4])
    return loss, g


def features(theta, beta0, w):
    """Network inputs of the learned loader."""
    return np.stack([np.full_like(w, (np.log10(theta) + 0.5) / 1.5), np.full_like(w, 2 * beta0 / 0.95 - 1),
                     special.ndtri(w) / 3.0])
