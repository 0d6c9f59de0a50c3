"""Oracle of the drifting Maxwell-Juttner loader (Sect. 4.3 and App. D of
Melzani et al., arXiv 1308.5892).  TEST INFRASTRUCTURE (see oracle/__init__).

Sampling of the distribution of Eq. Jutt, drift velocity beta0 along a unit
vector n, temperature theta = T/(m c^2), mu = 1/theta, Gamma0 = (1-beta0^2)^-1/2:
  1. the momentum along n, y, from its marginal j_Y (Eq. distr_y) by the exact
     inverse of its cumulative distribution, y = J^-1(w);
  2. u given y from the conditional of Eq. distr_u, solved as
     l(a_y u) = w' l(a_y), l(x) = (1 + x) exp(-x), a_y = mu Gamma0 sqrt(1+y^2)
     (Eq. finding_u), written for t = a_y (u - 1) and solved by bisection;
  3. r = sqrt(u^2 - 1), phi uniform, the perpendicular momenta gamma_y r (cos phi, sin phi),
     which undoes the change of variables of App. D.
Readings (listed in the design notes): w is a continuous uniform, not a random
table index; the cumulative distribution is integrated accurately instead of
by the step-halving scheme of App. D.

Random numbers: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC11, 2011), key =
the 64-bit seed, counter = (index low, index high, call, species); each
pair of 32-bit outputs gives one double in (0, 1).
"""
import numpy as np
from scipy import integrate, special

# ------------------------------------------------------------------ Philox

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32(ctr, key, rounds=10):
    """ctr: 4 arrays of uint32 (broadcastable), key: 2 uint32 scalars/arrays.
    Returns 4 uint32 arrays (the Philox-4x32 bijection of the counter)."""
    c = [np.asarray(x, dtype=np.uint64) & _MASK for x in ctr]
    k0 = np.asarray(key[0], dtype=np.uint64) & _MASK
    k1 = np.asarray(key[1], dtype=np.uint64) & _MASK
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [(hi1 ^ c[1] ^ k0) & _MASK, lo1, (hi0 ^ c[3] ^ k1) & _MASK, lo0]
    return [x.astype(np.uint32) for x in c]


def _to_double(hi, lo):
    """Two 32-bit words -> a double in (0, 1): (53 random bits + 1/2) * 2^-53."""
    hi = hi.astype(np.uint64) >> np.uint64(5)
    lo = lo.astype(np.uint64) >> np.uint64(6)
    return ((hi * np.uint64(1 << 26) + lo).astype(np.float64) + 0.5) * 2.0 ** -53


def uniforms(seed, species, idx):
    """Six uniforms per particle index: [w_x, w_y, w_z, w_py, w_u, w_phi]."""
    idx = np.asarray(idx, dtype=np.uint64)
    lo = (idx & _MASK).astype(np.uint32)
    hi = (idx >> np.uint64(32)).astype(np.uint32)
    key = (np.uint32(seed & 0xFFFFFFFF), np.uint32((seed >> 32) & 0xFFFFFFFF))
    out = []
    for call in range(3):
        r = philox4x32((lo, hi, np.full_like(lo, call), np.full_like(lo, species)), key)
        out.append(_to_double(r[0], r[1]))
        out.append(_to_double(r[2], r[3]))
    return np.stack(out)


# ------------------------------------------------------------------ marginal of the drift component

def _params(theta, beta0):
    mu = 1.0 / theta
    G0 = 1.0 / np.sqrt(1.0 - beta0 * beta0)
    return mu, G0


def marginal_pdf(y, theta, beta0):
    """j_Y(y) of Eq. distr_y, normalised to 1 (exponentially scaled Bessel K2)."""
    mu, G0 = _params(theta, beta0)
    gy = np.sqrt(1.0 + y * y)
    # exp(-mu G0 (gy - beta0 y)) = exp(-mu) exp(-mu (G0 (gy - beta0 y) - 1))
    arg = mu * (G0 * (gy - beta0 * y) - 1.0)
    return (1.0 + mu * G0 * gy) / (2.0 * mu * G0 ** 3 * special.kve(2, mu)) * np.exp(-arg)


def marginal_cdf_quad(y, theta, beta0):
    """J(y) by adaptive quadrature (scipy), for the statistical pins."""
    mu, G0 = _params(theta, beta0)
    psi = np.arctanh(beta0)
    center = np.sinh(psi)
    out = []
    for v in np.atleast_1d(y):
        pts = [center] if v > center else []
        val, _ = integrate.quad(marginal_pdf, -np.inf, v, args=(theta, beta0), limit=400, epsabs=1e-13,
                                epsrel=1e-12, points=None)
        out.append(val)
    return np.array(out)


class MarginalInverse:
    """Exact inverse of J by a dense table in s = asinh(y) (cumulative Simpson
    on 2^17 intervals of the density in s), monotone cubic interpolation of
    the table, and Newton polishing against the exact density."""

    def __init__(self, theta, beta0, n=1 << 17):
        mu, G0 = _params(theta, beta0)
        self.theta, self.beta0 = theta, beta0
        psi = np.arctanh(beta0)
        # support: the density in s falls below exp(-60) of its peak
        S = np.arccosh(1.0 + 60.0 / mu) + 1.0
        for _ in range(60):
            lo, hi = psi - S, psi + S
            g = self._g(np.array([lo, hi]))
            gm = self._g(np.linspace(psi - S, psi + S, 4001)).max()
            if np.all(g < 1e-27 * gm):
                break
            S *= 1.25
        s = np.linspace(psi - S, psi + S, 2 * n + 1)
        g = self._g(s)
        # composite Simpson per pair of sub-intervals
        seg = (s[2] - s[0]) / 6.0 * (g[0:-1:2] + 4.0 * g[1::2] + g[2::2])
        F = np.concatenate([[0.0], np.cumsum(seg)])
        self.total = F[-1]
        self.s = s[::2]
        self.F = F / F[-1]
        self.gs = g[::2] / F[-1]

    def _g(self, s):
        return marginal_pdf(np.sinh(s), self.theta, self.beta0) * np.cosh(s)

    def cdf_s(self, s):
        """Table CDF at arbitrary s (cubic Hermite with exact end slopes)."""
        k = np.clip(np.searchsorted(self.s, s) - 1, 0, len(self.s) - 2)
        h = self.s[k + 1] - self.s[k]
        t = (s - self.s[k]) / h
        h00 = 2 * t ** 3 - 3 * t ** 2 + 1
        h10 = t ** 3 - 2 * t ** 2 + t
        h01 = -2 * t ** 3 + 3 * t ** 2
        h11 = t ** 3 - t ** 2
        return h00 * self.F[k] + h10 * h * self.gs[k] + h01 * self.F[k + 1] + h11 * h * self.gs[k + 1]

    def __call__(self, w):
        w = np.asarray(w, dtype=np.float64)
        s = np.interp(w, self.F, self.s)
        for _ in range(4):
            g = self._g(s) / self.total
            s = s - (self.cdf_s(s) - w) / np.maximum(g, 1e-300)
            s = np.clip(s, self.s[0], self.s[-1])
        return np.sinh(s)


# ------------------------------------------------------------------ conditional and assembly

def conditional_t(a, w, iters=200):
    """t = a (u - 1) >= 0 with l(a + t) = w l(a) (Eq. finding_u), i.e.
    log1p(t / (1 + a)) - t = log w, solved by bisection (robust for any a)."""
    a = np.asarray(a, dtype=np.float64)
    lw = np.log(w)
    lo = np.zeros_like(a)
    hi = -lw * (1.0 + a) / a * 1.01 + 1e-300
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        f = np.log1p(mid / (1.0 + a)) - mid - lw
        pos = f > 0
        lo = np.where(pos, mid, lo)
        hi = np.where(pos, hi, mid)
    return 0.5 * (lo + hi)


def conditional_u(y, w, theta, beta0):
    """u >= 1 of Eq. finding_u given y (a = mu Gamma0 sqrt(1 + y^2))."""
    mu, G0 = _params(theta, beta0)
    a = mu * G0 * np.sqrt(1.0 + y * y)
    return 1.0 + conditional_t(a, w) / a


def conditional_u_lambertw(y, w, theta, beta0):
    """The same root in closed form, 1 + a u = -W_{-1}(-w l(a)/e), for moderate a."""
    mu, G0 = _params(theta, beta0)
    a = mu * G0 * np.sqrt(1.0 + y * y)
    logz = np.log(w) + np.log1p(a) - a - 1.0
    x1 = -np.real(special.lambertw(-np.exp(logz), k=-1))
    return (x1 - 1.0) / a


def basis(n):
    """Orthonormal (e1, e2) completing the unit vector n; n = 0 means z."""
    n = np.asarray(n, dtype=np.float64)
    nn = np.linalg.norm(n)
    n = np.array([0.0, 0.0, 1.0]) if nn == 0 else n / nn
    a = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = a - np.dot(a, n) * n
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    return n, e1, e2


def sample_momenta(w_py, w_u, w_phi, theta, beta):
    """Momenta (3, n) of the drifting Maxwell-Juttner distribution."""
    beta = np.asarray(beta, dtype=np.float64)
    b0 = float(np.linalg.norm(beta))
    n, e1, e2 = basis(beta)
    y = MarginalInverse(theta, b0)(w_py)
    mu, G0 = _params(theta, b0)
    a = mu * G0 * np.sqrt(1.0 + y * y)
    um1 = conditional_t(a, w_u) / a          # u - 1, accurate also when u is close to 1
    r = np.sqrt(um1 * (um1 + 2.0))
    gy = np.sqrt(1.0 + y * y)
    phi = 2.0 * np.pi * w_phi
    p1, p2 = gy * r * np.cos(phi), gy * r * np.sin(phi)
    return np.outer(n, y) + np.outer(e1, p1) + np.outer(e2, p2)


def naive_boost(w_py, w_u, w_phi, theta, beta):
    """Control of Sect. 4.2: rest-frame sample boosted particle by particle
    (positions unchanged), which is wrong for relativistic theta and beta."""
    beta = np.asarray(beta, dtype=np.float64)
    b0 = float(np.linalg.norm(beta))
    n, e1, e2 = basis(beta)
    p0 = sample_momenta(w_py, w_u, w_phi, theta, np.zeros(3))   # rest frame, axis z
    # components in the (e1, e2, n) frame of the rest sample (its axis is z)
    par0, q1, q2 = p0[2], p0[0], p0[1]
    g0 = np.sqrt(1.0 + (p0 ** 2).sum(0))
    G0 = 1.0 / np.sqrt(1.0 - b0 * b0)
    par = G0 * (par0 + b0 * g0)
    return np.outer(n, par) + np.outer(e1, q1) + np.outer(e2, q2)


def positions_uniform(w, nx, ny, nz, ndim):
    pos = np.zeros((3, w.shape[1]))
    pos[0] = nx * w[0]
    pos[1] = ny * w[1]
    if ndim == 3:
        pos[2] = nz * w[2]
    return pos


def positions_harris(w, nx, ny, nz, ndim, L, x0):
    """x from the sech^2((x - x0)/L) density truncated to [0, nx] (exact inverse CDF)."""
    ta, tb = np.tanh(-x0 / L), np.tanh((nx - x0) / L)
    pos = positions_uniform(w, nx, ny, nz, ndim)
    pos[0] = x0 + L * np.arctanh(ta + w[0] * (tb - ta))
    return pos


def harris_count(ppc, nx, ny, nz, ndim, L, x0):
    cells_t = ny * (nz if ndim == 3 else 1)
    return int(round(ppc * cells_t * L * (np.tanh((nx - x0) / L) - np.tanh(-x0 / L))))


def load(seed, species, n, theta, beta, ndim, nx, ny, nz, profile=0, L=1.0, x0=0.0, method="exact"):
    """Positions and momenta of n particles, as the loader defines them."""
    w = uniforms(seed, species, np.arange(n))
    if profile == 0:
        pos = positions_uniform(w, nx, ny, nz, ndim)
    else:
        pos = positions_harris(w, nx, ny, nz, ndim, L, x0)
    f = sample_momenta if method == "exact" else naive_boost
    u = f(w[3], w[4], w[5], theta, beta)
    return pos, u


# ------------------------------------------------------------------ closed-form moments (Table averages)

def moments(theta, beta0):
    """Averages over the drifting distribution (Table averages, App. E):
    <gamma>, <gamma v> along the drift, <p_perp v_perp>, <p_par v_par>."""
    mu, G0 = _params(theta, beta0)
    k32 = special.kve(3, mu) / special.kve(2, mu)
    return {"gamma": G0 * k32 - 1.0 / (mu * G0),
            "gamma_v_par": k32 * G0 * beta0,
            "pv_perp": theta / G0,
            "pv_par": theta / G0 + G0 * beta0 ** 2 * k32}
