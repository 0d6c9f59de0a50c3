"""Filament-merging diagnostic of the counter-streaming instability (Sect.
3.3) -- TEST INFRASTRUCTURE, like the rest of ``oracle/``.

The size of the current filaments is measured on the z-averaged current
amplitude: its two-dimensional autocorrelation in the x-y plane (of the
fluctuation about the mean, periodic box), averaged over azimuth to corr(r)
with corr(0) = 1; the filament scale is five times the radius where corr(r)
falls to 0.8.

The current of a step is recovered from two consecutive states of the
field solver: e^{t+dt} = e^t + dt curl b^{t+dt/2} + J (App. A.3.2, main-loop
steps 6 and 12), so J = e^{t+dt} - e^t - dt curl b^{t+dt/2}, the deposited
-alpha * flux sums of the step (smoothed, when the run smooths).
Arrays are (3, nz, ny, nx), component planes x, y, z, index (k, j, i).
"""
import numpy as np


def curl_b(b):
    """curl_h b at the e locations (the differences of the e advance)."""
    bx, by, bz = b
    back = lambda a, ax: np.roll(a, 1, axis=ax)     # a[idx - 1] along axis ax (0: z, 1: y, 2: x)
    cx = (bz - back(bz, 1)) - (by - back(by, 0))
    cy = (bx - back(bx, 0)) - (bz - back(bz, 2))
    cz = (by - back(by, 2)) - (bx - back(bx, 1))
    return np.stack([cx, cy, cz])


def step_current(e0, e1, b1, dt):
    """J added to e by the step e0 -> e1, with b1 = b^{t+dt/2} (periodic grid)."""
    return e1 - e0 - dt * curl_b(b1)


def radial_autocorrelation(a):
    """corr(r) of the 2D periodic field a (mean removed), averaged over unit
    bins of the minimum-image distance r, corr(0) = 1.  Returns (r, corr)."""
    f = a - a.mean()
    c = np.fft.ifft2(np.abs(np.fft.fft2(f)) ** 2).real
    c /= c[0, 0]
    ny, nx = a.shape
    dy = np.minimum(np.arange(ny), ny - np.arange(ny))[:, None]
    dx = np.minimum(np.arange(nx), nx - np.arange(nx))[None, :]
    r = np.sqrt(dx * dx + dy * dy)
    rb = np.rint(r).astype(int)
    nb = min(nx, ny) // 2
    sums = np.bincount(rb.ravel(), weights=c.ravel(), minlength=nb + 1)[: nb + 1]
    cnt = np.bincount(rb.ravel(), minlength=nb + 1)[: nb + 1]
    radius = np.arange(nb + 1, dtype=float)
    return radius, sums / np.maximum(cnt, 1)


def filament_scale(current, level=0.8, factor=5.0):
    """Five times the radius where the autocorrelation of the z-averaged
    current amplitude first falls to `level` (linear between bins)."""
    amp = np.sqrt((current ** 2).sum(axis=0)).mean(axis=0)      # (ny, nx)
    r, corr = radial_autocorrelation(amp)
    below = np.where(corr < level)[0]
    if below.size == 0:
        return np.inf
    m = below[0]
    r08 = r[m - 1] + (corr[m - 1] - level) / (corr[m - 1] - corr[m]) * (r[m] - r[m - 1])
    return factor * r08
