// smooth_cells.cuh -- per-cell bodies of the current smoothing (App. A.3.4,
// main-loop step 10): the fold of a cell's ghost images and one 1-2-1 pass of
// one cell, in the exact int64 arithmetic of the mixed path or in FP64.
// Shared by the smoothing kernels (smooth.cu) and the persistent ensemble step
// (walk.cu).
#pragma once
#include "pic_internal.cuh"

namespace pic {

namespace {

__device__ inline void compact_coords(const Geom &g, long long c, int &i, int &j, int &k) {
    i = (int)(c % g.nx);
    const long long q = c / g.nx;
    j = (int)(q % g.ny);
    k = (int)(q / g.ny);
}

// Value of a stored current: signed int64 fixed point (mixed) or double.
__device__ inline long long value_of(unsigned long long v) { return (long long)v; }
__device__ inline double value_of(double v) { return v; }

// Normalisation of the 1-2-1 product: / 64 (3D) or / 16 (2D).
__device__ inline long long norm64(long long s) { return (s + 32) >> 6; }
__device__ inline long long norm16(long long s) { return (s + 8) >> 4; }
__device__ inline double norm64(double s) { return s * 0.015625; }
__device__ inline double norm16(double s) { return s * 0.0625; }

// Sum of J over every padded image of interior cell (i,j,k), skipping the
// interior cell itself when skip_self (modular int64 arithmetic: exact).
template <typename JT>
__device__ inline JT image_sum(const Geom &g, const JT *J, int i, int j, int k, bool skip_self) {
    JT s = JT(0);
    const int zlo = g.ndim == 3 ? -1 : 0, zhi = g.ndim == 3 ? 1 : 0;
    for (int mz = zlo; mz <= zhi; ++mz) {
        const int qk = k + g.Gz + mz * g.nz;
        if (qk < 0 || qk >= g.pz) continue;
        for (int my = -1; my <= 1; ++my) {
            const int qj = j + g.G + my * g.ny;
            if (qj < 0 || qj >= g.py) continue;
            for (int mx = -1; mx <= 1; ++mx) {
                const int qi = i + g.G + mx * g.nx;
                if (qi < 0 || qi >= g.px || (skip_self && mx == 0 && my == 0 && mz == 0)) continue;
                s += J[((long long)qk * g.py + qj) * g.px + qi];
            }
        }
    }
    return s;
}

// Read views of the input of a pass: the interior of a padded current plane
// (first pass) or a compact plane.
template <typename JT>
struct PaddedPlane {
    const JT *a;
    __device__ inline typename SmoothValue<JT>::type at(const Geom &g, int i, int j, int k) const {
        return value_of(ldro(a + g.pidx(i, j, k)));
    }
};
template <typename T>
struct CompactPlane {
    const T *a;
    __device__ inline T at(const Geom &g, int i, int j, int k) const {
        return ldro(a + ((long long)k * g.ny + j) * g.nx + i);
    }
};

// Periodic neighbour indices of (i, j).
struct XYIndex {
    int i, im, ip, j, jm, jp;
    __device__ inline XYIndex(const Geom &g, int i_, int j_) : i(i_), j(j_) {
        im = i == 0 ? g.nx - 1 : i - 1;
        ip = i == g.nx - 1 ? 0 : i + 1;
        jm = j == 0 ? g.ny - 1 : j - 1;
        jp = j == g.ny - 1 ? 0 : j + 1;
    }
};

// x-y part of the stencil (unnormalised) at plane k, read through view v.
template <typename T, typename V>
__device__ inline T xy_sum(const Geom &g, const V &v, const XYIndex &x, int k) {
    auto row = [&](int jj) -> T {
        const T a = v.at(g, x.im, jj, k), b = v.at(g, x.i, jj, k), c = v.at(g, x.ip, jj, k);
        return (a + (b + b)) + c;
    };
    const T r0 = row(x.jm), r1 = row(x.j), r2 = row(x.jp);
    return (r0 + (r1 + r1)) + r2;
}

// One pass at cell c of one compact plane (per-cell form, batched kernel).
template <typename T>
__device__ inline void smooth_cell(const Geom &g, const T *a, T *out, long long c) {
    int i, j, k;
    compact_coords(g, c, i, j, k);
    const XYIndex x(g, i, j);
    const CompactPlane<T> v{a};
    T r;
    if (g.ndim == 3) {
        const int km = k == 0 ? g.nz - 1 : k - 1, kp = k == g.nz - 1 ? 0 : k + 1;
        const T pm = xy_sum<T>(g, v, x, km), p0 = xy_sum<T>(g, v, x, k), pp = xy_sum<T>(g, v, x, kp);
        r = norm64((pm + (p0 + p0)) + pp);
    } else {
        r = norm16(xy_sum<T>(g, v, x, k));
    }
    out[c] = r;
}

}  // namespace

}  // namespace pic
