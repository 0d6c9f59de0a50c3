"""FP64 CPU oracle of the Apar-T particle-in-cell step (arXiv 1308.5892).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never calls it.

The numerical scheme lives in ``pic_oracle.c`` (plain C, every operation in
double precision, in the order of App. A.3 of the paper); this module is the
ctypes marshalling around it plus small numpy helpers.  The Maxwell-Juttner
loader, its moments and the Harris relations are in ``oracle.mj`` and
``oracle.harris``.

Array conventions (shared with the CUDA library's host interface only by
documentation, not by code):
  fields  e, b : float64 arrays of shape (3, nz, ny, nx); component planes
                 x, y, z; index (k, j, i) with i fastest; staggering of App.
                 A.3.2 (e_x at (i+1/2, j, k), ..., b_z at (i+1/2, j+1/2, k)).
  particles    : pos (3, n) and u (3, n) float64, u = gamma v / c.
"""
import ctypes
import os
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import build as _build

BC_PERIODIC = 0
BC_CONDUCTOR = 1

_lib = None
_lib_omp = None


class _Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("dt", ctypes.c_double), ("bc_x", ctypes.c_int),
                ("smooth_passes", ctypes.c_int)]


class _Species(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("pos", ctypes.POINTER(ctypes.c_double)),
                ("u", ctypes.POINTER(ctypes.c_double)), ("q_over_e", ctypes.c_double),
                ("m_over_me", ctypes.c_double), ("alpha", ctypes.c_double)]


def lib():
    """Load (building if needed) the C oracle."""
    global _lib
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


def lib_parallel():
    """The OpenMP build of the same source: the particle loop is shared between
    threads, each depositing into its own current grid (only the order of the
    FP64 current sums differs).  Used for the all-cores timing of the CPU
    baseline; the plain build above is the parity reference."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _load(_build.build(openmp=True))
    return _lib_omp


def _load(path):
    """Load one build of the C oracle and declare its entry points."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    G = ctypes.POINTER(_Grid)
    S = ctypes.POINTER(_Species)
    i64 = ctypes.c_int64
    d = ctypes.c_double
    sigs = {
        "orc_abi_version": ([], ctypes.c_int),
        "orc_b_advance": ([G, P, P, d], None),
        "orc_e_advance": ([G, P, P, d], None),
        "orc_node_fields": ([G, P, P, P], None),
        "orc_gather": ([G, P, P, i64, P, P], None),
        "orc_boris": ([i64, P, P, d, d], None),
        "orc_deposit": ([G, P, i64, P, P, d], None),
        "orc_rho": ([G, i64, P, d, P], None),
        "orc_div_e": ([G, P, P], None),
        "orc_smooth": ([G, P, ctypes.c_int, ctypes.c_int], None),
        "orc_step": ([G, P, P, P, ctypes.c_int, S], None),
        "orc_run": ([G, P, P, P, ctypes.c_int, S, ctypes.c_int], None),
        "orc_stagger_back": ([G, P, P, ctypes.c_int, S], None),
        "orc_energies": ([G, P, P, ctypes.c_int, S, d, P], None),
        "orc_temperature": ([ctypes.c_int, S, P], None),
        "orc_threads": ([ctypes.c_int], ctypes.c_int),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "float64 C-contiguous array expected"
    return a.ctypes.data_as(ctypes.c_void_p)


def alpha_of(q_over_e, n_x, rho_sp0):
    """Current coupling of a species, Eq. alpha (App. A.2): 2 sgn(q) / (n_x^2 rho_sp0)."""
    return 2.0 * np.sign(q_over_e) / (n_x * n_x * rho_sp0)


@dataclass
class Species:
    pos: np.ndarray          # (3, n) float64
    u: np.ndarray            # (3, n) float64
    q_over_e: float
    m_over_me: float

    @property
    def n(self):
        return self.pos.shape[1]


@dataclass
class State:
    """Simulation state at the start of a step: x^t, u^{t-dt/2}, e^t, b^{t-dt/2}."""
    ndim: int
    nx: int
    ny: int
    nz: int
    dt: float
    n_x: float
    rho_sp0: float
    e: np.ndarray
    b: np.ndarray
    species: List[Species] = field(default_factory=list)
    bc_x: int = BC_PERIODIC
    smooth_passes: int = 0   # current smoothing passes per step (App. A.3.4), periodic grids only

    @classmethod
    def empty(cls, ndim, nx, ny, nz, dt, n_x, rho_sp0, bc_x=BC_PERIODIC, smooth_passes=0):
        if ndim == 2:
            nz = 1
        z = np.zeros((3, nz, ny, nx))
        return cls(ndim, nx, ny, nz, dt, n_x, rho_sp0, z.copy(), z.copy(), [], bc_x, smooth_passes)

    def copy(self):
        sp = [Species(s.pos.copy(), s.u.copy(), s.q_over_e, s.m_over_me) for s in self.species]
        return State(self.ndim, self.nx, self.ny, self.nz, self.dt, self.n_x, self.rho_sp0,
                     self.e.copy(), self.b.copy(), sp, self.bc_x, self.smooth_passes)

    def grid(self):
        return _Grid(self.ndim, self.nx, self.ny, self.nz, self.dt, self.bc_x, self.smooth_passes)

    def alpha(self, s):
        return alpha_of(self.species[s].q_over_e, self.n_x, self.rho_sp0)

    @property
    def inv_alpha_abs(self):
        return self.n_x * self.n_x * self.rho_sp0 / 2.0

    def _species_array(self):
        arr = (_Species * max(1, len(self.species)))()
        for k, s in enumerate(self.species):
            assert s.pos.dtype == np.float64 and s.pos.flags["C_CONTIGUOUS"]
            assert s.u.dtype == np.float64 and s.u.flags["C_CONTIGUOUS"]
            arr[k].n = s.n
            arr[k].pos = s.pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[k].u = s.u.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[k].q_over_e = s.q_over_e
            arr[k].m_over_me = s.m_over_me
            arr[k].alpha = self.alpha(k)
        return arr


def step(state: State, nsteps: int = 1, J=None):
    """Advance ``state`` in place by ``nsteps`` steps of the main loop (App. A.3.1).
    Returns the current block J (3, nz, ny, nx) of the last step: the sums
    -alpha*flux that were added to e."""
    g = state.grid()
    if J is None:
        J = np.zeros_like(state.e)
    sp = state._species_array()
    lib().orc_run(ctypes.byref(g), _ptr(state.e), _ptr(state.b), _ptr(J), len(state.species), sp, nsteps)
    return J


def step_parallel(state: State, nsteps: int = 1, threads: int = 0):
    """step() with the OpenMP build on `threads` threads (0: all the host's
    cores); returns the number of threads used."""
    L = lib_parallel()
    used = L.orc_threads(threads)
    g = state.grid()
    J = np.zeros_like(state.e)
    sp = state._species_array()
    L.orc_run(ctypes.byref(g), _ptr(state.e), _ptr(state.b), _ptr(J), len(state.species), sp, nsteps)
    return used


def stagger_back(state: State):
    """Initial staggering (App. A.3.1): u^0 -> u^{-dt/2} by a Boris step of -dt/2,
    and b^0 -> b^{-dt/2} = b^0 + (dt/2) curl e^0."""
    g = state.grid()
    sp = state._species_array()
    lib().orc_stagger_back(ctypes.byref(g), _ptr(state.e), _ptr(state.b), len(state.species), sp)
    lib().orc_b_advance(ctypes.byref(g), _ptr(state.e), _ptr(state.b), -0.5 * state.dt)


def b_advance(state: State, h):
    g = state.grid()
    lib().orc_b_advance(ctypes.byref(g), _ptr(state.e), _ptr(state.b), h)


def e_advance(state: State, h):
    g = state.grid()
    lib().orc_e_advance(ctypes.byref(g), _ptr(state.e), _ptr(state.b), h)


def node_fields(state: State):
    g = state.grid()
    out = np.zeros((6,) + state.e.shape[1:])
    lib().orc_node_fields(ctypes.byref(g), _ptr(state.e), _ptr(state.b), _ptr(out))
    return out


def gather(state: State, pos):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[1]
    out = np.zeros((6, n))
    g = state.grid()
    lib().orc_gather(ctypes.byref(g), _ptr(state.e), _ptr(state.b), n, _ptr(pos), _ptr(out))
    return out


def boris(u, EB, h, dt):
    u = np.array(u, dtype=np.float64, order="C")
    EB = np.ascontiguousarray(EB, dtype=np.float64)
    lib().orc_boris(u.shape[1], _ptr(u), _ptr(EB), h, dt)
    return u


def deposit(state: State, pos0, disp, alpha):
    pos0 = np.ascontiguousarray(pos0, dtype=np.float64)
    disp = np.ascontiguousarray(disp, dtype=np.float64)
    J = np.zeros_like(state.e)
    g = state.grid()
    lib().orc_deposit(ctypes.byref(g), _ptr(J), pos0.shape[1], _ptr(pos0), _ptr(disp), alpha)
    return J


def rho(state: State, species=None):
    """Node charge density sum alpha_s W (CIC); all species unless one is named."""
    out = np.zeros(state.e.shape[1:])
    g = state.grid()
    idx = range(len(state.species)) if species is None else [species]
    for s in idx:
        sp = state.species[s]
        lib().orc_rho(ctypes.byref(g), sp.n, _ptr(np.ascontiguousarray(sp.pos)), state.alpha(s), _ptr(out))
    return out


def div_e(state: State):
    out = np.zeros(state.e.shape[1:])
    g = state.grid()
    lib().orc_div_e(ctypes.byref(g), _ptr(state.e), _ptr(out))
    return out


def smooth(state: State, a, passes=1):
    """The current smoothing of App. A.3.4 applied ``passes`` times to every
    plane of ``a`` (shape (nz, ny, nx) or (m, nz, ny, nx)); returns a new array."""
    out = np.array(a, dtype=np.float64, order="C", copy=True)
    nplanes = 1 if out.ndim == 3 else out.shape[0]
    g = state.grid()
    lib().orc_smooth(ctypes.byref(g), _ptr(out), nplanes, passes)
    return out


def gauss_residual(state: State):
    """(max |div e - S^P rho~|, max over species of max |rho~_s|), S^P the
    current smoothing of the run (identity when it is off): smoothing the
    current by S conserves div e - S rho~ instead of div e - rho~."""
    rho_all = rho(state)
    if state.smooth_passes > 0:
        rho_all = smooth(state, rho_all, state.smooth_passes)
    r = div_e(state) - rho_all
    rmax = max((np.abs(rho(state, s)).max() for s in range(len(state.species))), default=0.0)
    return float(np.abs(r).max()), float(rmax)


def energies(state: State):
    """dict: kinetic per species and field energy per component, units p m_e c^2."""
    nsp = len(state.species)
    out = np.zeros(nsp + 6)
    g = state.grid()
    sp = state._species_array()
    lib().orc_energies(ctypes.byref(g), _ptr(state.e), _ptr(state.b), nsp, sp, state.inv_alpha_abs, _ptr(out))
    return {"kinetic": out[:nsp].copy(), "field_e": out[nsp:nsp + 3].copy(), "field_b": out[nsp + 3:].copy()}


def temperature(state: State):
    """Temperature per species in units of m_e c^2: (m_s/m_e) <u . v> / 3
    (Sect. 3.1.3); equals (m_s/m_e) Theta for a Maxwell-Juttner population."""
    nsp = len(state.species)
    out = np.zeros(max(1, nsp))
    sp = state._species_array()
    lib().orc_temperature(nsp, sp, _ptr(out))
    return out[:nsp].copy()
