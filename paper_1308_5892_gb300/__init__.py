"""Python binding of libpic_gb300.so, the GB300 particle-in-cell step library
(C ABI in include/pic.h).

Argument marshalling only: every step of the particle-in-cell path runs in
the library's CUDA kernels.  PyTorch is used, when available, for device
memory (its caching allocator, passed to the library as a pic_allocator) and
for the CUDA stream.  If the compiled library is missing, importing the
binding raises: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ETIMEOUT, PIC_ENUMERIC, PIC_ESTATE = range(7)
STATUS_NAMES = ["PIC_OK", "PIC_EINVAL", "PIC_ENOMEM", "PIC_ECUDA", "PIC_ETIMEOUT", "PIC_ENUMERIC", "PIC_ESTATE"]
PIC_FP64, PIC_MIXED = 0, 1
PIC_BC_PERIODIC, PIC_BC_CONDUCTOR = 0, 1
PIC_PROFILE_UNIFORM, PIC_PROFILE_HARRIS = 0, 1
PIC_MJ_EXACT, PIC_MJ_MLP, PIC_MJ_NAIVE_BOOST = 0, 1, 2
PIC_FLAG_ASYNC, PIC_FLAG_NO_GRAPH, PIC_FLAG_TIMING, PIC_FLAG_PHASE_LAUNCHES, PIC_FLAG_INJECT_STALL = 1, 2, 4, 8, 16
PIC_KERNEL_PUSH, PIC_KERNEL_FIELD, PIC_KERNEL_SORT, PIC_KERNEL_SMOOTH = 0, 1, 2, 3
MAX_SPECIES = 4

ABI_FUNCTIONS = [
    "pic_abi_version", "pic_init", "pic_destroy", "pic_last_error", "pic_set_state", "pic_get_state",
    "pic_set_uniform_field", "pic_load_maxwell_juttner", "pic_step", "pic_sync", "pic_diagnostics",
    "pic_energy_history", "pic_get_tuning", "pic_get_counters", "pic_kernel_time", "pic_get_particles",
    "pic_alu_peak", "pic_mlp_train", "pic_mlp_set_weights", "pic_mlp_get_weights", "pic_mlp_gradients", "pic_mlp_infer",
    "pic_mj_sample_marginal", "pic_gauss_residual_static", "pic_autotune", "pic_set_flags",
]
MLP_PARAMS = 8641


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status


class SpeciesDesc(ctypes.Structure):
    _fields_ = [("q_over_e", ctypes.c_double), ("m_over_me", ctypes.c_double), ("capacity", ctypes.c_int64)]


class RunDesc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("n_x", ctypes.c_double), ("rho_sp0", ctypes.c_double), ("dt", ctypes.c_double),
                ("bc", ctypes.c_int * 3), ("nspecies", ctypes.c_int), ("species", SpeciesDesc * MAX_SPECIES),
                ("smooth_passes", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("sort_interval", ctypes.c_int), ("tile", ctypes.c_int * 3),
                ("stream", ctypes.c_void_p), ("allocator", ctypes.POINTER(Allocator)), ("flags", ctypes.c_uint32)]


class StateView(ctypes.Structure):
    _fields_ = [("fields", ctypes.POINTER(ctypes.c_double)), ("count", ctypes.c_int64 * MAX_SPECIES),
                ("particles", ctypes.POINTER(ctypes.c_double) * MAX_SPECIES), ("step", ctypes.c_int64)]


class Diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("nspecies", ctypes.c_int), ("count", ctypes.c_int64 * MAX_SPECIES),
                ("kinetic", ctypes.c_double * MAX_SPECIES), ("field_e", ctypes.c_double * 3),
                ("field_b", ctypes.c_double * 3), ("sum_u", (ctypes.c_double * 3) * MAX_SPECIES),
                ("temperature", ctypes.c_double * MAX_SPECIES), ("gauss_max", ctypes.c_double),
                ("rho_max", ctypes.c_double), ("nonfinite", ctypes.c_int64)]


_lib = None


def library_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load libpic_gb300.so (building it first when stale and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and (_build.stale()):
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libpic_gb300.so is not built; run __graft_entry__.build() (no CPU fallback exists)")
    L = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    st = ctypes.c_int
    sigs = {
        "pic_abi_version": ([], ctypes.c_int),
        "pic_init": ([ctypes.POINTER(RunDesc), ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(P)], st),
        "pic_destroy": ([P], None),
        "pic_last_error": ([P], ctypes.c_char_p),
        "pic_set_state": ([P, ctypes.c_int, ctypes.POINTER(StateView)], st),
        "pic_get_state": ([P, ctypes.c_int, ctypes.POINTER(StateView)], st),
        "pic_set_uniform_field": ([P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], st),
        "pic_load_maxwell_juttner": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_int, ctypes.c_int, ctypes.c_uint64], st),
        "pic_step": ([P, ctypes.c_int], st),
        "pic_sync": ([P], st),
        "pic_diagnostics": ([P, ctypes.c_int, ctypes.POINTER(Diag)], st),
        "pic_energy_history": ([P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                ctypes.POINTER(ctypes.c_int64)], st),
        "pic_get_tuning": ([P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int)], st),
        "pic_get_counters": ([P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)], st),
        "pic_set_flags": ([P, ctypes.c_uint32], st),
        "pic_kernel_time": ([P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_int64)], st),
        "pic_get_particles": ([P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_double)], st),
        "pic_mlp_train": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                           ctypes.POINTER(ctypes.c_double)], st),
        "pic_mlp_set_weights": ([P, ctypes.POINTER(ctypes.c_float)], st),
        "pic_mlp_get_weights": ([P, ctypes.POINTER(ctypes.c_float)], st),
        "pic_mlp_gradients": ([P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                               ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)], st),
        "pic_mlp_infer": ([P, ctypes.POINTER(ctypes.c_float), ctypes.c_int64, ctypes.POINTER(ctypes.c_float)], st),
        "pic_mj_sample_marginal": ([P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(ctypes.c_double)], st),
        "pic_autotune": ([P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_int)], st),
        "pic_alu_peak": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], st),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def run_desc(ndim, nx, ny, nz, n_x, rho_sp0, dt, species, bc=(0, 0, 0), smooth_passes=0):
    """species: list of (q_over_e, m_over_me, capacity); smooth_passes: current
    smoothing passes per step (App. A.3.4), 0 = off."""
    d = RunDesc()
    d.smooth_passes = smooth_passes
    d.ndim, d.nx, d.ny, d.nz = ndim, nx, ny, nz
    d.n_x, d.rho_sp0, d.dt = n_x, rho_sp0, dt
    for a in range(3):
        d.bc[a] = bc[a]
    d.nspecies = len(species)
    for k, (q, m, cap) in enumerate(species):
        d.species[k].q_over_e = q
        d.species[k].m_over_me = m
        d.species[k].capacity = int(cap)
    return d


PIC_PEAK_FP32_FMA, PIC_PEAK_FP64_FMA = 0, 1


def alu_peak(kind):
    """Measured FMA throughput of the current device in TFLOP/s (pic_alu_peak)."""
    tf = ctypes.c_double()
    ms = ctypes.c_double()
    st = lib().pic_alu_peak(kind, ctypes.byref(tf), ctypes.byref(ms))
    if st != PIC_OK:
        raise PicError(st, "pic_alu_peak failed")
    return tf.value


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Context:
    """Owns a pic_ctx.  ``runs`` is a list of RunDesc; ``precision`` PIC_FP64
    or PIC_MIXED.  With ``torch_memory`` the device buffers come from torch's
    caching allocator and work is queued on torch's current stream."""

    def __init__(self, runs, precision=PIC_MIXED, sort_interval=0, tile=(0, 0, 0), flags=0, torch_memory=True,
                 stream=None):
        L = lib()
        self._L = L
        self.runs = list(runs)
        arr = (RunDesc * len(self.runs))(*self.runs)
        o = Opts()
        o.precision = precision
        o.sort_interval = sort_interval
        for a in range(3):
            o.tile[a] = tile[a]
        o.flags = flags
        self._alloc = None
        if torch_memory:
            import torch
            dev = torch.cuda.current_device()
            s = torch.cuda.current_stream() if stream is None else stream
            o.stream = ctypes.c_void_p(s.cuda_stream)
            self._torch_stream = s

            def _a(n, user):
                return torch.cuda.caching_allocator_alloc(int(n), dev, s)

            def _f(p, n, user):
                torch.cuda.caching_allocator_delete(int(p))

            self._afn, self._ffn = ALLOC_FN(_a), FREE_FN(_f)
            self._alloc = Allocator(self._afn, self._ffn, None)
            o.allocator = ctypes.pointer(self._alloc)
        elif stream is not None:
            o.stream = ctypes.c_void_p(stream)
        self._opts = o
        h = ctypes.c_void_p()
        st = L.pic_init(arr, len(self.runs), ctypes.byref(o), ctypes.byref(h))
        if st != PIC_OK:
            raise PicError(st, "pic_init rejected the descriptors")
        self.h = h
        self.precision = precision

    def _check(self, st):
        if st != PIC_OK:
            raise PicError(st, self._L.pic_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self._L.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, run, fields, particles):
        """fields: (6, nz, ny, nx) float64 (e at t, b at t-dt/2); particles:
        list per species of (6, n) float64 planes x, y, z, u_x, u_y, u_z."""
        fields = np.ascontiguousarray(fields, dtype=np.float64)
        v = StateView()
        v.fields = _dptr(fields)
        keep = [fields]
        for s, p in enumerate(particles):
            p = np.ascontiguousarray(p, dtype=np.float64)
            keep.append(p)
            v.count[s] = p.shape[1]
            v.particles[s] = _dptr(p)
        return self._check(self._L.pic_set_state(self.h, run, ctypes.byref(v)))

    def get_state(self, run, out=None, fields_only=False):
        d = self.runs[run]
        nz = 1 if d.ndim == 2 else d.nz
        fields = np.zeros((6, nz, d.ny, d.nx)) if out is None else out[0]
        v = StateView()
        v.fields = _dptr(fields)
        parts = []
        for s in range(d.nspecies):
            if fields_only:
                parts.append(None)
                continue
            p = np.zeros((6, int(d.species[s].capacity))) if out is None else out[1][s]
            parts.append(p)
            v.count[s] = p.shape[1]
            v.particles[s] = _dptr(p)
        self._check(self._L.pic_get_state(self.h, run, ctypes.byref(v)))
        if fields_only:
            return fields, [int(v.count[s]) for s in range(d.nspecies)], v.step
        res = []
        for s in range(d.nspecies):
            n = v.count[s]
            p = parts[s]
            if n != p.shape[1]:
                flat = p.reshape(-1)[: 6 * n]
                p = flat.reshape(6, n).copy()
            res.append(p)
        return fields, res, v.step

    def set_uniform_field(self, run, e0, b0):
        e = (ctypes.c_double * 3)(*e0)
        b = (ctypes.c_double * 3)(*b0)
        return self._check(self._L.pic_set_uniform_field(self.h, run, e, b))

    def load_maxwell_juttner(self, run, species, ppc, theta, beta=(0.0, 0.0, 0.0), profile=PIC_PROFILE_UNIFORM,
                             profile_params=(0.0, 0.0), method=PIC_MJ_EXACT, colocate_with=-1, seed=1):
        b = (ctypes.c_double * 3)(*beta)
        pp = (ctypes.c_double * 4)(*(list(profile_params) + [0.0] * (4 - len(profile_params))))
        return self._check(self._L.pic_load_maxwell_juttner(self.h, run, species, ppc, theta, b, profile, pp,
                                                            method, colocate_with, seed))

    def step(self, n=1):
        return self._check(self._L.pic_step(self.h, n))

    def sync(self):
        return self._check(self._L.pic_sync(self.h))

    def diagnostics(self, run=0):
        d = Diag()
        self._check(self._L.pic_diagnostics(self.h, run, ctypes.byref(d)))
        ns = d.nspecies
        return {
            "step": d.step,
            "count": [d.count[s] for s in range(ns)],
            "kinetic": np.array([d.kinetic[s] for s in range(ns)]),
            "field_e": np.array(list(d.field_e)),
            "field_b": np.array(list(d.field_b)),
            "sum_u": np.array([[d.sum_u[s][c] for c in range(3)] for s in range(ns)]),
            "temperature": np.array([d.temperature[s] for s in range(ns)]),
            "gauss_max": d.gauss_max,
            "rho_max": d.rho_max,
            "nonfinite": d.nonfinite,
        }

    def energy_history(self, run=0, max_steps=1 << 16):
        out = np.zeros(4 * max_steps)
        n = ctypes.c_int64()
        self._check(self._L.pic_energy_history(self.h, run, _dptr(out), max_steps, ctypes.byref(n)))
        return out[: 4 * n.value].reshape(n.value, 4)

    def tuning(self):
        t = (ctypes.c_int * 3)()
        k = ctypes.c_int()
        hh = ctypes.c_int()
        self._check(self._L.pic_get_tuning(self.h, t, ctypes.byref(k), ctypes.byref(hh)))
        return {"tile": tuple(t), "sort_interval": k.value, "halo": hh.value}

    def counters(self):
        n = ctypes.c_int64()
        b = ctypes.c_double()
        self._check(self._L.pic_get_counters(self.h, ctypes.byref(n), ctypes.byref(b)))
        return {"launches_per_step": n.value, "bytes_per_particle_step": b.value}

    def set_flags(self, flags):
        """Replace the PIC_FLAG_* bits (takes effect at the next call)."""
        self._check(self._L.pic_set_flags(self.h, int(flags)))

    def kernel_time(self, kernel_class, reset=False):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self._L.pic_kernel_time(self.h, kernel_class, int(reset), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def get_particles(self, run, species, ids):
        """Particles of one species by id: (6, len(ids)) planes x, y, z, u_x, u_y, u_z."""
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        out = np.zeros((6, len(ids)))
        self._check(self._L.pic_get_particles(self.h, run, species, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                              len(ids), _dptr(out)))
        return out

    # ---- learned sampler of the loader
    def mlp_train(self, steps=4000, batch=4096, lr=3e-3, seed=1):
        loss = ctypes.c_double()
        self._check(self._L.pic_mlp_train(self.h, steps, batch, lr, seed, ctypes.byref(loss)))
        return loss.value

    def mlp_set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == MLP_PARAMS
        self._check(self._L.pic_mlp_set_weights(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def mlp_get_weights(self):
        w = np.zeros(MLP_PARAMS, dtype=np.float32)
        self._check(self._L.pic_mlp_get_weights(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return w

    def mlp_gradients(self, x, target):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(target, dtype=np.float32)
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        f = ctypes.POINTER(ctypes.c_float)
        self._check(self._L.pic_mlp_gradients(self.h, x.ctypes.data_as(f), t.ctypes.data_as(f), t.size,
                                               g.ctypes.data_as(f), ctypes.byref(loss)))
        return g, loss.value

    def mlp_infer(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        out = np.zeros(x.shape[1], dtype=np.float32)
        f = ctypes.POINTER(ctypes.c_float)
        self._check(self._L.pic_mlp_infer(self.h, x.ctypes.data_as(f), x.shape[1], out.ctypes.data_as(f)))
        return out

    def mj_sample_marginal(self, theta, beta0, w, method=PIC_MJ_EXACT):
        w = np.ascontiguousarray(w, dtype=np.float64)
        y = np.zeros_like(w)
        ms = ctypes.c_double()
        self._check(self._L.pic_mj_sample_marginal(self.h, theta, beta0, _dptr(w), w.size, _dptr(y), method,
                                                    ctypes.byref(ms)))
        return y, ms.value

    def autotune(self, max_steps=200):
        """Pick tile shape and sort interval on real steps; returns the choice."""
        t = (ctypes.c_int * 3)()
        k = ctypes.c_int()
        n = ctypes.c_int()
        self._check(self._L.pic_autotune(self.h, max_steps, t, ctypes.byref(k), ctypes.byref(n)))
        return {"tile": tuple(t), "sort_interval": k.value, "steps_taken": n.value}
