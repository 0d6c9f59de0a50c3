"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point declared in include/pic.h, and rejects invalid descriptors
in pic_init before any device work (these calls need no GPU)."""
import ctypes
import os
import re

import pytest

import paper_1308_5892_gb300 as pic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = pic.lib()
    names = _declared()
    assert "pic_step" in names and "pic_init" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(pic.ABI_FUNCTIONS) | {n for n in names if n.startswith("pic_")}
    assert L.pic_abi_version() == 2


def _init(desc, precision=pic.PIC_FP64):
    L = pic.lib()
    o = pic.Opts()
    o.precision = precision
    h = ctypes.c_void_p()
    return L.pic_init(ctypes.byref(desc), 1, ctypes.byref(o), ctypes.byref(h)), h


@pytest.mark.parametrize("kw,why", [
    (dict(dt=0.75), "2D Courant limit"),
    (dict(ndim=3, nz=8, dt=0.6), "3D Courant limit"),
    (dict(nz=4), "nz != 1 in 2D"),
    (dict(nx=1), "grid too small"),
    (dict(n_x=0.0), "n_x"),
    (dict(rho_sp0=-1.0), "rho_sp0"),
    (dict(species=[]), "no species"),
    (dict(species=[(0.0, 1.0, 10)]), "zero charge"),
    (dict(species=[(-1.0, 0.0, 10)]), "zero mass"),
    (dict(species=[(-1.0, 1.0, -5)]), "negative capacity"),
    (dict(bc=(0, 1, 0)), "conductor along y"),
    (dict(smooth_passes=5), "too many smoothing passes"),
    (dict(smooth_passes=-1), "negative smoothing passes"),
    (dict(smooth_passes=1, bc=(1, 0, 0)), "smoothing with a conductor"),
])
def test_init_rejects_invalid_descriptors(kw, why):
    args = dict(ndim=2, nx=16, ny=16, nz=1, n_x=2.0, rho_sp0=8.0, dt=0.5, species=[(-1.0, 1.0, 10)], bc=(0, 0, 0),
                smooth_passes=0)
    args.update(kw)
    d = pic.run_desc(args["ndim"], args["nx"], args["ny"], args["nz"], args["n_x"], args["rho_sp0"], args["dt"],
                     args["species"], args["bc"], smooth_passes=args["smooth_passes"])
    st, h = _init(d)
    assert st == pic.PIC_EINVAL, why
    assert not h.value


def test_init_rejects_bad_precision():
    d = pic.run_desc(2, 16, 16, 1, 2.0, 8.0, 0.5, [(-1.0, 1.0, 10)])
    st, h = _init(d, precision=7)
    assert st == pic.PIC_EINVAL


def test_null_arguments_are_rejected():
    L = pic.lib()
    assert L.pic_init(None, 1, None, None) == pic.PIC_EINVAL
    assert L.pic_step(None, 1) == pic.PIC_EINVAL
    assert L.pic_sync(None) == pic.PIC_EINVAL
    L.pic_destroy(None)
