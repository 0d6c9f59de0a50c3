"""The Gauss-law check for callers that cannot allocate device memory
(pic_gauss_residual_static, C ABI), compared with the same numbers from the
context's own diagnostics (pic_diagnostics) on one FP64 state, twice in a row
(the static scratch is reused by the second call).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import paper_1308_5892_gb300 as pic
import synth

pytestmark = pytest.mark.gpu


def test_static_gauss_residual_matches_diagnostics_twice():
    import torch
    ndim, nx, ny, nz = 3, 20, 16, 12
    arr = synth.random_state_arrays(77, ndim, nx, ny, nz, ppc=4, spread=1.0, amp_e=0.02, amp_b=0.02,
                                    colocate=False)
    n = arr["species"][0]["pos"].shape[1]
    d = pic.run_desc(ndim, nx, ny, nz, 2.0, 8.0, 0.5, [(-1.0, 1.0, n), (1.0, 1.0, n)])
    fields = np.concatenate([arr["e"], arr["b"]])
    parts = [np.concatenate([s["pos"], s["u"]]) for s in arr["species"]]
    with pic.Context([d], precision=pic.PIC_FP64) as ctx:
        ctx.set_state(0, fields, parts)
        ctx.step(2)
        ref = ctx.diagnostics(0)
        f, p, _ = ctx.get_state(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    e = torch.from_numpy(np.ascontiguousarray(f[:3])).to(dev)
    pos = [torch.from_numpy(np.ascontiguousarray(q[:3])).to(dev) for q in p]
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    counts = (ctypes.c_int64 * 2)(n, n)
    ptrs = (ctypes.c_void_p * 2)(pos[0].data_ptr(), pos[1].data_ptr())
    alpha = (ctypes.c_double * 2)(-2.0 / (4.0 * 8.0), 2.0 / (4.0 * 8.0))
    L = pic.lib()
    fn = L.pic_gauss_residual_static
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                   ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                   ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        st = fn(ndim, nx, ny, nz, e.data_ptr(), 2, counts, ctypes.cast(ptrs, ctypes.c_void_p), alpha,
                out.data_ptr(), stream)
        assert st == pic.PIC_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - ref["gauss_max"]) <= 1e-12 * ref["rho_max"] + 1e-15
        assert abs(got[1] - ref["rho_max"]) <= 1e-12 * ref["rho_max"]
    # a grid above the static limit is refused without touching the device
    st = fn(3, 128, 128, 128, e.data_ptr(), 0, None, None, None, out.data_ptr(), stream)
    assert st == pic.PIC_EINVAL
