"""The Gauss-law check for callers that cannot allocate device memory
(pic_gauss_residual_static, C ABI).  Its two numbers, max |div e - rho~| and
max |rho~_s|, are compared on one FP64 state with the context's own
diagnostics (pic_diagnostics) and with the FP64 oracle's gauss_residual, on
calls in a row (the static scratch is reused and must be cleared by each
call), in 2D and in 3D.  The calls must leave device memory as they found it:
neither torch's allocator nor the device's free memory may change across
them.  Collected last on purpose: a failure here leaves every other test run."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1308_5892_gb300 as pic
import synth

pytestmark = pytest.mark.gpu


def _entry():
    fn = pic.lib().pic_gauss_residual_static
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                   ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                   ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


@pytest.mark.parametrize("ndim,shape", [(3, (20, 16, 12)), (2, (40, 24, 1))])
def test_static_gauss_residual_matches_diagnostics_and_oracle(ndim, shape):
    import torch
    nx, ny, nz = shape
    arr = synth.random_state_arrays(77 + ndim, ndim, nx, ny, nz, ppc=4, spread=1.0, amp_e=0.02, amp_b=0.02,
                                    colocate=False)
    n = arr["species"][0]["pos"].shape[1]
    n_x, rho_sp0 = 2.0, 8.0
    d = pic.run_desc(ndim, nx, ny, nz, n_x, rho_sp0, 0.5, [(-1.0, 1.0, n), (1.0, 1.0, n)])
    fields = np.concatenate([arr["e"], arr["b"]])
    parts = [np.concatenate([s["pos"], s["u"]]) for s in arr["species"]]
    with pic.Context([d], precision=pic.PIC_FP64) as ctx:
        ctx.set_state(0, fields, parts)
        ctx.step(2)
        ref = ctx.diagnostics(0)
        f, p, _ = ctx.get_state(0)
    st = oracle.State.empty(ndim, nx, ny, nz, 0.5, n_x, rho_sp0)
    st.e[:] = f[:3]
    st.b[:] = f[3:]
    for q, s in zip(p, arr["species"]):
        st.species.append(oracle.Species(np.ascontiguousarray(q[:3]), np.ascontiguousarray(q[3:]),
                                         s["q_over_e"], s["m_over_me"]))
    g_orc, rmax_orc = oracle.gauss_residual(st)

    dev = torch.device("cuda", torch.cuda.current_device())
    e = torch.from_numpy(np.ascontiguousarray(f[:3])).to(dev)
    pos = [torch.from_numpy(np.ascontiguousarray(q[:3])).to(dev) for q in p]
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    counts = (ctypes.c_int64 * 2)(n, n)
    ptrs = (ctypes.c_void_p * 2)(pos[0].data_ptr(), pos[1].data_ptr())
    alpha = (ctypes.c_double * 2)(*(st.alpha(s) for s in range(2)))
    fn = _entry()
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        return fn(ndim, nx, ny, nz, e.data_ptr(), 2, counts, ctypes.cast(ptrs, ctypes.c_void_p), alpha,
                  out.data_ptr(), stream)

    # the first call on the device resolves the static array (and may load the
    # library's module that holds it); the calls after it are measured
    assert call() == pic.PIC_OK
    torch.cuda.synchronize()
    torch_before = torch.cuda.memory_allocated(dev)
    free_before = torch.cuda.mem_get_info(dev)[0]
    results = []
    for _ in range(2):
        out.fill_(-1.0)
        assert call() == pic.PIC_OK
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    assert torch.cuda.memory_allocated(dev) == torch_before
    assert torch.cuda.mem_get_info(dev)[0] == free_before
    for got in results:
        assert abs(got[0] - ref["gauss_max"]) <= 1e-12 * ref["rho_max"] + 1e-15, (got, ref["gauss_max"])
        assert abs(got[1] - ref["rho_max"]) <= 1e-12 * ref["rho_max"]
        assert abs(got[0] - g_orc) <= 1e-12 * rmax_orc + 1e-15, (got, g_orc)
        assert abs(got[1] - rmax_orc) <= 1e-12 * rmax_orc
    # a grid above the static limit is refused without touching the device
    st_code = fn(3, 128, 128, 128, e.data_ptr(), 0, None, None, None, out.data_ptr(), stream)
    assert st_code == pic.PIC_EINVAL
