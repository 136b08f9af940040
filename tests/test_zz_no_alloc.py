"""gf_occupation_static, the entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc (code inside another
framework's memory pool or allocator hooks, plugins that must not grow the
device footprint after start-up).  Its scratch is a fixed device array inside
the library.  This test calls it through the C-ABI twice in a row and checks
each result against gf_occupation of a regular context, at the FP64 parity
tolerance.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1111_2157_gb300 import gf, synth
from tests.parity import make_gf

pytestmark = pytest.mark.gpu
TOL = 1e-10


def test_static_occupation_matches_context_api():
    import torch
    lib = gf.load()
    s = synth.ce_like(nk=24, n_iw=96).systems[0]
    dev = torch.device("cuda:0")
    # the C-ABI takes raw pointers to packed row-major arrays
    H = torch.from_numpy(s.H).to(dev).contiguous()
    P = torch.from_numpy(s.P).to(dev).contiguous()
    S = torch.from_numpy(s.sigma).to(dev).contiguous()
    Si = torch.from_numpy(s.sigma_inf).to(dev).contiguous()
    stream = torch.cuda.current_stream(dev).cuda_stream
    nb = s.H.shape[-1]
    assert s.P.shape[-1] == nb and s.H.shape[-2] == nb
    g = make_gf([s])
    for mu in (0.35, -0.8):
        n, dn = ctypes.c_double(), ctypes.c_double()
        st = lib.gf_occupation_static(ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(P.data_ptr()),
                                      ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(Si.data_ptr()),
                                      s.nk, nb, s.m, s.n_iw, s.beta, mu, 2, ctypes.c_void_p(stream),
                                      ctypes.byref(n), ctypes.byref(dn))
        assert st == gf.GF_OK, lib.gf_last_error(None).decode()
        n_ref, dn_ref = g.occupation([mu])
        assert abs(n.value - n_ref[0]) <= TOL * abs(n_ref[0])
        assert abs(dn.value - dn_ref[0]) <= TOL * abs(dn_ref[0])
    g.close()


def test_static_occupation_rejects_oversized_problem():
    import torch
    lib = gf.load()
    x = torch.zeros(4, dtype=torch.complex128, device="cuda:0")
    n = ctypes.c_double()
    ptr = ctypes.c_void_p(x.data_ptr())
    # 200000 k-points need far more than the 4 MiB static scratch: refused before any launch
    st = lib.gf_occupation_static(ptr, ptr, ptr, ptr, 200000, 8, 2, 1024, 10.0, 0.0, 2, None,
                                  ctypes.byref(n), None)
    assert st == gf.GF_EINVAL
    assert "4 MiB" in lib.gf_last_error(None).decode()


def test_static_occupation_across_contexts():
    """The scratch's device address is looked up on every call, in whatever context is current:
    a call in the primary context, then through the context API, then in a second CUDA context
    made current on the same device (where the library's module has another address), then in the
    primary context again, all give the same N."""
    import torch
    lib = gf.load()
    s = synth.ce_like(nk=8, n_iw=32).systems[0]
    nb = s.H.shape[-1]
    host = [np.ascontiguousarray(a, dtype=np.complex128) for a in (s.H, s.P, s.sigma, s.sigma_inf)]

    def static_call(ptrs):
        n = ctypes.c_double()
        st = lib.gf_occupation_static(*[ctypes.c_void_p(int(q)) for q in ptrs], s.nk, nb, s.m, s.n_iw,
                                      s.beta, 0.2, 2, None, ctypes.byref(n), None)
        assert st == gf.GF_OK, lib.gf_last_error(None).decode()
        return n.value

    dev = torch.device("cuda:0")
    tens = [torch.from_numpy(a).to(dev) for a in host]
    torch.cuda.synchronize()
    first = static_call([t.data_ptr() for t in tens])
    g = make_gf([s])
    n_ctx, _ = g.occupation([0.2])
    g.close()
    assert abs(first - n_ctx[0]) <= TOL * abs(n_ctx[0])

    try:
        cuda = ctypes.CDLL("libcuda.so.1")
    except OSError:
        pytest.skip("libcuda.so.1 not loadable")

    class CtxParams(ctypes.Structure):
        _fields_ = [("exec_affinity", ctypes.c_void_p), ("n_exec_affinity", ctypes.c_int),
                    ("cig", ctypes.c_void_p)]

    assert cuda.cuInit(0) == 0
    cudev = ctypes.c_int()
    assert cuda.cuDeviceGet(ctypes.byref(cudev), torch.cuda.current_device()) == 0
    ctx = ctypes.c_void_p()
    params = CtxParams()
    if cuda.cuCtxCreate_v4(ctypes.byref(ctx), ctypes.byref(params), 0, cudev) != 0:
        pytest.skip("cuCtxCreate failed")
    dptrs = []
    try:
        for a in host:
            d = ctypes.c_uint64()
            assert cuda.cuMemAlloc_v2(ctypes.byref(d), ctypes.c_size_t(a.nbytes)) == 0
            dptrs.append(d)
            assert cuda.cuMemcpyHtoD_v2(d, ctypes.c_void_p(a.ctypes.data), ctypes.c_size_t(a.nbytes)) == 0
        second = static_call([d.value for d in dptrs])
    finally:
        for d in dptrs:
            cuda.cuMemFree_v2(d)
        cuda.cuCtxDestroy_v2(ctx)
    third = static_call([t.data_ptr() for t in tens])
    torch.cuda.synchronize()
    assert second == first and third == first
