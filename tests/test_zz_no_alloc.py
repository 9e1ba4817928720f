"""cheb_expmv_noalloc (the entry point for callers that cannot allocate device
memory) gives the same result as cheb_expmv with a caller workspace.

The two results must be bit-identical: both entry points run the same
deterministic kernels on the same kernel path.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test. It passes alone in a fresh process
and after the other GPU tests (the scratch array keeps the previous call's data,
which the entry point must not depend on).
"""
import ctypes

import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _call_regular(L, n, h, J, gamma, t, x, prec, tol, stream):
    from paper_2608_12058_b300 import api

    ws = api.workspace(n, "fp32" if prec == 0 else "fp64", x.device)
    p, nb = api._ws_ptr(ws)
    from paper_2608_12058_b300._lib import Info

    info = Info()
    rc = L.cheb_expmv(n, _dp(h), _dp(J), gamma, t, ctypes.c_void_p(x.data_ptr()), prec, tol, 0, 0,
                      ctypes.c_void_p(p), nb, stream, ctypes.byref(info))
    return rc, info


def _call_noalloc(L, n, h, J, gamma, t, x, prec, tol, stream):
    from paper_2608_12058_b300._lib import Info

    info = Info()
    rc = L.cheb_expmv_noalloc(n, _dp(h), _dp(J), gamma, t, ctypes.c_void_p(x.data_ptr()), prec, tol, 0, 0,
                              stream, ctypes.byref(info))
    return rc, info


@pytest.mark.parametrize("n,prec", [(10, 1), (15, 1), (18, 1), (13, 0), (16, 0), (19, 0)])
def test_noalloc_matches_workspace_entry_point(cuda_lib, n, prec):
    import torch

    L = cuda_lib
    h, J = I.sk_instance(n, 700 + n, "uniform")
    h = np.ascontiguousarray(h)
    J = np.ascontiguousarray(J)
    psi0 = I.random_state(n, 800 + n)
    dt = torch.complex64 if prec == 0 else torch.complex128
    tol = 2.0 ** -23 if prec == 0 else 1e-12
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    gamma, t = 0.9, 3.5

    ref = torch.from_numpy(psi0).to(dt).cuda()
    rc, rinfo = _call_regular(L, n, h, J, gamma, t, ref, prec, tol, stream)
    assert rc == 0
    ref = ref.cpu()

    for call in range(2):  # two calls in a row share (and reuse) the scratch array
        x = torch.from_numpy(psi0).to(dt).cuda()
        rc, info = _call_noalloc(L, n, h, J, gamma, t, x, prec, tol, stream)
        assert rc == 0, (call, rc)
        torch.cuda.synchronize()
        # same deterministic kernels on the same path: the results agree bit for bit,
        # so a stale read of the shared scratch array cannot hide behind a tolerance
        assert torch.equal(x.cpu(), ref), call
        assert info.K == rinfo.K and abs(info.radius - rinfo.radius) < 1e-12 * rinfo.radius


def test_noalloc_rejects_sizes_beyond_its_scratch(cuda_lib):
    import torch

    L = cuda_lib
    for n, prec in [(20, 0), (19, 1)]:
        h, J = I.sk_instance(n, 1, "uniform")
        x = torch.zeros(1 << n, dtype=torch.complex64 if prec == 0 else torch.complex128, device="cuda")
        rc, _ = _call_noalloc(L, n, np.ascontiguousarray(h), np.ascontiguousarray(J), 1.0, 1.0, x, prec, 1e-6,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 6  # CHEB_ERR_UNSUPPORTED
