"""Accuracy at the full Clenshaw depth of the benchmarked workloads, and the
evaluation-error bound of Sec. II.B.3.

The other parity tests keep K in the tens so that the oracle finishes quickly.
Rounding errors of the recurrence grow with the number of steps (Sec. II.B.3: the
bound sums one term per step), so these tests run the n=24 workload (SK seed 0,
h ~ N(0,1), gamma = 0.8, t = 10, uniform psi0: K = 498 at tol 1e-12, 475 at
tol 2^-23) and a fused-split case with K > 400 against the FP64 oracle.

The oracle runs once per method at tol 1e-12; the FP32 result (tol 2^-23) differs
from it by at most its own truncation bound (~1.1e-7), far inside the FP32 bar.
"""
import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _run(h, J, gamma, t, psi_np, prec, tol, method="chebyshev", path="auto", eval_bound=False):
    import torch

    from paper_2608_12058_b300 import api

    dt = torch.complex64 if prec == "fp32" else torch.complex128
    psi = torch.from_numpy(psi_np.astype(np.complex128)).to(dt).cuda()
    info = api.expmv(h, J, gamma, t, psi, tol=tol, method=method, path=path, eval_bound=eval_bound)
    torch.cuda.synchronize()
    return psi.cpu().numpy().astype(np.complex128), info


def _rel(y, ref):
    return float(np.linalg.norm(y - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def c2_reference(oracle):
    """Oracle results of the n=24 workload, one per method, computed once."""
    cache = {}

    def get(method):
        if method not in cache:
            h, J = I.sk_instance(24, 0)
            psi = I.uniform_state(24)
            cache[method] = oracle.expmv(h, J, 0.8, 10.0, psi, 1e-12, method=method)
        return cache[method]

    return get


@pytest.mark.slow
@pytest.mark.parametrize("method", ["chebyshev", "cf"])
def test_n24_full_depth_matches_oracle(cuda_lib, c2_reference, method):
    """n=24, gamma=0.8, t=10 at full depth: FP64 (K = 498 / 497) within 1e-12 and
    FP32 (K = 475 / 474) within 1e-5 of the oracle, on every FP64 kernel path."""
    ref, oinfo = c2_reference(method)
    h, J = I.sk_instance(24, 0)
    psi = I.uniform_state(24)
    for path in ("plain", "auto"):
        y, info = _run(h, J, 0.8, 10.0, psi, "fp64", 1e-12, method, path)
        assert info["K"] == oinfo["K"] and info["K"] >= 490
        err = _rel(y, ref)
        print(f"n=24 {method} fp64 {path}: K={info['K']} rel L2 vs oracle {err:.3e}")
        assert err <= TOL["fp64"], (path, err)
    y, info = _run(h, J, 0.8, 10.0, psi, "fp32", 2.0 ** -23, method)
    assert info["K"] >= 470
    err = _rel(y, ref)
    print(f"n=24 {method} fp32: K={info['K']} rel L2 vs oracle {err:.3e}")
    assert err <= TOL["fp32"], err


@pytest.fixture(scope="module")
def deep22(oracle):
    """n=22, t=9: K = 439 at tol 2^-23 (oracle at tol 1e-12, K = 461)."""
    n = 22
    h, J = I.sk_instance(n, 222)
    psi = I.random_state(n, 223)
    ref, oinfo = oracle.expmv(h, J, 0.9, 9.0, psi, 1e-12)
    return h, J, psi, ref, oinfo


@pytest.mark.slow
@pytest.mark.parametrize("split,comp", [(None, False), ((0, 11), False), ((4, 7), False), (None, True),
                                        ((0, 11), True)])
def test_fused_splits_at_depth(cuda_lib, deep22, split, comp):
    """The fused FP32 step at K > 400 under its default split (one strided pass of 9
    bits, two L2 partner bits), two strided passes (6 + 5 bits) and four partner bits,
    with plain and with compensated flip sums."""
    from paper_2608_12058_b300 import api

    h, J, psi, ref, oinfo = deep22
    n = 22
    if split is not None:
        api.set_fused_split(n, *split)
    api.set_fused_compensated(comp)
    try:
        y, info = _run(h, J, 0.9, 9.0, psi, "fp32", 2.0 ** -23, path="fused")
    finally:
        api.set_fused_split(n, -1)
        api.set_fused_compensated(False)
    assert info["K"] > 400
    err = _rel(y, ref)
    print(f"n=22 split {split} compensated {comp}: K={info['K']} rel L2 vs oracle {err:.3e}")
    assert err <= TOL["fp32"], err


def _oracle_bound(oracle, h, J, gamma, t, psi, tol, u):
    """The bound of Sec. II.B.3 from the oracle's own FP64 Clenshaw vectors, at unit roundoff u."""
    emin, emax, c, r = oracle.bounds(h, J, gamma)
    D = (oracle.energies(h, J) - c) / r
    coef, K, _ = oracle.cheb_coeffs(t * r, tol, np.exp(-1j * t * c))
    y, norms = oracle.clenshaw(D, gamma / r, coef, psi, with_norms=True)
    return y, oracle.eval_bound(h.shape[0], norms, u)


@pytest.mark.parametrize("n,prec,path", [(12, "fp32", "auto"), (12, "fp64", "auto"), (20, "fp32", "auto"),
                                         (20, "fp64", "plain"), (16, "fp32", "fused")])
def test_eval_bound(cuda_lib, oracle, n, prec, path):
    """info['eval_bound'] (CHEB_FLAG_EVAL_BOUND) equals the oracle's bound at the same
    unit roundoff (computed from the oracle's own vectors; FP32 and the native FP64
    kernels here, the float-float step in its own test file), and bounds the observed
    difference from the oracle's FP64 result (the same polynomial, so the truncation
    error cancels)."""
    h, J = I.sk_instance(n, 500 + n)
    psi = I.random_state(n, 501 + n)
    tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    u = 2.0 ** -24 if prec == "fp32" else 2.0 ** -53
    ref, ob = _oracle_bound(oracle, h, J, 1.1, 4.0, psi, tol, u)
    y, info = _run(h, J, 1.1, 4.0, psi, prec, tol, path=path, eval_bound=True)
    gb = info["eval_bound"]
    err_abs = float(np.linalg.norm(y - ref))
    print(f"n={n} {prec}: eval_bound {gb:.3e} (oracle {ob:.3e}), observed {err_abs:.3e}")
    assert gb > 0 and abs(gb - ob) <= 1e-3 * ob
    assert err_abs <= gb


def test_eval_bound_needs_info(cuda_lib):
    import ctypes

    import torch

    from paper_2608_12058_b300 import api

    n = 10
    h, J = I.sk_instance(n, 3)
    x = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    ws = api.workspace(n, "fp32", x.device)
    p, nb = api._ws_ptr(ws)
    rc = cuda_lib.cheb_expmv_path(n, api._dp(h), api._dp(J), 1.0, 1.0, ctypes.c_void_p(x.data_ptr()), 0, 1e-6, 0, 0,
                                  api.EVAL_BOUND_FLAG, ctypes.c_void_p(p), nb, api._stream_ptr(x.device), None)
    assert rc == 1  # CHEB_ERR_INVALID_ARG


def test_workspace_status_reports_and_clears(cuda_lib):
    """cheb_workspace_status: OK after a clean call; a timeout recorded in the status
    word (planted from the host) is reported once and then cleared."""
    import ctypes

    import torch

    from paper_2608_12058_b300 import api

    n = 12
    h, J = I.sk_instance(n, 4)
    x = torch.from_numpy(I.random_state(n, 5)).to(torch.complex64).cuda()
    ws = api.workspace(n, "fp32", x.device)
    p, nb = api._ws_ptr(ws)
    st = api._stream_ptr(x.device)
    rc = cuda_lib.cheb_expmv(n, api._dp(h), api._dp(J), 1.0, 1.0, ctypes.c_void_p(x.data_ptr()), 0, 1e-6, 0, 0,
                             ctypes.c_void_p(p), nb, st, None)
    assert rc == 0
    assert cuda_lib.cheb_workspace_status(ctypes.c_void_p(p), nb, st) == 0
    off = p - ws.data_ptr()  # the aligned workspace start holds the status word
    torch.cuda.synchronize()
    ws[off:off + 4].view(torch.int32).fill_(1)  # kFlagTimeout
    torch.cuda.synchronize()
    assert cuda_lib.cheb_workspace_status(ctypes.c_void_p(p), nb, st) == 4  # CHEB_ERR_TIMEOUT
    assert cuda_lib.cheb_workspace_status(ctypes.c_void_p(p), nb, st) == 0
