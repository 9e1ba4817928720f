"""cheb_anneal (piecewise-constant schedule) against the oracle's segment loop."""
import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.mark.parametrize("n,prec,S", [(9, "fp64", 8), (13, "fp32", 8), (15, "fp64", 5), (16, "fp32", 12)])
def test_anneal_matches_oracle(cuda_lib, oracle, n, prec, S):
    import torch

    from paper_2608_12058_b300 import api

    a = I.config_anneal(n=n, S=S, seed=n)
    psi0 = I.uniform_state(n)
    tol = 1e-12 if prec == "fp64" else 2.0 ** -23
    ref, starts = oracle.anneal(a.h, a.J, a.gammas, a.ts, psi0, tol)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    x = torch.from_numpy(psi0).to(dt).cuda()
    bnd = torch.empty((S, 1 << n), dtype=dt, device="cuda")
    infos = api.anneal(a.h, a.J, a.gammas, a.ts, x, tol=tol, boundaries=bnd)
    y = x.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= TOL[prec]
    b = bnd.cpu().numpy().astype(np.complex128)
    for s in range(S):
        assert np.linalg.norm(b[s] - starts[s]) / np.linalg.norm(starts[s]) <= TOL[prec]
    assert len(infos) == S and all(i["K"] > 0 for i in infos)
    assert abs(infos[-1]["norm"] - 1.0) < (1e-5 if prec == "fp32" else 1e-11)


def test_anneal_single_segment_is_expmv(cuda_lib):
    import torch

    from paper_2608_12058_b300 import api

    n = 14
    h, J = I.sk_instance(n, 3)
    psi0 = I.random_state(n, 4)
    x1 = torch.from_numpy(psi0).cuda()
    x2 = torch.from_numpy(psi0).cuda()
    api.anneal(h, J, [0.8], [2.5], x1, tol=1e-12)
    api.expmv(h, J, 0.8, 2.5, x2, tol=1e-12)
    assert torch.equal(x1, x2)
