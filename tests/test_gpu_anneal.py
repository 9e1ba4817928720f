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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [7, 14])
def test_anneal_general_matches_oracle(cuda_lib, oracle, prec, n):
    """Segments b_s H_P + a_s sum_j X_j (b_s of both signs and zero) against the oracle."""
    import torch

    from paper_2608_12058_b300 import api

    h, J = I.sk_instance(n, 40 + n)
    psi = I.random_state(n, 41 + n)
    a_s = np.array([1.2, 0.0, -0.4, 0.8, 0.3])
    b_s = np.array([0.3, 1.1, -0.7, 0.0, 2.0])
    ts = np.array([0.6, 0.4, 0.9, 0.5, 0.7])
    tol = 1e-12 if prec == "fp64" else 2.0 ** -23
    ref = oracle.anneal_general(h, J, a_s, b_s, ts, psi, tol)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    x = torch.from_numpy(psi).to(dt).cuda()
    api.anneal_general(h, J, a_s, b_s, ts, x, tol=tol, info=False)
    y = x.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,steps", [(8, 6), (16, 4)])
def test_magnus4_matches_oracle(cuda_lib, oracle, prec, n, steps):
    """cheb_magnus4 against the oracle's Magnus integrator on the same Gauss-node samples
    of a smooth annealing schedule."""
    import torch

    from paper_2608_12058_b300 import api

    T = 2.0
    h, J = I.sk_instance(n, 50 + n)
    psi = I.random_state(n, 51 + n)
    A = lambda t: 1.5 * (1 - t / T) + 0.3 * np.sin(3 * t)
    B = lambda t: t / T + 0.2 * np.cos(2 * t)
    dt, nodes = api.magnus4_nodes(A, B, T, steps)
    dto, nodeso = oracle.magnus4_nodes(A, B, T, steps)
    tol = 1e-12 if prec == "fp64" else 2.0 ** -23
    ref = oracle.magnus4(h, J, dto, nodeso, psi, tol)
    dtype = torch.complex64 if prec == "fp32" else torch.complex128
    x = torch.from_numpy(psi).to(dtype).cuda()
    infos = api.magnus4(h, J, dt, nodes, x, tol=tol, info=True)
    assert len(infos) == 2 * steps
    y = x.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= (1e-12 if prec == "fp64" else 1e-5)


def test_magnus4_adaptive_reaches_tolerance(cuda_lib, oracle):
    """The a-posteriori step count meets the requested integration error against an
    ODE solution of the dense system (FP64, n = 6)."""
    import torch
    from scipy.integrate import solve_ivp

    from paper_2608_12058_b300 import api

    n, T = 6, 2.0
    h, J = I.sk_instance(n, 63)
    psi = I.random_state(n, 64)
    A = lambda t: 1.5 * (1 - t / T) + 0.3 * np.sin(3 * t)
    B = lambda t: t / T + 0.2 * np.cos(2 * t)
    HP = np.diag(oracle.energies(h, J))
    HX = oracle.dense_hamiltonian(np.zeros(n), np.zeros((n, n)), 1.0)
    sol = solve_ivp(lambda t, y: -1j * (A(t) * HX + B(t) * HP) @ y, (0, T), psi, method="DOP853",
                    rtol=1e-13, atol=1e-13)
    x = torch.from_numpy(psi).cuda()
    M = api.magnus4_adaptive(h, J, A, B, T, x, tol=1e-8)
    err = np.linalg.norm(x.cpu().numpy() - sol.y[:, -1])
    assert M >= 16 and err <= 3e-8


@pytest.mark.parametrize("n,dtype_name,S", [(12, "complex64", 5), (18, "complex64", 4), (22, "complex64", 3),
                                            (14, "complex128", 3), (20, "complex128", 2)])
def test_anneal_graph_replays_anneal(cuda_lib, n, dtype_name, S):
    """A schedule captured into a CUDA graph (cheb_anneal_graph_create) and replayed
    equals cheb_anneal bit for bit, boundaries included, on every path (whole-run CTA,
    fused FP32, float-float FP64); a second replay applies the schedule again."""
    import torch

    from paper_2608_12058_b300 import api

    dt = getattr(torch, dtype_name)
    a = I.config_anneal(n=n, S=S, seed=21)
    x0 = torch.from_numpy(I.random_state(n, 22)).to(dt).cuda()
    y_ref = x0.clone()
    b_ref = torch.empty((S, 1 << n), dtype=dt, device="cuda")
    api.anneal(a.h, a.J, a.gammas, a.ts, y_ref, boundaries=b_ref, info=False)
    y2_ref = y_ref.clone()
    api.anneal(a.h, a.J, a.gammas, a.ts, y2_ref, info=False)
    x = x0.clone()
    bnd = torch.empty((S, 1 << n), dtype=dt, device="cuda")
    c0 = api.launch_count()
    g = api.AnnealGraph(a.h, a.J, a.gammas, a.ts, x, boundaries=bnd)
    c1 = api.launch_count()
    try:
        assert torch.equal(x, x0)  # capture does not run the work
        g.launch()
        g.status()
        replay = api.launch_count() - c1
        assert 0 < replay < c1 - c0  # the captured kernels, without the spectral scan
        assert torch.equal(x, y_ref)
        assert torch.equal(bnd, b_ref)
        g.launch()
        g.status()
        assert torch.equal(x, y2_ref)
    finally:
        g.close()


def test_anneal_graph_general_segments_and_slicing(cuda_lib):
    """Segments b_s H_P + a_s sum_j X_j (cheb_anneal_general), one of them long enough to
    be time-sliced: the replay equals the stream run."""
    import torch

    from paper_2608_12058_b300 import api

    n = 10
    a = I.config_anneal(n=n, S=3, seed=23)
    b_s = np.array([1.0, -0.5, 0.8])
    ts = np.array([0.5, 10000.0, 0.7])  # the middle segment exceeds the coefficient table
    x0 = torch.from_numpy(I.random_state(n, 24)).to(torch.complex128).cuda()
    y_ref = x0.clone()
    inf = api.anneal_general(a.h, a.J, a.gammas, b_s, ts, y_ref, tol=1e-10)
    assert inf[1]["time_splits"] > 1
    x = x0.clone()
    g = api.AnnealGraph(a.h, a.J, a.gammas, ts, x, b_s=b_s, tol=1e-10)
    try:
        g.launch()
        g.status()
        assert torch.equal(x, y_ref)
    finally:
        g.close()
