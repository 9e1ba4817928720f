"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 against the oracle's result on the same seeded input):
FP64 recurrence 1e-12, FP32 recurrence 1e-5, the bars stated for the method.
Sizes span the whole-vector shared-memory kernel (n <= 13 FP32 / 12 FP64), the
boundary, and several tiles of the multi-tile paths.
"""
import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _torch():
    import torch

    return torch


def _run(h, J, gamma, t, psi_np, prec, tol, method="chebyshev", path="auto", splits=0):
    torch = _torch()
    from paper_2608_12058_b300 import api

    dt = torch.complex64 if prec == "fp32" else torch.complex128
    psi = torch.from_numpy(psi_np.astype(np.complex128)).to(dt).cuda()
    info = api.expmv(h, J, gamma, t, psi, tol=tol, method=method, path=path, time_splits=splits)
    torch.cuda.synchronize()
    return psi.cpu().numpy().astype(np.complex128), info


def _rel(y, ref):
    return np.linalg.norm(y - ref) / np.linalg.norm(ref)


CASES = [
    # n, seed, gamma, t, psi kind
    (1, 1, 0.7, 2.0, "random"),
    (3, 2, 1.3, 5.0, "random"),
    (10, 0, 1.0, 1.0, "uniform"),     # the n=10 SK workload
    (12, 3, 0.8, 6.0, "random"),
    (13, 4, 1.1, 4.0, "random"),
    (14, 5, 0.6, 8.0, "random"),
    (16, 6, 1.0, 5.0, "uniform"),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,seed,gamma,t,kind", CASES)
def test_expmv_matches_oracle(cuda_lib, oracle, prec, n, seed, gamma, t, kind):
    h, J = I.sk_instance(n, seed)
    psi = I.uniform_state(n) if kind == "uniform" else I.random_state(n, seed + 7)
    tol = 1e-12 if prec == "fp64" else 2.0 ** -23
    ref, oinfo = oracle.expmv(h, J, gamma, t, psi, tol)
    y, info = _run(h, J, gamma, t, psi, prec, tol)
    assert info["K"] == oinfo["K"]
    assert abs(info["radius"] - oinfo["radius"]) <= 1e-13 * oinfo["radius"]
    err = _rel(y, ref)
    assert err <= TOL[prec], err
    assert abs(info["norm"] - np.linalg.norm(y)) < (1e-6 if prec == "fp32" else 1e-12)
    assert abs(info["energy"] - oinfo["energy"]) < (1e-4 if prec == "fp32" else 1e-10) * max(1, abs(oinfo["energy"]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [4, 11, 15])
def test_plain_path_matches_oracle(cuda_lib, oracle, prec, n):
    """The one-pass kernel (every partner read from global memory) at sizes where
    the automatic choice would take another kernel."""
    h, J = I.sk_instance(n, 40 + n)
    psi = I.random_state(n, 41 + n)
    tol = 1e-12 if prec == "fp64" else 2.0 ** -23
    ref, _ = oracle.expmv(h, J, 0.9, 3.0, psi, tol)
    y, _ = _run(h, J, 0.9, 3.0, psi, prec, tol, path="plain")
    assert _rel(y, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cf_method_matches_oracle(cuda_lib, oracle, prec):
    n = 12
    h, J = I.sk_instance(n, 77)
    psi = I.random_state(n, 78)
    tol = 1e-10 if prec == "fp64" else 2.0 ** -23
    ref, oinfo = oracle.expmv(h, J, 1.2, 6.0, psi, tol, method="cf")
    y, info = _run(h, J, 1.2, 6.0, psi, prec, tol, method="cf")
    assert info["K"] == oinfo["K"]
    assert _rel(y, ref) <= TOL[prec]


def test_two_strided_passes_match_oracle(cuda_lib, oracle):
    """n = 25, the smallest size whose default plan has two strided passes (7 + 7 bits;
    the n = 30 benchmark runs two of 9), against the oracle."""
    from paper_2608_12058_b300 import api

    n = 25
    assert api.get_fused_split(n) == (0, 14)
    h, J = I.sk_instance(n, 125)
    psi = I.random_state(n, 126)
    ref, oinfo = oracle.expmv(h, J, 0.9, 0.15, psi, 2.0 ** -23)
    y, info = _run(h, J, 0.9, 0.15, psi, "fp32", 2.0 ** -23, path="fused")
    assert info["K"] == oinfo["K"] and info["K"] > 3
    assert _rel(y, ref) <= TOL["fp32"]


@pytest.mark.parametrize("n,l,h", [(24, 0, 13), (26, 0, 15)])
def test_wide_row_passes_match_oracle(cuda_lib, oracle, n, l, h):
    """Splits whose top strided pass (6 or 7 bits starting at bit 18 or 19) runs on rows
    of 32 amplitudes (256 B), against the oracle (FP32)."""
    from paper_2608_12058_b300 import api

    hq, Jq = I.sk_instance(n, 400 + n)
    psi = I.random_state(n, 401 + n)
    ref, oinfo = oracle.expmv(hq, Jq, 0.9, 0.15, psi, 2.0 ** -23)
    api.set_fused_split(n, l, h)
    try:
        y, info = _run(hq, Jq, 0.9, 0.15, psi, "fp32", 2.0 ** -23, path="fused")
    finally:
        api.set_fused_split(n, -1)
    assert info["K"] == oinfo["K"] and info["K"] > 3
    assert _rel(y, ref) <= TOL["fp32"]


@pytest.mark.parametrize("prec,n", [("fp32", 14), ("fp32", 15), ("fp32", 17), ("fp64", 13), ("fp64", 16)])
def test_cluster_path_matches_oracle(cuda_lib, oracle, prec, n):
    """The whole run on one thread-block cluster (vectors in distributed shared memory,
    2..16 CTAs) against the oracle, forced and through the automatic choice."""
    h, J = I.sk_instance(n, 120 + n)
    psi = I.random_state(n, 121 + n)
    tol = 1e-12 if prec == "fp64" else 2.0 ** -23
    ref, oinfo = oracle.expmv(h, J, 0.8, 3.0, psi, tol)
    for path in ("cluster", "auto"):
        y, info = _run(h, J, 0.8, 3.0, psi, prec, tol, path=path)
        assert info["K"] == oinfo["K"]
        assert _rel(y, ref) <= TOL[prec], path


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_remez_method_matches_dense_exponential(cuda_lib, oracle, prec):
    """Remez minimax coefficients (the product's host generator; the oracle has no
    Remez) through the GPU path agree with the dense exp(-itH) psi to within the
    series tolerance plus the precision's rounding."""
    n = 9
    h, J = I.sk_instance(n, 79)
    psi = I.random_state(n, 80)
    tol = 1e-10 if prec == "fp64" else 2.0 ** -23
    ref = oracle.dense_expmv(h, J, 0.9, 5.0, psi)
    y, info = _run(h, J, 0.9, 5.0, psi, prec, tol, method="remez")
    _, cinfo = oracle.expmv(h, J, 0.9, 5.0, psi, tol, method="cf")
    assert info["K"] == cinfo["K"]
    assert _rel(y, ref) <= tol + TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [9, 14])
def test_time_splits_match_oracle(cuda_lib, oracle, prec, n):
    h, J = I.sk_instance(n, 90 + n)
    psi = I.random_state(n, 91)
    tol = 1e-12 if prec == "fp64" else 2.0 ** -23
    ref, oinfo = oracle.expmv(h, J, 0.7, 9.0, psi, tol, splits=3)
    y, info = _run(h, J, 0.7, 9.0, psi, prec, tol, splits=3)
    assert info["time_splits"] == 3 and info["K"] == oinfo["K"]
    assert _rel(y, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_degenerate_degrees(cuda_lib, oracle, prec):
    """t = 0 (degree 0: y = psi) and a tiny t with a loose tolerance (degree 1)."""
    n = 11
    h, J = I.sk_instance(n, 5)
    psi = I.random_state(n, 6)
    y, info = _run(h, J, 1.0, 0.0, psi, prec, 1e-6)
    assert info["K"] == 0
    assert _rel(y, psi) <= TOL[prec]
    ref, oinfo = oracle.expmv(h, J, 1.0, 1e-3, psi, 1e-3)
    y, info = _run(h, J, 1.0, 1e-3, psi, prec, 1e-3)
    assert info["K"] == oinfo["K"] == 1
    assert _rel(y, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [8, 17])
def test_closed_forms(cuda_lib, prec, n):
    """H_P = 0: product of cos(gt) I - i sin(gt) X over qubits; gamma = 0: pure phases."""
    gamma, t = 0.9, 1.7
    y, _ = _run(np.zeros(n), np.zeros((n, n)), gamma, t, I.basis_state(n, 0), prec, 1e-13 if prec == "fp64" else 2.0 ** -23)
    w = np.array([bin(v).count("1") for v in range(1 << n)])
    ref = np.cos(gamma * t) ** (n - w) * (-1j * np.sin(gamma * t)) ** w
    assert _rel(y, ref) <= TOL[prec]
    h, J = I.sk_instance(n, 3)
    psi = I.random_state(n, 4)
    y, _ = _run(h, J, 0.0, 3.0, psi, prec, 1e-13 if prec == "fp64" else 2.0 ** -23)
    from oracle import oracle as O

    E = O.energies(h, J)
    assert _rel(y, np.exp(-3j * E) * psi) <= TOL[prec]


def test_bounds_and_energy_entry_points(cuda_lib, oracle):
    torch = _torch()
    from paper_2608_12058_b300 import api

    for n in [5, 13, 18]:
        h, J = I.sk_instance(n, 60 + n, "uniform")
        lo, hi = api.ising_bounds(h, J)
        emin, emax, _, _ = oracle.bounds(h, J, 1.0)
        assert abs(lo - emin) < 1e-12 and abs(hi - emax) < 1e-12
        psi = I.random_state(n, 3)
        e, nn = api.energy(h, J, torch.from_numpy(psi).cuda())
        re, rn = oracle.energy_norm(h, J, psi)
        assert abs(e - re) < 1e-12 * max(1, abs(re)) and abs(nn - rn) < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_poly_apply_matches_oracle_clenshaw(cuda_lib, oracle, prec):
    """Caller-supplied Chebyshev coefficients (degree-50 random series, the kind of
    polynomial timed in Fig. 4 / Fig. 6), same Ht as the oracle's Clenshaw."""
    torch = _torch()
    from paper_2608_12058_b300 import api

    n = 14
    h, J = I.sk_instance(n, 101)
    rng = np.random.default_rng(5)
    c = (rng.standard_normal(51) + 1j * rng.standard_normal(51)) / 8
    emin, emax, center, r = oracle.bounds(h, J, 0.6)
    D = (oracle.energies(h, J) - center) / r
    psi = I.random_state(n, 102)
    ref = oracle.clenshaw(D, 0.6 / r, c, psi)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    x = torch.from_numpy(psi).to(dt).cuda()
    api.poly_apply(h, J, 0.6, center, r, c, x)
    y = x.cpu().numpy().astype(np.complex128)
    assert _rel(y, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,seed", [(5, 11), (10, 12), (16, 13), (20, 14)])
def test_monomial_polynomial_matches_oracle(cuda_lib, oracle, prec, n, seed):
    """The Fig. 4 / Fig. 6 workload: a degree-50 polynomial with N(0,1) coefficients in
    the monomial basis, applied to Ht = (H - c)/r of an SK instance. The product converts
    to the Chebyshev basis on the host and runs the Clenshaw kernels; the oracle sums
    a_m Ht^m psi by repeated matvecs."""
    torch = _torch()
    from paper_2608_12058_b300 import api

    h, J = I.sk_instance(n, seed)
    a = I.monomial_polynomial(50, seed)
    emin, emax, center, r = oracle.bounds(h, J, 0.9)
    D = (oracle.energies(h, J) - center) / r
    psi = I.random_state(n, seed + 100)
    ref = oracle.monomial_apply(D, 0.9 / r, a, psi)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    x = torch.from_numpy(psi).to(dt).cuda()
    api.poly_apply_monomial(h, J, 0.9, center, r, a, x)
    y = x.cpu().numpy().astype(np.complex128)
    assert _rel(y, ref) <= TOL[prec]


SPLITS = [
    # n, l, h: L2 partner bits of the low pass and strided bits (11 + l + h = n);
    # h > 9 runs two strided passes
    (11, 0, 0),
    (12, 1, 0),
    (15, 4, 0),
    (16, 2, 3),
    (16, 0, 5),
    (17, 6, 0),
    (17, 3, 3),
    (18, 1, 6),
    (19, 0, 8),
    (20, 2, 7),
    (21, 1, 9),
    (21, 6, 4),
    (22, 0, 11),
    (22, 4, 7),
    (23, 0, 12),
]


@pytest.mark.parametrize("n,l,h", SPLITS)
def test_fused_splits_match_oracle(cuda_lib, oracle, n, l, h):
    """Every way of splitting the bit flips between the shared-memory tile, the L2
    partner tiles and the strided high pass gives the oracle's result (FP32)."""
    from paper_2608_12058_b300 import api

    hq, Jq = I.sk_instance(n, 200 + n + l)
    psi = I.random_state(n, 300 + n)
    t = 0.6 if n >= 20 else 2.5
    ref, oinfo = oracle.expmv(hq, Jq, 0.8, t, psi, 2.0 ** -23)
    api.set_fused_split(n, l, h)
    try:
        y, info = _run(hq, Jq, 0.8, t, psi, "fp32", 2.0 ** -23, path="fused")
    finally:
        api.set_fused_split(n, -1)
    assert info["K"] == oinfo["K"]
    assert _rel(y, ref) <= TOL["fp32"]


@pytest.mark.parametrize("prec,n", [("fp32", 22), ("fp32", 25), ("fp64", 22)])
def test_programmatic_launch_gives_identical_results(cuda_lib, prec, n):
    """The fused step kernels launched with programmatic dependent launch (the default)
    and without it give bit-identical results: each kernel waits for its predecessor
    before reading what it wrote."""
    import torch

    from paper_2608_12058_b300 import api

    h, J = I.sk_instance(n, 300 + n)
    psi = I.random_state(n, 301 + n)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    out = []
    for on in (True, False):
        api.set_programmatic_launch(on)
        try:
            x = torch.from_numpy(psi).to(dt).cuda()
            api.expmv(h, J, 0.9, 2.0, x, tol=2.0 ** -23 if prec == "fp32" else 1e-12, path="fused")
            torch.cuda.synchronize()
            out.append(x.cpu())
        finally:
            api.set_programmatic_launch(True)
    assert torch.equal(out[0], out[1])
