"""The fused float-float step of the FP64 path (complex128 storage, arithmetic on the
FP32 units with error-free transformations) against the FP64 oracle at the FP64 bar,
relative L2 1e-12, under its default splits and forced ones: the low pass alone, one
and two strided passes, 256-byte rows, several L2 partner bits, time slices, CF
coefficients, degenerate degrees and the evaluation bound with u = 2^-47."""
import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu

BAR = 1e-12


def _run(h, J, gamma, t, psi_np, tol=1e-12, method="chebyshev", path="fused", splits=0, eval_bound=False):
    import torch

    from paper_2608_12058_b300 import api

    psi = torch.from_numpy(psi_np.astype(np.complex128)).cuda()
    info = api.expmv(h, J, gamma, t, psi, tol=tol, method=method, path=path, time_splits=splits,
                     eval_bound=eval_bound)
    torch.cuda.synchronize()
    return psi.cpu().numpy(), info


def _rel(y, ref):
    return float(np.linalg.norm(y - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("n,split,t", [
    (11, None, 3.0),          # low pass with one partner bit
    (13, None, 3.0),          # three partner bits
    (15, (5, 0), 2.0),        # five partner bits
    (16, None, 2.0),          # one strided pass of 6 bits
    (17, (1, 6), 2.0),
    (18, (0, 8), 2.0),
    (19, None, 1.5),          # a 9-bit pass
    (20, (4, 6), 1.0),        # four partner bits and a 6-bit pass
    (21, None, 1.0),          # one pass and two partner bits
    (22, (0, 12), 0.6),       # two passes of 6 bits, the top one at bit 16
    (23, (0, 13), 0.4),       # 7 + 6, top pass on wide rows
    (24, None, 0.3),          # the n=24 default (7 + 7, top pass on wide rows)
])
def test_ff_fused_matches_oracle(cuda_lib, oracle, n, split, t):
    from paper_2608_12058_b300 import api

    h, J = I.sk_instance(n, 600 + n)
    psi = I.random_state(n, 601 + n)
    ref, oinfo = oracle.expmv(h, J, 0.9, t, psi, 1e-12)
    if split is not None:
        api.set_fused_split_fp64(n, *split)
    try:
        y, info = _run(h, J, 0.9, t, psi)
    finally:
        api.set_fused_split_fp64(n, -1)
    assert info["K"] == oinfo["K"] and info["K"] >= 10
    err = _rel(y, ref)
    print(f"n={n} split {split or api.get_fused_split_fp64(n)}: K={info['K']} rel L2 vs oracle {err:.3e}")
    assert err <= BAR, err
    assert abs(info["norm"] - oinfo["norm"]) <= 1e-12


def test_ff_auto_path_is_fused_above_16(cuda_lib, oracle):
    """AUTO takes the float-float fused step for FP64 from n = 17 (launch count per step:
    one strided pass + one low pass at n = 17)."""
    from paper_2608_12058_b300 import api

    n = 17
    h, J = I.sk_instance(n, 17)
    psi = I.random_state(n, 18)
    ref, oinfo = oracle.expmv(h, J, 1.1, 2.0, psi, 1e-12)
    c0 = api.launch_count()
    y, info = _run(h, J, 1.1, 2.0, psi, path="auto")
    launches = api.launch_count() - c0
    assert _rel(y, ref) <= BAR
    assert launches >= 2 * info["K"]


@pytest.mark.parametrize("method", ["chebyshev", "cf"])
def test_ff_time_splits_and_cf(cuda_lib, oracle, method):
    n = 18
    h, J = I.sk_instance(n, 33)
    psi = I.random_state(n, 34)
    ref, oinfo = oracle.expmv(h, J, 0.7, 4.0, psi, 1e-12, method=method, splits=3)
    y, info = _run(h, J, 0.7, 4.0, psi, method=method, splits=3)
    assert info["time_splits"] == 3 and info["K"] == oinfo["K"]
    assert _rel(y, ref) <= BAR


def test_ff_degenerate_degrees(cuda_lib, oracle):
    """Degree 0 (y = c_0 psi) and degree 1 (the final step alone, b_2 = 0)."""
    from paper_2608_12058_b300 import api
    import torch

    n = 16
    h, J = I.sk_instance(n, 44)
    psi = I.random_state(n, 45)
    for coef in (np.array([0.3 - 0.2j]), np.array([0.3 - 0.2j, -0.1 + 0.4j]), np.array([0.3, 0.2j, -0.1])):
        emin, emax, c, r = oracle.bounds(h, J, 0.8)
        D = (oracle.energies(h, J) - c) / r
        ref = oracle.clenshaw(D, 0.8 / r, coef, psi)
        x = torch.from_numpy(psi).cuda()
        api.poly_apply(h, J, 0.8, c, r, coef, x, path="fused")
        assert _rel(x.cpu().numpy(), ref) <= BAR, coef


def test_ff_eval_bound(cuda_lib, oracle):
    """The evaluation bound of the float-float step uses u = 2^-47 and bounds the
    observed difference from the oracle."""
    n = 20
    h, J = I.sk_instance(n, 520)
    psi = I.random_state(n, 521)
    emin, emax, c, r = oracle.bounds(h, J, 1.1)
    D = (oracle.energies(h, J) - c) / r
    coef, K, _ = oracle.cheb_coeffs(4.0 * r, 1e-12, np.exp(-1j * 4.0 * c))
    ref, norms = oracle.clenshaw(D, 1.1 / r, coef, psi, with_norms=True)
    ob = oracle.eval_bound(n, norms, 2.0 ** -47)
    y, info = _run(h, J, 1.1, 4.0, psi, eval_bound=True)
    gb = info["eval_bound"]
    err = float(np.linalg.norm(y - ref))
    print(f"n={n} float-float: eval_bound {gb:.3e} (oracle {ob:.3e}), observed {err:.3e}")
    assert abs(gb - ob) <= 1e-3 * ob
    assert err <= gb


# ---------------------------------------------------------------------------
# The L2-blocked strided pair on the float-float step (cheb_set_fused_blocking(2)): the
# same Sum2 flip sums in the same order as the separate launches, so the results agree
# bit for bit; against the oracle at the FP64 bar.

@pytest.mark.parametrize("n,split", [(22, (0, 12)), (23, (0, 13)), (25, (1, 14))])
def test_ff_blocked_pair_matches_oracle_and_separate(cuda_lib, oracle, n, split):
    """Range pairs 6+6, 7+6 and 7+7 against the FP64 oracle and, bit for bit, against
    the separate launches (two launches per step instead of three)."""
    from paper_2608_12058_b300 import api

    h, J = I.sk_instance(n, 640 + n)
    psi = I.random_state(n, 641 + n)
    ref, oinfo = oracle.expmv(h, J, 0.9, 0.3, psi, 1e-12)
    api.set_fused_split_fp64(n, *split)
    try:
        api.set_fused_blocking(2)
        c0 = api.launch_count()
        y, info = _run(h, J, 0.9, 0.3, psi)
        paired = api.launch_count() - c0
        api.set_fused_blocking(0)
        c1 = api.launch_count()
        y_sep, _ = _run(h, J, 0.9, 0.3, psi)
        separate = api.launch_count() - c1
    finally:
        api.set_fused_blocking(None)
        api.set_fused_split_fp64(n, -1)
    assert info["K"] == oinfo["K"] and info["K"] >= 10
    assert separate - paired == info["K"]
    assert np.array_equal(y, y_sep)
    assert _rel(y, ref) <= BAR


def _ff_poly(n, coef, mode):
    import torch

    from paper_2608_12058_b300 import api

    c = I.config_family(n, 1.0, 1.0, 0, "uniform")
    api.set_fused_blocking(mode)
    g = torch.Generator(device="cuda").manual_seed(70 + n)
    x = torch.randn(1 << n, dtype=torch.complex128, device="cuda", generator=g)
    x /= torch.linalg.vector_norm(x)
    api.poly_apply(c.h, c.J, 1.0, 0.0, 80.0, coef, x, path="fused")
    api.check_status(n, "fp64")
    return x


@pytest.mark.parametrize("n,split", [(26, (0, 16)), (28, (1, 17)), (29, (2, 17))])
def test_ff_blocked_pair_bit_identical(cuda_lib, n, split):
    """8+8, 9+8 and 9+8 ranges up to 2^29 float-float amplitudes: the blocked pair equals
    the separate launches bit for bit, including steps with c_k = 0 and the final step
    alone."""
    from paper_2608_12058_b300 import api

    rng = np.random.default_rng(n)
    coef = (rng.standard_normal(6) + 1j * rng.standard_normal(6)) / 32
    coef[2] = 0.0
    api.set_fused_split_fp64(n, *split)
    try:
        a = _ff_poly(n, coef, 2)
        b = _ff_poly(n, coef, 0)
        assert bool((a == b).all())
        del a, b
        one = np.array([0.3 + 0.1j, 0.5 - 0.2j])
        a = _ff_poly(n, one, 2)
        b = _ff_poly(n, one, 0)
        assert bool((a == b).all())
    finally:
        api.set_fused_blocking(None)
        api.set_fused_split_fp64(n, -1)
