"""The L2-blocked step tail (the last strided pass and the low pass of the fused FP32
step in one persistent launch, cheb_set_fused_blocking) against the oracle and
against the separate launches.

Per amplitude the blocked tail performs the same FP32 operations in the same order as
the separate launches, so the two agree bit for bit; the oracle comparison uses the
FP32 bar (relative L2 1e-5). Splits cover last strided ranges of 6..9 bits, zero and
one L2 partner bit, c_k = 0 steps (the psi tile is skipped), the final step written
into psi, and the adjoint chain."""
import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _blocking(on):
    from paper_2608_12058_b300 import api

    api.set_fused_blocking(on)


@pytest.fixture
def split():
    """Set a fused split for one test and restore the default afterwards."""
    from paper_2608_12058_b300 import api

    used = []

    def set_(n, l, h):
        api.set_fused_split(n, l, h)
        used.append(n)

    yield set_
    for n in used:
        api.set_fused_split(n, -1)
    _blocking(None)  # back to the automatic choice


def _expmv(h, J, gamma, t, psi_np, blocking):
    import torch

    from paper_2608_12058_b300 import api

    _blocking(blocking)
    psi = torch.from_numpy(psi_np.astype(np.complex64)).cuda()
    info = api.expmv(h, J, gamma, t, psi, tol=2.0 ** -23, path="fused")
    torch.cuda.synchronize()
    return psi.cpu().numpy(), info


def _rel(y, ref):
    return np.linalg.norm(y.astype(np.complex128) - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("n,l,h", [(23, 0, 12), (24, 1, 12), (25, 0, 14)])
def test_blocked_tail_matches_oracle(cuda_lib, oracle, split, n, l, h):
    """Last strided range of 6 or 7 bits, l = 0 and 1, against the FP64 oracle."""
    from paper_2608_12058_b300 import api

    split(n, l, h)
    hq, Jq = I.sk_instance(n, 900 + n + l)
    psi = I.random_state(n, 950 + n)
    ref, oinfo = oracle.expmv(hq, Jq, 0.8, 0.25, psi, 2.0 ** -23)
    c0 = api.launch_count()
    y, info = _expmv(hq, Jq, 0.8, 0.25, psi, True)
    # per step: the first strided pass and one blocked tail (not three launches)
    blocked = api.launch_count() - c0
    assert info["K"] == oinfo["K"] and info["K"] > 3
    assert _rel(y, ref) <= 1e-5
    c1 = api.launch_count()
    y_sep, _ = _expmv(hq, Jq, 0.8, 0.25, psi, False)
    assert (api.launch_count() - c1) - blocked == info["K"]
    assert np.array_equal(y, y_sep)


def _poly(n, coef, blocking, seed=0):
    import torch

    from paper_2608_12058_b300 import api

    c = I.config_family(n, 1.0, 1.0, seed, "uniform")
    _blocking(blocking)
    g = torch.Generator(device="cuda").manual_seed(40 + n)
    x = torch.randn(1 << n, dtype=torch.complex64, device="cuda", generator=g)
    x /= torch.linalg.vector_norm(x)
    api.poly_apply(c.h, c.J, 1.0, 0.0, 80.0, coef, x, path="fused")
    api.check_status(n, "fp32")  # no bounded wait ran out
    return x


@pytest.mark.parametrize("n,l,h", [(26, 1, 14), (28, 0, 17), (29, 0, 18), (30, 1, 18)])
def test_blocked_tail_bit_identical(cuda_lib, split, n, l, h):
    """Last ranges of 7, 8 and 9 bits at up to 2^30 amplitudes: the blocked tail equals
    the separate launches bit for bit, including steps with c_k = 0 (no psi read) and a
    degree-1 term (the final step alone, written into psi)."""
    split(n, l, h)
    rng = np.random.default_rng(n)
    coef = (rng.standard_normal(8) + 1j * rng.standard_normal(8)) / 32
    coef[2] = 0.0  # a step with c_k = 0
    coef[5] = 0.0
    a = _poly(n, coef, True)
    b = _poly(n, coef, False)
    assert bool((a == b).all())
    assert bool(torch_isfinite(a))
    del a, b
    one = np.array([0.3 + 0.1j, 0.5 - 0.2j])
    a = _poly(n, one, True)
    b = _poly(n, one, False)
    assert bool((a == b).all())


def torch_isfinite(x):
    import torch

    return torch.isfinite(torch.view_as_real(x)).all()


def test_blocked_tail_adjoint_identical(cuda_lib, split):
    """The adjoint's reverse Clenshaw chain (c_k = 0 steps on the fused kernels) gives
    the same gradients with the blocked tail as with the separate launches."""
    import torch

    from paper_2608_12058_b300 import api

    n = 23
    split(n, 0, 12)
    a = I.config_anneal(n=n, S=4)
    outs = []
    for blocking in (True, False):
        _blocking(blocking)
        x = torch.full((1 << n,), 2 ** (-n / 2), dtype=torch.complex64, device="cuda")
        bnd = torch.empty((a.gammas.shape[0], 1 << n), dtype=torch.complex64, device="cuda")
        api.anneal(a.h, a.J, a.gammas, a.ts, x, boundaries=bnd, info=False)
        _, g, _, _ = api.energy_grad(a.h, a.J, x)
        out = api.anneal_adjoint(a.h, a.J, a.gammas, a.ts, bnd, x, g)
        torch.cuda.synchronize()
        outs.append((x.cpu().numpy(), out))
    (x1, o1), (x2, o2) = outs
    assert np.array_equal(x1, x2)
    for key in ("gamma", "t", "h", "J"):
        assert np.array_equal(np.asarray(o1[key]), np.asarray(o2[key])), key


def test_blocked_tail_bit_identical_compensated(cuda_lib, split):
    """With compensated flip sums the blocked tail and the separate launches still
    perform the same operations in the same order: bit-identical results."""
    from paper_2608_12058_b300 import api

    n = 26
    split(n, 1, 14)
    rng = np.random.default_rng(7)
    coef = (rng.standard_normal(8) + 1j * rng.standard_normal(8)) / 32
    api.set_fused_compensated(True)
    try:
        a = _poly(n, coef, True)
        b = _poly(n, coef, False)
        api.set_fused_compensated(False)
        c = _poly(n, coef, False)
    finally:
        api.set_fused_compensated(False)
    assert bool((a == b).all())
    assert not bool((a == c).all())  # the switch changes the arithmetic


# ---------------------------------------------------------------------------
# The L2-blocked strided pair (cheb_set_fused_blocking(2)): both strided passes of a
# two-pass split in one launch. The same flip sums in the same order as the separate
# launches, so results are bit-identical; the oracle comparison uses the FP32 bar.

@pytest.mark.parametrize("n,l,h", [(23, 0, 12), (25, 0, 14), (26, 1, 14)])
def test_blocked_pair_matches_oracle(cuda_lib, oracle, split, n, l, h):
    """Ranges of 6+6, 7+7 and 7+7 bits, against the FP64 oracle and the separate
    launches (two launches per step instead of three)."""
    from paper_2608_12058_b300 import api

    split(n, l, h)
    hq, Jq = I.sk_instance(n, 700 + n + l)
    psi = I.random_state(n, 750 + n)
    ref, oinfo = oracle.expmv(hq, Jq, 0.8, 0.25, psi, 2.0 ** -23)
    c0 = api.launch_count()
    y, info = _expmv(hq, Jq, 0.8, 0.25, psi, 2)
    paired = api.launch_count() - c0
    assert info["K"] == oinfo["K"] and info["K"] > 3
    assert _rel(y, ref) <= 1e-5
    c1 = api.launch_count()
    y_sep, _ = _expmv(hq, Jq, 0.8, 0.25, psi, 0)
    assert (api.launch_count() - c1) - paired == info["K"]
    assert np.array_equal(y, y_sep)


@pytest.mark.parametrize("n,l,h", [(24, 0, 13), (27, 0, 16), (28, 1, 16), (29, 0, 18), (30, 2, 17),
                                   (30, 3, 16), (30, 4, 15)])
def test_blocked_pair_bit_identical(cuda_lib, split, n, l, h):
    """Range pairs 7+6, 8+8, 9+9, 9+8, 8+8 and 8+7 up to 2^30 amplitudes: the blocked
    pair equals the separate launches bit for bit, including steps with c_k = 0 and the
    final step alone."""
    split(n, l, h)
    rng = np.random.default_rng(n + l)
    coef = (rng.standard_normal(8) + 1j * rng.standard_normal(8)) / 32
    coef[2] = 0.0
    coef[5] = 0.0
    a = _poly(n, coef, 2)
    b = _poly(n, coef, 0)
    assert bool((a == b).all())
    assert bool(torch_isfinite(a))
    del a, b
    one = np.array([0.3 + 0.1j, 0.5 - 0.2j])
    a = _poly(n, one, 2)
    b = _poly(n, one, 0)
    assert bool((a == b).all())


def test_blocked_pair_adjoint_identical(cuda_lib, split):
    """The adjoint chain on the blocked pair gives the same gradients as on the
    separate launches."""
    import torch

    from paper_2608_12058_b300 import api

    n = 24
    split(n, 0, 13)
    a = I.config_anneal(n=n, S=3)
    outs = []
    for mode in (2, 0):
        _blocking(mode)
        x = torch.full((1 << n,), 2 ** (-n / 2), dtype=torch.complex64, device="cuda")
        bnd = torch.empty((a.gammas.shape[0], 1 << n), dtype=torch.complex64, device="cuda")
        api.anneal(a.h, a.J, a.gammas, a.ts, x, boundaries=bnd, info=False)
        _, g, _, _ = api.energy_grad(a.h, a.J, x)
        out = api.anneal_adjoint(a.h, a.J, a.gammas, a.ts, bnd, x, g)
        torch.cuda.synchronize()
        outs.append((x.cpu().numpy(), out))
    (x1, o1), (x2, o2) = outs
    assert np.array_equal(x1, x2)
    for key in ("gamma", "t", "h", "J"):
        assert np.array_equal(np.asarray(o1[key]), np.asarray(o2[key])), key
