"""The full n = 30 size in the launch configuration the benchmark times (complex64,
fused split (2, 17): the low pass with two L2 partner bits, a strided pass of 9 bits and
one of 8 bits in 256-byte rows).

The oracle cannot hold or evolve 2^30 amplitudes in test time, so the checks are
closed forms evaluated on sampled amplitudes and properties that hold at any size:
  * H_P = 0: the exact product over qubits of cos(gt) I - i sin(gt) X;
  * gamma = 0: pure phases exp(-i t E(z)), E(z) from the definition at sampled z;
  * the SK n=30 workload: norm and <H> conservation (H = c + r Ht, Ht psi from the
    library's polynomial entry point with coefficients (0, 1))."""
import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu

N30 = 30


def _energy_at(h, J, z):
    """E(z) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i, s_i = 1 - 2 bit_i(z), at sampled z."""
    n = h.shape[0]
    s = 1.0 - 2.0 * ((z[:, None] >> np.arange(n)[None, :]) & 1)
    return np.einsum("ki,ij,kj->k", s, np.triu(J, 1), s) + s @ h


def _samples(seed, count=1 << 20):
    return np.random.default_rng(seed).integers(0, 1 << N30, size=count, dtype=np.int64)


def test_n30_fused_split_is_the_benchmarked_one(cuda_lib):
    from paper_2608_12058_b300 import api

    assert api.get_fused_split(N30) == (2, 17)


def test_n30_transverse_field_closed_form(cuda_lib):
    import torch

    from paper_2608_12058_b300 import api

    gamma, t = 1.0, 0.6
    x = torch.zeros(1 << N30, dtype=torch.complex64, device="cuda")
    x[0] = 1.0
    info = api.expmv(np.zeros(N30), np.zeros((N30, N30)), gamma, t, x, tol=2.0 ** -23)
    assert info["K"] > 3
    z = _samples(1)
    w = np.array([bin(int(v)).count("1") for v in z])
    ref = np.cos(gamma * t) ** (N30 - w) * (-1j * np.sin(gamma * t)) ** w
    got = x[torch.from_numpy(z).cuda()].cpu().numpy().astype(np.complex128)
    # relative to the largest amplitudes (the sampled set holds tiny ones too)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 1e-5 * scale
    nrm = float(torch.linalg.vector_norm(x.to(torch.complex128)))
    assert abs(nrm - 1.0) < 1e-5


def test_n30_zero_field_pure_phase(cuda_lib):
    import torch

    from paper_2608_12058_b300 import api

    c = I.config_n30()
    t = 2.0
    x = torch.full((1 << N30,), 2 ** (-N30 / 2), dtype=torch.complex64, device="cuda")
    api.expmv(c.h, c.J, 0.0, t, x, tol=2.0 ** -23)
    z = _samples(2)
    ref = np.exp(-1j * t * _energy_at(c.h, c.J, z)) * 2 ** (-N30 / 2)
    got = x[torch.from_numpy(z).cuda()].cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= 1e-5 * 2 ** (-N30 / 2)


def test_n30_workload_conserves_norm_and_energy(cuda_lib):
    """The benchmark's exp(-itH)psi (t = 20, K = 1166): ||y|| = 1 and <y|H|y> = <psi|H|psi>."""
    import torch

    from paper_2608_12058_b300 import api

    c = I.config_n30()

    def mean_H(v, center, radius):
        w = v.clone()
        api.poly_apply(c.h, c.J, c.gamma, center, radius, np.array([0.0, 1.0]), w)
        e = torch.vdot(v.to(torch.complex128), w.to(torch.complex128)).real.item()
        del w
        return center + radius * e

    x = torch.full((1 << N30,), 2 ** (-N30 / 2), dtype=torch.complex64, device="cuda")
    info = api.expmv(c.h, c.J, c.gamma, c.t, x, tol=2.0 ** -23, info=True)
    assert info["K"] == 1166
    assert abs(info["norm"] - 1.0) < 2e-5
    center, radius = info["center"], info["radius"]
    y_H = mean_H(x, center, radius)
    x0 = torch.full((1 << N30,), 2 ** (-N30 / 2), dtype=torch.complex64, device="cuda")
    x0_H = mean_H(x0, center, radius)
    del x0
    # uniform start: <H_X> = n and <H_P> = mean of E over all z = 0 (each s_i and each
    # s_i s_j sums to zero), so <H> = gamma n exactly
    assert abs(x0_H - c.gamma * N30) <= 1e-5 * radius
    assert abs(y_H - x0_H) <= 2e-4 * radius


def test_n30_adjoint_gradients(cuda_lib):
    """Reverse-Clenshaw gradients at the full n = 30 size (one segment of the SK
    workload, t = 0.15, K = 20): the complex64 checkpointed forward keeps its start state
    and places one anchor pair, the adjoint regenerates the Clenshaw vectors in a ring
    of 6 from it, and
    dL/dgamma, dL/dt and dL/dh_i of L = <psi_T|H_P|psi_T> match central differences of
    the FP64 forward map within 1e-4."""
    import torch

    from paper_2608_12058_b300 import api

    c = I.config_n30()
    gamma, t = np.array([c.gamma]), np.array([0.15])
    store = 8
    ws_bytes = int(cuda_lib.cheb_adjoint_workspace_bytes(N30, 0, store))
    print(f"n=30 adjoint workspace ({store} state vectors): {ws_bytes / 2**30:.1f} GiB")
    y = torch.full((1 << N30,), 2 ** (-N30 / 2), dtype=torch.complex64, device="cuda")
    bnd = torch.empty((1, 1 << N30), dtype=torch.complex64, device="cuda")
    ck = api.anneal_checkpointed(c.h, c.J, gamma, t, y, bnd, store_vectors=store)
    e, g, gh, gJ = api.energy_grad(c.h, c.J, y)
    torch.cuda.empty_cache()
    out = api.anneal_adjoint(c.h, c.J, gamma, t, bnd, y, g, checkpoint=ck)
    del ck
    got = {"gamma": out["gamma"][0], "t": out["t"][0], "h": out["h"][5] + gh[5]}
    del y, bnd, g
    api.release_workspaces()
    torch.cuda.empty_cache()

    def loss(h_, g_, t_):
        x = torch.full((1 << N30,), 2 ** (-N30 / 2), dtype=torch.complex128, device="cuda")
        api.anneal(h_, c.J, g_, t_, x, tol=1e-13, info=False)
        v = api.energy(h_, c.J, x)[0]
        del x
        return v

    eps = 1e-4
    refs = {}
    for key in ("gamma", "t", "h"):
        vals = []
        for sgn in (+1, -1):
            h_, g_, t_ = c.h.copy(), gamma.copy(), t.copy()
            {"gamma": g_, "t": t_, "h": h_}[key][0 if key != "h" else 5] += sgn * eps
            vals.append(loss(h_, g_, t_))
        refs[key] = (vals[0] - vals[1]) / (2 * eps)
    api.release_workspaces()
    scale = max(abs(v) for v in refs.values())
    for key, ref in refs.items():
        print(f"n=30 dL/d{key}: adjoint {got[key]:.8e}, central difference {ref:.8e}")
        assert abs(got[key] - ref) <= 1e-4 * max(abs(ref), scale), (key, got[key], ref)
