"""Reverse-Clenshaw gradients (cheb_anneal_adjoint, cheb_energy_grad) through the
torch.autograd wrappers, against the FP64 oracle's exact Frechet-derivative
gradients and against central finite differences of the GPU forward map."""
import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _params(h, J, gammas, ts):
    import torch

    t = lambda x: torch.tensor(np.asarray(x, dtype=np.float64), requires_grad=True)
    return t(h), t(J), t(gammas), t(ts)


def test_expmv_gradients_match_frechet_oracle(cuda_lib, oracle):
    import torch

    from paper_2608_12058_b300 import autograd as AG

    n = 5
    h, J = I.sk_instance(n, 21)
    psi0 = I.random_state(n, 22)
    gam, tt = 0.8, 1.3
    ref = oracle.dense_energy_gradients(h, J, gam, tt, psi0)
    th, tJ, tg, tT = _params(h, J, [gam], [tt])
    x = torch.from_numpy(psi0).cuda().requires_grad_(True)
    y = AG.anneal(x, th, tJ, tg, tT, tol=1e-13)
    L = AG.energy(y, th, tJ)
    L.backward()
    assert abs(L.item() - ref["loss"]) < 1e-11
    assert abs(tg.grad[0].item() - ref["gamma"]) < 1e-9 * max(1, abs(ref["gamma"]))
    assert abs(tT.grad[0].item() - ref["t"]) < 1e-9 * max(1, abs(ref["t"]))
    np.testing.assert_allclose(th.grad.numpy(), ref["h"], atol=1e-9)
    np.testing.assert_allclose(np.triu(tJ.grad.numpy(), 1), np.triu(ref["J"], 1), atol=1e-9)
    np.testing.assert_allclose(x.grad.cpu().numpy(), ref["psi0"], atol=1e-9)


def _energy_after(h, J, gammas, ts, psi0, dtype):
    import torch

    from paper_2608_12058_b300 import api

    x = torch.from_numpy(psi0).to(dtype).cuda()
    api.anneal(h, J, gammas, ts, x, tol=1e-13 if dtype == torch.complex128 else 2.0 ** -23, info=False)
    return api.energy(h, J, x)[0]


@pytest.mark.parametrize("n,S", [(8, 4), (12, 3)])
def test_anneal_gradients_vs_finite_differences(cuda_lib, n, S):
    import torch

    from paper_2608_12058_b300 import autograd as AG

    a = I.config_anneal(n=n, S=S, seed=5)
    psi0 = I.uniform_state(n)
    th, tJ, tg, tT = _params(a.h, a.J, a.gammas, a.ts)
    x = torch.from_numpy(psi0).cuda()
    L = AG.energy(AG.anneal(x, th, tJ, tg, tT, tol=1e-13), th, tJ)
    L.backward()
    eps = 1e-5

    def fd(mod):
        hp, Jp, gp, tp = [np.array(v, dtype=np.float64) for v in (a.h, a.J, a.gammas, a.ts)]
        hm, Jm, gm, tm = [np.array(v, dtype=np.float64) for v in (a.h, a.J, a.gammas, a.ts)]
        mod(hp, Jp, gp, tp, +eps)
        mod(hm, Jm, gm, tm, -eps)
        return (_energy_after(hp, Jp, gp, tp, psi0, torch.complex128) -
                _energy_after(hm, Jm, gm, tm, psi0, torch.complex128)) / (2 * eps)

    for s in range(S):
        def mg(h_, J_, g_, t_, e, s=s):
            g_[s] += e
        def mt(h_, J_, g_, t_, e, s=s):
            t_[s] += e
        assert abs(fd(mg) - tg.grad[s].item()) < 1e-6, ("gamma", s)
        assert abs(fd(mt) - tT.grad[s].item()) < 1e-6, ("t", s)
    for i in [0, n // 2, n - 1]:
        def mh(h_, J_, g_, t_, e, i=i):
            h_[i] += e
        assert abs(fd(mh) - th.grad[i].item()) < 1e-6, ("h", i)
    for (i, j) in [(0, 1), (1, n - 1), (n - 2, n - 1)]:
        def mJ(h_, J_, g_, t_, e, i=i, j=j):
            J_[i, j] += e
        assert abs(fd(mJ) - tJ.grad[i, j].item()) < 1e-6, ("J", i, j)


def test_fp32_adjoint_close_to_fp64(cuda_lib):
    """The FP32 path (fused kernels forward, FP32 adjoint vectors, FP64 reductions)
    agrees with the FP64 gradients to 1e-4 relative."""
    import torch

    from paper_2608_12058_b300 import autograd as AG

    n, S = 15, 6
    a = I.config_anneal(n=n, S=S, seed=9)
    psi0 = I.uniform_state(n)
    grads = {}
    for dt in (torch.complex64, torch.complex128):
        th, tJ, tg, tT = _params(a.h, a.J, a.gammas, a.ts)
        x = torch.from_numpy(psi0).to(dt).cuda().requires_grad_(True)
        L = AG.energy(AG.anneal(x, th, tJ, tg, tT), th, tJ)
        L.backward()
        grads[dt] = (tg.grad.numpy(), tT.grad.numpy(), th.grad.numpy(), tJ.grad.numpy(),
                     x.grad.cpu().numpy().astype(np.complex128))
    for k in range(5):
        g32, g64 = grads[torch.complex64][k], grads[torch.complex128][k]
        assert np.linalg.norm(g32 - g64) <= 1e-4 * np.linalg.norm(g64), k


def test_anneal_workload_n22_gradients(cuda_lib):
    """The differentiable-anneal workload (n=22, 64 segments, complex64 forward, FP64
    reductions): gradients for sampled parameters within 1e-4 of central finite
    differences of the FP64 forward map."""
    import torch

    from paper_2608_12058_b300 import autograd as AG

    a = I.config_anneal()
    n, S = a.n, len(a.gammas)
    psi0 = I.uniform_state(n)
    th, tJ, tg, tT = _params(a.h, a.J, a.gammas, a.ts)
    x = torch.from_numpy(psi0).to(torch.complex64).cuda()
    L = AG.energy(AG.anneal(x, th, tJ, tg, tT), th, tJ)
    L.backward()
    eps = 1e-4

    def fd(which, idx):
        vals = []
        for sgn in (+1, -1):
            h_, J_, g_, t_ = [np.array(v, dtype=np.float64) for v in (a.h, a.J, a.gammas, a.ts)]
            {"gamma": g_, "t": t_, "h": h_, "J": J_}[which][idx] += sgn * eps
            vals.append(_energy_after(h_, J_, g_, t_, psi0, torch.complex128))
        return (vals[0] - vals[1]) / (2 * eps)

    checks = [("gamma", 10, tg.grad[10].item()), ("gamma", 60, tg.grad[60].item()),
              ("t", 31, tT.grad[31].item()), ("h", 3, th.grad[3].item()), ("J", (2, 17), tJ.grad[2, 17].item())]
    scale = max(abs(c[2]) for c in checks)
    for which, idx, got in checks:
        ref = fd(which, idx)
        assert abs(got - ref) <= 1e-4 * max(abs(ref), scale), (which, idx, got, ref)


def test_anneal_workload_n22_gradients_fp64_each_component(cuda_lib):
    """The same workload with the FP64 forward and adjoint: every sampled gradient,
    large or small, within 1e-6 (relative) of its own central finite difference (the
    FP32 test above bounds its components by the FP32 noise floor of the largest one)."""
    import torch

    from paper_2608_12058_b300 import autograd as AG

    a = I.config_anneal()
    n = a.n
    psi0 = I.uniform_state(n)
    th, tJ, tg, tT = _params(a.h, a.J, a.gammas, a.ts)
    x = torch.from_numpy(psi0).to(torch.complex128).cuda()
    L = AG.energy(AG.anneal(x, th, tJ, tg, tT, tol=1e-13), th, tJ)
    L.backward()
    eps = 1e-4

    def fd(which, idx):
        vals = []
        for sgn in (+1, -1):
            h_, J_, g_, t_ = [np.array(v, dtype=np.float64) for v in (a.h, a.J, a.gammas, a.ts)]
            {"gamma": g_, "t": t_, "h": h_, "J": J_}[which][idx] += sgn * eps
            vals.append(_energy_after(h_, J_, g_, t_, psi0, torch.complex128))
        return (vals[0] - vals[1]) / (2 * eps)

    checks = [("gamma", 10, tg.grad[10].item()), ("gamma", 60, tg.grad[60].item()),
              ("t", 31, tT.grad[31].item()), ("t", 63, tT.grad[63].item()), ("h", 3, th.grad[3].item()),
              ("J", (2, 17), tJ.grad[2, 17].item())]
    for which, idx, got in checks:
        ref = fd(which, idx)
        # the absolute term is the finite difference's own rounding: FP64 energies accurate
        # to ~1e-13 relative (|L| ~ 10) over 2 eps
        assert abs(got - ref) <= 1e-6 * abs(ref) + 1e-7, (which, idx, got, ref)


@pytest.mark.parametrize("n,dtype_name,tol", [(12, "complex128", 1e-11), (16, "complex64", 2e-5)])
def test_regenerated_and_stored_forward_vectors_agree(cuda_lib, n, dtype_name, tol):
    """The two ways of providing b_k to the adjoint - all kept, or regenerated upward
    from anchor pairs in a ring of 6 - give the same gradients (regeneration from
    (b_1, b_2) drifts only by round-off over the few steps between anchors)."""
    import torch

    from paper_2608_12058_b300 import api

    dt = getattr(torch, dtype_name)
    a = I.config_anneal(n=n, S=3, seed=4)
    x = torch.from_numpy(I.uniform_state(n)).to(dt).cuda()
    bnd = torch.empty((3, 1 << n), dtype=dt, device="cuda")
    infos = api.anneal(a.h, a.J, a.gammas, a.ts, x, boundaries=bnd)
    # the host-side degree bound that sizes the automatic pool covers the library's K
    tol_ = 1e-12 if dtype_name == "complex128" else 2.0 ** -23
    kb = api._degree_upper_bound(np.asarray(a.h), np.asarray(a.J), np.asarray(a.gammas), np.asarray(a.ts),
                                 tol_, "chebyshev")
    assert max(i["K"] for i in infos) <= kb
    _, g, _, _ = api.energy_grad(a.h, a.J, x)
    outs, psibars = [], []
    for sv in (None, 8, 14):
        gr = g.clone()
        outs.append(api.anneal_adjoint(a.h, a.J, a.gammas, a.ts, bnd, x, gr, store_vectors=sv))
        psibars.append(gr.cpu().numpy().astype(np.complex128))
    for o, pb in zip(outs[1:], psibars[1:]):
        for key in ("gamma", "t", "h", "J"):
            ref = outs[0][key]
            assert np.linalg.norm(o[key] - ref) <= tol * np.linalg.norm(ref), key
        assert np.linalg.norm(pb - psibars[0]) <= tol * np.linalg.norm(psibars[0])


def test_adjoint_special_segments_vs_finite_differences(cuda_lib):
    """Segments the general formulas do not cover: gamma_s = 0 (dL/dgamma from explicit
    flip sums), a negative gamma_s, and a segment of duration 0 (degree K = 0)."""
    import torch

    from paper_2608_12058_b300 import autograd as AG

    n = 7
    h, J = I.sk_instance(n, 88)
    gammas = np.array([1.1, 0.0, -0.6, 0.8])
    ts = np.array([0.7, 0.5, 0.4, 0.0])
    psi0 = I.random_state(n, 89)
    th, tJ, tg, tT = _params(h, J, gammas, ts)
    x = torch.from_numpy(psi0).cuda().requires_grad_(True)
    L = AG.energy(AG.anneal(x, th, tJ, tg, tT, tol=1e-13), th, tJ)
    L.backward()
    eps = 1e-6

    def loss(g_, t_):
        return _energy_after(h, J, g_, t_, psi0, torch.complex128)

    for s in range(len(gammas)):
        gp, gm = gammas.copy(), gammas.copy()
        gp[s] += eps
        gm[s] -= eps
        assert abs((loss(gp, ts) - loss(gm, ts)) / (2 * eps) - tg.grad[s].item()) < 1e-7, ("gamma", s)
    for s in range(len(ts) - 1):  # a negative duration is not a valid input
        tp, tm = ts.copy(), ts.copy()
        tp[s] += eps
        tm[s] -= eps
        assert abs((loss(gammas, tp) - loss(gammas, tm)) / (2 * eps) - tT.grad[s].item()) < 1e-7, ("t", s)
    # the zero-length segment: one-sided second-order difference at t = 0
    e1 = 1e-5
    t1, t2 = ts.copy(), ts.copy()
    t1[-1] += e1
    t2[-1] += 2 * e1
    fd = (-3 * loss(gammas, ts) + 4 * loss(gammas, t1) - loss(gammas, t2)) / (2 * e1)
    assert abs(fd - tT.grad[-1].item()) < 1e-6, "t at 0"


def _general_energy(h, J, a_s, b_s, ts, psi0):
    import torch

    from paper_2608_12058_b300 import api

    x = torch.from_numpy(psi0).cuda()
    api.anneal_general(h, J, a_s, b_s, ts, x, tol=1e-13, info=False)
    return api.energy(h, J, x)[0]


def test_general_segments_gradients_vs_finite_differences(cuda_lib):
    """Segments b_s H_P + a_s sum_j X_j (b_s = 0, a_s = 0 and negative values included):
    dL/da_s, dL/db_s, dL/dt_s, dL/dh, dL/dJ against central differences (FP64)."""
    import torch

    from paper_2608_12058_b300 import autograd as AG

    n = 6
    h, J = I.sk_instance(n, 93)
    a_s = np.array([1.1, 0.0, -0.6, 0.8])
    b_s = np.array([0.5, 1.2, -0.8, 0.0])
    ts = np.array([0.6, 0.5, 0.4, 0.7])
    psi0 = I.random_state(n, 94)
    t = lambda v: torch.tensor(np.asarray(v, dtype=np.float64), requires_grad=True)
    th, tJ, ta, tb, tt = t(h), t(J), t(a_s), t(b_s), t(ts)
    x = torch.from_numpy(psi0).cuda()
    L = AG.energy(AG.anneal_general(x, th, tJ, ta, tb, tt, tol=1e-13), th, tJ)
    L.backward()
    eps = 1e-6
    base = {"h": h, "J": J, "a": a_s, "b": b_s, "t": ts}
    grads = {"h": th.grad.numpy(), "J": tJ.grad.numpy(), "a": ta.grad.numpy(), "b": tb.grad.numpy(),
             "t": tt.grad.numpy()}
    picks = [("a", 0), ("a", 1), ("a", 2), ("a", 3), ("b", 0), ("b", 1), ("b", 2), ("b", 3),
             ("t", 0), ("t", 1), ("t", 2), ("t", 3), ("h", 2), ("J", (1, 4))]
    for key, idx in picks:
        vals = []
        for sgn in (1, -1):
            v = {k: np.array(val, dtype=np.float64) for k, val in base.items()}
            v[key][idx] += sgn * eps
            vals.append(_general_energy(v["h"], v["J"], v["a"], v["b"], v["t"], psi0))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - grads[key][idx]) < 1e-7, (key, idx, fd, grads[key][idx])


def test_magnus4_schedule_parameter_gradients(cuda_lib):
    """Gradients of the energy after Magnus propagation with respect to the parameters
    of a smooth schedule A(t) = p0 (1 - t/T) + p2 sin t, B(t) = p1 t/T (torch composes
    the node values from p; cheb_magnus4_adjoint chains the Gauss-node weights and
    supplies the segment adjoint)."""
    import torch

    from paper_2608_12058_b300 import api
    from paper_2608_12058_b300 import autograd as AG

    n, T, steps = 6, 2.0, 5
    h, J = I.sk_instance(n, 95)
    psi0 = I.random_state(n, 96)
    p = torch.tensor([1.4, 0.9, 0.3], dtype=torch.float64, requires_grad=True)

    def nodes_of(pv):
        dt = T / steps
        m = torch.arange(steps, dtype=torch.float64)
        t1 = m * dt + (0.5 - 3 ** 0.5 / 6) * dt
        t2 = m * dt + (0.5 + 3 ** 0.5 / 6) * dt
        A = lambda tt: pv[0] * (1 - tt / T) + pv[2] * torch.sin(tt)
        B = lambda tt: pv[1] * tt / T
        return torch.full((steps,), dt, dtype=torch.float64), torch.stack([A(t1), B(t1), A(t2), B(t2)], dim=1)

    dt, nodes = nodes_of(p)
    th, tJ = torch.tensor(h), torch.tensor(J)
    L = AG.energy(AG.magnus4(torch.from_numpy(psi0).cuda(), th, tJ, dt, nodes, tol=1e-13), th, tJ)
    L.backward()

    def loss(pv):
        d, nd = nodes_of(torch.tensor(pv, dtype=torch.float64))
        x = torch.from_numpy(psi0).cuda()
        api.magnus4(h, J, d.numpy(), nd.numpy(), x, tol=1e-13)
        return api.energy(h, J, x)[0]

    eps = 1e-6
    for i in range(3):
        pp, pm = p.detach().numpy().copy(), p.detach().numpy().copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (loss(pp) - loss(pm)) / (2 * eps)
        assert abs(fd - p.grad[i].item()) < 1e-7, (i, fd, p.grad[i].item())


@pytest.mark.parametrize("n,dtype_name,S,sv", [(16, "complex64", 3, 8), (16, "complex64", 1, None),
                                               (12, "complex128", 2, 8), (9, "complex64", 2, None)])
def test_checkpointed_forward_skips_recomputation(cuda_lib, n, dtype_name, S, sv):
    """cheb_anneal_checkpointed gives the forward result of cheb_anneal, and the adjoint
    that uses its checkpoint returns bit for bit what the adjoint returns when it
    recomputes the last segment itself from the same boundaries and psi_T (the pool
    holds the same vectors either way: all b_k (sv = None), or the ring and anchors)."""
    import torch

    from paper_2608_12058_b300 import api

    dt = getattr(torch, dtype_name)
    a = I.config_anneal(n=n, S=S, seed=7)
    x0 = torch.from_numpy(I.uniform_state(n)).to(dt).cuda()
    tol = 1e-12 if dtype_name == "complex128" else 2.0 ** -23
    y_ref = x0.clone()
    b_ref = torch.empty((S, 1 << n), dtype=dt, device="cuda")
    api.anneal(a.h, a.J, a.gammas, a.ts, y_ref, boundaries=b_ref)
    y = x0.clone()
    bnd = torch.empty((S, 1 << n), dtype=dt, device="cuda")
    ck = api.anneal_checkpointed(a.h, a.J, a.gammas, a.ts, y, bnd, store_vectors=sv)
    # segments before the last run on the same path as cheb_anneal
    assert torch.equal(bnd, b_ref)
    rel = (torch.linalg.vector_norm(y - y_ref) / torch.linalg.vector_norm(y_ref)).item()
    assert rel <= (1e-12 if dtype_name == "complex128" else 2e-6), rel
    _, g, _, _ = api.energy_grad(a.h, a.J, y)
    g_ck, g_re = g.clone(), g.clone()
    o_ck = api.anneal_adjoint(a.h, a.J, a.gammas, a.ts, bnd, y, g_ck, checkpoint=ck)
    o_re = api.anneal_adjoint(a.h, a.J, a.gammas, a.ts, bnd, y, g_re, store_vectors=ck.store_vectors)
    assert torch.equal(g_ck, g_re)
    for key in ("gamma", "t", "h", "J"):
        assert np.array_equal(o_ck[key], o_re[key]), key
    # the checkpoint is consumed: a second adjoint call on its workspace recomputes
    g_again = g.clone()
    o_again = api.anneal_adjoint(a.h, a.J, a.gammas, a.ts, bnd, y, g_again, checkpoint=ck)
    assert torch.equal(g_again, g_re)
    assert np.array_equal(o_again["gamma"], o_re["gamma"])


def test_checkpoint_with_other_arguments_is_not_used(cuda_lib):
    """A checkpoint taken for one tolerance does not serve an adjoint call with another:
    the adjoint recomputes, and its gradients equal those of a fresh workspace."""
    import torch

    from paper_2608_12058_b300 import api

    n, S = 14, 2
    a = I.config_anneal(n=n, S=S, seed=9)
    y = torch.from_numpy(I.uniform_state(n)).to(torch.complex64).cuda()
    bnd = torch.empty((S, 1 << n), dtype=torch.complex64, device="cuda")
    ck = api.anneal_checkpointed(a.h, a.J, a.gammas, a.ts, y, bnd, tol=1e-6, store_vectors=8)
    _, g, _, _ = api.energy_grad(a.h, a.J, y)
    g1, g2 = g.clone(), g.clone()
    o1 = api.anneal_adjoint(a.h, a.J, a.gammas, a.ts, bnd, y, g1, tol=2.0 ** -23, checkpoint=ck)
    o2 = api.anneal_adjoint(a.h, a.J, a.gammas, a.ts, bnd, y, g2, tol=2.0 ** -23, store_vectors=8)
    assert torch.equal(g1, g2)
    assert np.array_equal(o1["h"], o2["h"])


def test_general_checkpointed_forward_skips_recomputation(cuda_lib):
    """The same for cheb_anneal_general_checkpointed (segments b_s H_P + a_s sum_j X_j)."""
    import torch

    from paper_2608_12058_b300 import api

    n, S = 15, 3
    a = I.config_anneal(n=n, S=S, seed=11)
    b_s = np.array([0.5, -0.8, 1.2])
    y = torch.from_numpy(I.uniform_state(n)).to(torch.complex64).cuda()
    bnd = torch.empty((S, 1 << n), dtype=torch.complex64, device="cuda")
    ck = api.anneal_general_checkpointed(a.h, a.J, a.gammas, b_s, a.ts, y, bnd, store_vectors=8)
    y_ref = torch.from_numpy(I.uniform_state(n)).to(torch.complex64).cuda()
    api.anneal_general(a.h, a.J, a.gammas, b_s, a.ts, y_ref)
    assert (torch.linalg.vector_norm(y - y_ref) / torch.linalg.vector_norm(y_ref)).item() <= 2e-6
    _, g, _, _ = api.energy_grad(a.h, a.J, y)
    g1, g2 = g.clone(), g.clone()
    o1 = api.anneal_general_adjoint(a.h, a.J, a.gammas, b_s, a.ts, bnd, y, g1, checkpoint=ck)
    o2 = api.anneal_general_adjoint(a.h, a.J, a.gammas, b_s, a.ts, bnd, y, g2, store_vectors=8)
    assert torch.equal(g1, g2)
    for key in ("a", "b", "t", "h", "J"):
        assert np.array_equal(o1[key], o2[key]), key
