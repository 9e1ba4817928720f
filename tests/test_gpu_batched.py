"""cheb_expmv_batched against the oracle run instance by instance."""
import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _batch(ns, seed):
    rng = np.random.default_rng(seed)
    hs, Js, gs, ts = [], [], [], []
    for i, n in enumerate(ns):
        h, J = I.sk_instance(n, seed * 100 + i)
        hs.append(h)
        Js.append(J)
        gs.append(float(rng.uniform(0.2, 2.0)))
        ts.append(float(rng.uniform(0.5, 4.0)))
    return hs, Js, np.array(gs), np.array(ts)


@pytest.mark.parametrize("prec,persistent", [("fp64", 0), ("fp32", 1), ("fp32", 2), ("fp32", 0)])
def test_mixed_batch_matches_oracle(cuda_lib, oracle, prec, persistent):
    import torch

    from paper_2608_12058_b300 import api

    # sizes of every path. Persistent launch (FP32, one or two CTAs per SM): one CTA per
    # instance up to n = 12, teams of 1..64 CTAs above (n = 13..15 without a strided
    # pass, n >= 16 with one).
    # Per-size launches: one CTA per instance (n <= 13 FP32, <= 12 FP64), one
    # thread-block cluster per instance (n = 14..17 FP32, 13..16 FP64; repeated sizes
    # share a launch), step kernels on the stream pool (larger)
    ns = [1, 3, 8, 12, 13, 14, 16, 9, 15, 12, 17, 14, 17, 18, 19, 20, 18]
    api.set_batch_persistent(persistent)
    hs, Js, gs, ts = _batch(ns, 3)
    offs, total = api.batch_offsets(ns)
    tol = 1e-12 if prec == "fp64" else 2.0 ** -23
    states = [I.random_state(n, 50 + i) for i, n in enumerate(ns)]
    cat = np.zeros(total, dtype=np.complex128)
    for o, s in zip(offs, states):
        cat[o:o + s.shape[0]] = s
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    x = torch.from_numpy(cat).to(dt).cuda()
    try:
        infos = api.expmv_batched(ns, hs, Js, gs, ts, x, tol=tol)
    finally:
        api.set_batch_persistent(1)
    y = x.cpu().numpy().astype(np.complex128)
    for i, n in enumerate(ns):
        ref, oinfo = oracle.expmv(hs[i], Js[i], gs[i], ts[i], states[i], tol)
        got = y[offs[i]:offs[i] + (1 << n)]
        assert infos[i]["K"] == oinfo["K"], i
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL[prec], (i, n)


def test_full_512_instance_batch_sampled(cuda_lib, oracle):
    """The 512-instance workload (n ~ U{12..20}, gamma ~ U(0.2,2), t ~ U(0.5,20),
    complex64, tol 1e-6) in one call; sampled instances checked against the oracle
    one by one, all norms checked."""
    import torch

    from paper_2608_12058_b300 import api

    b = I.config_batch()
    offs, total = api.batch_offsets(b.ns)
    cat = np.zeros(total, dtype=np.complex64)
    for n, o in zip(b.ns, offs):
        cat[o:o + (1 << n)] = 2.0 ** (-n / 2)
    x = torch.from_numpy(cat).cuda()
    infos = api.expmv_batched(b.ns, b.hs, b.Js, b.gammas, b.ts, x, tol=1e-6)
    assert all(abs(i["norm"] - 1.0) < 2e-5 for i in infos)
    y = x.cpu().numpy().astype(np.complex128)
    ns = np.array(b.ns)
    Ks = np.array([i["K"] for i in infos])
    order = np.argsort(ns * 100 + np.arange(len(ns)) % 100)
    # the three smallest, one n = 16, one each of n = 18 and 19, and the largest n = 20
    # instance (the highest degree, a team of 32 CTAs)
    picks = list(order[:3]) + [int(np.argmax(ns == 16)), int(np.argmax(ns == 18)), int(np.argmax(ns == 19)),
                               int(np.argmax(np.where(ns == 20, Ks, -1)))]
    for i in picks:
        n = b.ns[i]
        ref, oinfo = oracle.expmv(b.hs[i], b.Js[i], b.gammas[i], b.ts[i], I.uniform_state(n), 1e-6)
        got = y[offs[i]:offs[i] + (1 << n)]
        assert infos[i]["K"] == oinfo["K"]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5, (i, n)
