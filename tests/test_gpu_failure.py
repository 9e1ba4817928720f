"""Failure detection without a GPU fault: the bounded device waits that run out (an
mbarrier that nothing arrives on; a team barrier of the persistent batch kernel whose
teammate never comes) are reported as CHEB_ERR_TIMEOUT, and the context keeps working
afterwards (the fused path and the persistent batch launch)."""
import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(cuda_lib, oracle):
    import torch

    from paper_2608_12058_b300 import api
    from paper_2608_12058_b300._lib import ChebError

    with pytest.raises(ChebError) as e:
        api.wait_selftest()
    assert e.value.code == 4  # CHEB_ERR_TIMEOUT
    # the same context still runs the fused path correctly
    n = 16
    h, J = I.sk_instance(n, 31)
    psi = I.random_state(n, 32)
    ref, _ = oracle.expmv(h, J, 0.7, 2.0, psi, 2.0 ** -23)
    x = torch.from_numpy(psi).to(torch.complex64).cuda()
    api.expmv(h, J, 0.7, 2.0, x, tol=2.0 ** -23, path="fused")
    y = x.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-5
    # and the persistent batch launch (team barriers) after it
    ns = [12, 16, 18]
    hs, Js = zip(*[I.sk_instance(m, 60 + m) for m in ns])
    states = [I.random_state(m, 70 + m) for m in ns]
    offs, total = api.batch_offsets(ns)
    cat = np.zeros(total, dtype=np.complex64)
    for o, st in zip(offs, states):
        cat[o:o + st.shape[0]] = st
    xb = torch.from_numpy(cat).cuda()
    api.expmv_batched(ns, list(hs), list(Js), np.full(3, 0.8), np.full(3, 1.5), xb, tol=2.0 ** -23)
    yb = xb.cpu().numpy().astype(np.complex128)
    for i, m in enumerate(ns):
        r, _ = oracle.expmv(hs[i], Js[i], 0.8, 1.5, states[i], 2.0 ** -23)
        got = yb[offs[i]:offs[i] + (1 << m)]
        assert np.linalg.norm(got - r) / np.linalg.norm(r) <= 1e-5, m
