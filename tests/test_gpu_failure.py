"""Failure detection without a GPU fault: a bounded device wait that runs out (on a
barrier that nothing arrives on) is reported as CHEB_ERR_TIMEOUT, and the context
keeps working afterwards."""
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
