"""The autotuner (cheb_autotune): it times the candidate configurations of the Clenshaw
step on the device, installs the fastest one for AUTO, records it in the cache file named
by CHEB_AUTOTUNE_CACHE, and the tuned configuration stays correct against the oracle."""
import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,prec", [(20, "fp32"), (24, "fp32"), (22, "fp64")])
def test_autotune_installs_a_valid_choice(cuda_lib, oracle, n, prec, tmp_path, monkeypatch):
    import torch

    from paper_2608_12058_b300 import api

    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("CHEB_AUTOTUNE_CACHE", str(cache))
    try:
        r = api.autotune(n, prec, steps=4)
        print(f"n={n} {prec}: {r}")
        assert r["candidates"] >= 2 and r["path"] in ("plain", "fused")
        # the default is one of the candidates, so the best is not slower beyond timing noise
        assert r["best_ms_per_step"] <= 1.10 * r["default_ms_per_step"]
        if r["path"] == "fused":
            split = api.get_fused_split(n) if prec == "fp32" else api.get_fused_split_fp64(n)
            assert split == (r["l"], r["h"])
        line = cache.read_text().strip().splitlines()[-1].split()
        assert line[0] == "cheb-tune-1" and int(line[2]) == (0 if prec == "fp32" else 1) and int(line[3]) == n
        h, J = I.sk_instance(n, 77 + n)
        psi = I.random_state(n, 78 + n)
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
        ref, oinfo = oracle.expmv(h, J, 0.8, 0.3, psi, tol)
        x = torch.from_numpy(psi).to(torch.complex64 if prec == "fp32" else torch.complex128).cuda()
        info = api.expmv(h, J, 0.8, 0.3, x, tol=tol)
        y = x.cpu().numpy().astype(np.complex128)
        assert info["K"] == oinfo["K"]
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= (1e-5 if prec == "fp32" else 1e-12)
    finally:
        api.autotune_reset()
