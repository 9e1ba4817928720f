"""Small profiling driver: a few fused Clenshaw steps on one seeded SK instance.

    python -m paper_2608_12058_b300.prof_case N L H [STEPS]

Runs cheb_poly_apply (Algorithm 2 with random coefficients) on the FP32 fused path
with the bit split (L, H) at n = N, for use under ncu (kernel names k_low and
k_strided). Prints the final norm so the run is checked for finiteness.
"""
import sys

import numpy as np


def main(argv):
    import torch

    from . import api
    from . import inputs as I

    n, l, h = int(argv[0]), int(argv[1]), int(argv[2])
    steps = int(argv[3]) if len(argv) > 3 else 6
    c = I.config_family(n, 1.0, 1.0, 0, "uniform")
    x = torch.full((1 << n,), 2 ** (-n / 2), dtype=torch.complex64, device="cuda")
    api.set_fused_split(n, l, h)
    rng = np.random.default_rng(0)
    coef = (rng.standard_normal(steps + 1) + 1j * rng.standard_normal(steps + 1)) / (4 * steps)
    api.poly_apply(c.h, c.J, 1.0, 0.0, 80.0, coef, x, path="fused")
    torch.cuda.synchronize()
    nrm = float(torch.linalg.vector_norm(x))
    assert np.isfinite(nrm)
    print("ok", nrm)


if __name__ == "__main__":
    main(sys.argv[1:])
