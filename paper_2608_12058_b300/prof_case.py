"""Small profiling driver for the library's kernels on seeded SK instances.

    python -m paper_2608_12058_b300.prof_case N L H [STEPS]
        STEPS fused Clenshaw steps (cheb_poly_apply with random coefficients) at n = N
        with the bit split (L, H) (kernel names k_low and k_strided*).
    python -m paper_2608_12058_b300.prof_case tail N L H [STEPS]
        the same with the L2-blocked step tail on (kernel names k_strided* for the
        earlier strided passes, k_mixed for the last strided pass + low pass).
    python -m paper_2608_12058_b300.prof_case pair N L H [STEPS]
        the same with the L2-blocked strided pair (kernel names k_pair and k_low).
    python -m paper_2608_12058_b300.prof_case compare N [STEPS [L H]]
        times STEPS fused steps at n = N (default split, or (L, H)) with the separate
        launches, the L2-blocked step tail and the L2-blocked strided pair, twice each
        (CUDA events around the call; then a run with the library's per-kind event
        timing), and prints ms per step and per launch.
    python -m paper_2608_12058_b300.prof_case ffcompare N [STEPS [L H]]
        float-float (FP64 path) step time at n = N with separate launches and with the
        L2-blocked strided pair.
    python -m paper_2608_12058_b300.prof_case ff N L H [STEPS]
        STEPS float-float fused steps of the FP64 path (complex128 states) at n = N with
        the split (L, H) (kernel names k_low_ff and k_strided_ff).
    python -m paper_2608_12058_b300.prof_case batch [MODE]
        the 512-instance batch workload by size group and whole, in the batch launch
        mode MODE (1 persistent, the default; 2 persistent with two CTAs per SM; 0
        per-size launches).
    python -m paper_2608_12058_b300.prof_case anneal
        the n=22 64-segment anneal forward with and without programmatic dependent launch,
        and replayed from a CUDA graph.
    python -m paper_2608_12058_b300.prof_case l2
        copy bandwidth of L2-resident buffers (8..96 MB).
    python -m paper_2608_12058_b300.prof_case adjoint N S
        the first S segments of the anneal schedule at n = N (complex64): forward with
        segment-start states, energy gradient, full reverse pass (k_adj_acc_f32x2,
        k_dt, k_fold and the step kernels of both recurrences).
    python -m paper_2608_12058_b300.prof_case cluster N COUNT
        a batch of COUNT instances of size N (complex64) run whole on thread-block
        clusters (k_cluster_run).

Each mode prints a finite summary so the run is checked.
"""
import sys

import numpy as np


def fused_steps(n, l, h, steps, blocking=0):
    import torch

    from . import api
    from . import inputs as I

    c = I.config_family(n, 1.0, 1.0, 0, "uniform")
    x = torch.full((1 << n,), 2 ** (-n / 2), dtype=torch.complex64, device="cuda")
    api.set_fused_split(n, l, h)
    api.set_fused_blocking(blocking)
    rng = np.random.default_rng(0)
    coef = (rng.standard_normal(steps + 1) + 1j * rng.standard_normal(steps + 1)) / (4 * steps)
    api.poly_apply(c.h, c.J, 1.0, 0.0, 80.0, coef, x, path="fused")
    api.check_status(n, "fp32")
    nrm = float(torch.linalg.vector_norm(x))
    assert np.isfinite(nrm)
    print("ok", nrm)


def ff_steps(n, l, h, steps):
    """STEPS float-float fused steps of the FP64 path at n with the split (l, h)."""
    import torch

    from . import api
    from . import inputs as I

    c = I.config_family(n, 1.0, 1.0, 0, "uniform")
    x = torch.full((1 << n,), 2 ** (-n / 2), dtype=torch.complex128, device="cuda")
    api.set_fused_split_fp64(n, l, h)
    rng = np.random.default_rng(0)
    coef = (rng.standard_normal(steps + 1) + 1j * rng.standard_normal(steps + 1)) / (4 * steps)
    try:
        api.poly_apply(c.h, c.J, 1.0, 0.0, 80.0, coef, x, path="fused")
        torch.cuda.synchronize()
    finally:
        api.set_fused_split_fp64(n, -1)
    nrm = float(torch.linalg.vector_norm(x))
    assert np.isfinite(nrm)
    print("ok", nrm)


def compare(n, steps, split=None):
    """Step time of the fused FP32 step at n with separate launches (mode 0), the
    L2-blocked tail (1) and the L2-blocked strided pair (2): CUDA events without
    profiling, then a profiled run for the per-kernel split."""
    import torch

    from . import api
    from . import inputs as I

    if split is not None:
        api.set_fused_split(n, split[0], split[1])
    c = I.config_family(n, 1.0, 1.0, 0, "uniform")
    x = torch.full((1 << n,), 2 ** (-n / 2), dtype=torch.complex64, device="cuda")
    rng = np.random.default_rng(0)
    coef = (rng.standard_normal(steps + 1) + 1j * rng.standard_normal(steps + 1)) / (4 * steps)
    print("n", n, "split", api.get_fused_split(n), "steps", steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    try:
        for _ in range(2):
            for mode in (0, 1, 2):
                api.set_fused_blocking(mode)
                api.poly_apply(c.h, c.J, 1.0, 0.0, 80.0, coef[:4], x, path="fused")  # warm-up
                torch.cuda.synchronize()
                e0.record()
                api.poly_apply(c.h, c.J, 1.0, 0.0, 80.0, coef, x, path="fused")
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                api.check_status(n, "fp32")
                assert np.isfinite(float(torch.linalg.vector_norm(x)))
                api.profile_reset()
                api.profile_enable(True)
                api.poly_apply(c.h, c.J, 1.0, 0.0, 80.0, coef, x, path="fused")
                torch.cuda.synchronize()
                api.profile_enable(False)
                parts = []
                for kind in ("low", "high", "tail", "pair"):
                    cnt, tot = api.profile_read(kind)
                    if cnt:
                        parts.append(f"{kind} {cnt} x {tot / cnt * 1e3:.1f} us")
                print(f"  blocking {mode}: {ms / steps:.3f} ms/step, "
                      f"{(1 << n) * steps / ms * 1e3:.3e} amplitude-updates/s; profiled: " + ", ".join(parts))
    finally:
        api.set_fused_blocking(None)
        if split is not None:
            api.set_fused_split(n, -1)


def ff_compare(n, steps, split=None):
    """Step time of the float-float fused step (FP64 path) at n with separate launches
    (mode 0) and the L2-blocked strided pair (2), CUDA events, twice each."""
    import torch

    from . import api
    from . import inputs as I

    if split is not None:
        api.set_fused_split_fp64(n, split[0], split[1])
    c = I.config_family(n, 1.0, 1.0, 0, "uniform")
    x = torch.full((1 << n,), 2 ** (-n / 2), dtype=torch.complex128, device="cuda")
    rng = np.random.default_rng(0)
    coef = (rng.standard_normal(steps + 1) + 1j * rng.standard_normal(steps + 1)) / (4 * steps)
    print("n", n, "fp64 split", api.get_fused_split_fp64(n), "steps", steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    try:
        for _ in range(2):
            for mode in (0, 2):
                api.set_fused_blocking(mode)
                api.poly_apply(c.h, c.J, 1.0, 0.0, 80.0, coef[:4], x, path="fused")  # warm-up
                torch.cuda.synchronize()
                e0.record()
                api.poly_apply(c.h, c.J, 1.0, 0.0, 80.0, coef, x, path="fused")
                e1.record()
                torch.cuda.synchronize()
                api.check_status(n, "fp64")
                ms = e0.elapsed_time(e1)
                print(f"  blocking {mode}: {ms / steps:.3f} ms/step, {(1 << n) * steps / ms * 1e3:.3e} "
                      "amplitude-updates/s")
    finally:
        api.set_fused_blocking(None)
        if split is not None:
            api.set_fused_split_fp64(n, -1)


def adjoint(n, S):
    import torch

    from . import api
    from . import inputs as I

    a = I.config_anneal(n=n, S=64)
    g_s, t_s = a.gammas[:S], a.ts[:S]
    x = torch.full((1 << n,), 2 ** (-n / 2), dtype=torch.complex64, device="cuda")
    bnd = torch.empty((S, 1 << n), dtype=torch.complex64, device="cuda")
    api.anneal(a.h, a.J, g_s, t_s, x, boundaries=bnd, info=False)
    _, g, _, _ = api.energy_grad(a.h, a.J, x)
    out = api.anneal_adjoint(a.h, a.J, g_s, t_s, bnd, x, g)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out["gamma"]))
    print("ok", out["gamma"])


def cluster(n, count):
    import torch

    from . import api
    from . import inputs as I

    ns = [n] * count
    hs, Js = [], []
    for i in range(count):
        h, J = I.sk_instance(n, 700 + i)
        hs.append(h)
        Js.append(J)
    gam = np.linspace(0.5, 1.5, count)
    ts = np.full(count, 10.0)
    offs, total = api.batch_offsets(ns)
    x = torch.full((total,), 2 ** (-n / 2), dtype=torch.complex64, device="cuda")
    mode = api.get_batch_persistent()
    api.set_batch_persistent(0)  # per-size launches: n = 14..17 on thread-block clusters
    try:
        infos = api.expmv_batched(ns, hs, Js, gam, ts, x, tol=1e-6)
    finally:
        api.set_batch_persistent(mode)
    torch.cuda.synchronize()
    assert all(abs(i["norm"] - 1.0) < 1e-4 for i in infos)
    print("ok", sum(i["K"] for i in infos))


def batch(mode):
    """The 512-instance workload by size group (n <= 13, 14-17, 18, 19, 20) and whole, with
    the batch launch mode MODE (cheb_set_batch_persistent); one timed run after a warm-up."""
    import torch

    from . import api
    from . import inputs as I

    api.set_batch_persistent(mode)
    b = I.config_batch()
    ns = np.asarray(b.ns)
    groups = [("all", np.ones_like(ns, dtype=bool)), ("n<=13", ns <= 13), ("14-17", (ns >= 14) & (ns <= 17)),
              ("18", ns == 18), ("19", ns == 19), ("20", ns == 20)]
    try:
        for name, m in groups:
            idx = np.nonzero(m)[0]
            sub = [int(b.ns[i]) for i in idx]
            offs, total = api.batch_offsets(sub)
            cat = np.zeros(total, dtype=np.complex64)
            for nn, o in zip(sub, offs):
                cat[o:o + (1 << nn)] = 2.0 ** (-nn / 2)
            x0 = torch.from_numpy(cat).cuda()
            args = ([b.hs[i] for i in idx], [b.Js[i] for i in idx], [b.gammas[i] for i in idx],
                    [b.ts[i] for i in idx])
            x = x0.clone()
            infos = api.expmv_batched(sub, *args, x, tol=1e-6)
            work = float(sum((1 << nn) * i["K"] * i["time_splits"] for nn, i in zip(sub, infos)))
            x.copy_(x0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            api.expmv_batched(sub, *args, x, tol=1e-6, info=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            assert np.isfinite(float(torch.linalg.vector_norm(x)))
            print(f"{name:6s} {len(idx):4d} instances {ms:9.2f} ms {work / ms * 1e3:.3e} amplitude-updates/s")
            del x, x0
            api.release_workspaces()
            torch.cuda.empty_cache()
    finally:
        api.set_batch_persistent(1)


def anneal_time(reps=3):
    """The n=22, 64-segment anneal forward (complex64) timed with and without programmatic
    dependent launch of the step kernels, `reps` times each after a warm-up (CUDA events)."""
    import torch

    from . import api
    from . import inputs as I

    a = I.config_anneal()
    n = a.n
    x0 = torch.full((1 << n,), 2 ** (-n / 2), dtype=torch.complex64, device="cuda")
    infos = api.anneal(a.h, a.J, a.gammas, a.ts, x0.clone())
    K = sum(i["K"] for i in infos)
    try:
        for on in (True, False, True, False):
            api.set_programmatic_launch(on)
            ts = []
            for _ in range(reps):
                x = x0.clone()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                api.anneal(a.h, a.J, a.gammas, a.ts, x, info=False)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = min(ts)
            print(f"programmatic launch {'on ' if on else 'off'}: {ms:.2f} ms, {(1 << n) * K / ms * 1e3:.3e} "
                  f"amplitude-updates/s ({K} steps, {ms / K * 1e3:.1f} us per step)")
        # the same schedule captured into a CUDA graph and replayed
        api.set_programmatic_launch(True)
        x = x0.clone()
        g = api.AnnealGraph(a.h, a.J, a.gammas, a.ts, x)
        ts = []
        for _ in range(reps):
            x.copy_(x0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            g.launch()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        g.status()
        g.close()
        ms = min(ts)
        print(f"graph replay (programmatic launch on): {ms:.2f} ms, {(1 << n) * K / ms * 1e3:.3e} "
              f"amplitude-updates/s ({ms / K * 1e3:.1f} us per step)")
    finally:
        api.set_programmatic_launch(True)


def l2_copy():
    """Copy bandwidth of L2-resident buffers (torch copy_ of 8..96 MB, 200 repetitions,
    CUDA events): the roofline for the batch and anneal workloads, whose vectors stay in
    the 126 MB L2."""
    import torch

    for mb in (8, 16, 32, 48, 64, 96):
        n = mb * (1 << 20) // 4
        x = torch.ones(n, dtype=torch.float32, device="cuda")
        y = torch.empty_like(x)
        for _ in range(10):
            y.copy_(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(200):
            y.copy_(x)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(f"{mb:3d} MB: {2 * x.numel() * 4 * 200 / (ms / 1e3) / 1e9:8.1f} GB/s (read + write)")
        del x, y


def main(argv):
    if argv[0] == "adjoint":
        adjoint(int(argv[1]), int(argv[2]))
    elif argv[0] == "cluster":
        cluster(int(argv[1]), int(argv[2]))
    elif argv[0] == "compare":
        split = (int(argv[3]), int(argv[4])) if len(argv) > 4 else None
        compare(int(argv[1]), int(argv[2]) if len(argv) > 2 else 40, split)
    elif argv[0] == "ffcompare":
        split = (int(argv[3]), int(argv[4])) if len(argv) > 4 else None
        ff_compare(int(argv[1]), int(argv[2]) if len(argv) > 2 else 10, split)
    elif argv[0] == "anneal":
        anneal_time()
    elif argv[0] == "l2":
        l2_copy()
    elif argv[0] == "batch":
        batch(int(argv[1]) if len(argv) > 1 else 1)
    elif argv[0] == "ff":
        n, l, h = int(argv[1]), int(argv[2]), int(argv[3])
        ff_steps(n, l, h, int(argv[4]) if len(argv) > 4 else 6)
    elif argv[0] == "tail":
        n, l, h = int(argv[1]), int(argv[2]), int(argv[3])
        fused_steps(n, l, h, int(argv[4]) if len(argv) > 4 else 6, blocking=1)
    elif argv[0] == "pair":
        n, l, h = int(argv[1]), int(argv[2]), int(argv[3])
        fused_steps(n, l, h, int(argv[4]) if len(argv) > 4 else 6, blocking=2)
    else:
        n, l, h = int(argv[0]), int(argv[1]), int(argv[2])
        fused_steps(n, l, h, int(argv[3]) if len(argv) > 3 else 6)


if __name__ == "__main__":
    main(sys.argv[1:])
