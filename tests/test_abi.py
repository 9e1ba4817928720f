"""The C-ABI library builds, loads and exports every declared symbol; its host-only
entry points (coefficient generator, workspace query, argument checks) work
without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2608_12058_b300 import _lib, api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(cheb_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    declared = _declared_functions()
    assert len(declared) >= 8
    for name in declared:
        assert hasattr(L, name), name
    # the binding describes each of them
    for name in declared:
        assert name in _lib.SIGNATURES, name


def test_status_strings_and_version():
    L = _lib.lib()
    for code in range(7):
        assert L.cheb_status_string(code)
    assert b"sm_103a" in L.cheb_version()


def test_workspace_bytes():
    L = _lib.lib()
    assert L.cheb_workspace_bytes(0, 0) == 0
    assert L.cheb_workspace_bytes(34, 0) == 0
    assert L.cheb_workspace_bytes(10, 2) == 0
    w24 = L.cheb_workspace_bytes(24, 0)
    assert w24 >= 2 * (1 << 24) * 8
    assert L.cheb_workspace_bytes(24, 1) >= 2 * (1 << 24) * 16
    # two Clenshaw vectors plus small tables: the state is the caller's (Sec. II.D's
    # in-place b2 += H b1 leaves psi, b1, b2 as the only vectors)
    assert w24 < 2 * (1 << 24) * 8 * 1.05
    # the largest accepted sizes (n = 31..33, beyond 2^32 bytes per vector) keep the same
    # layout, without overflow in the size arithmetic
    for n in (31, 32, 33):
        for prec, amp in ((0, 8), (1, 16)):
            w = L.cheb_workspace_bytes(n, prec)
            assert 2 * (1 << n) * amp <= w < 2 * (1 << n) * amp * 1.05, (n, prec, w)


def test_adjoint_workspace_bytes():
    """The adjoint's pool grows by one (256-byte aligned) state vector per stored
    vector on top of a fixed part: 6 adjoint ring vectors, G (8 B/amp), Gs (8 B/amp)."""
    L = _lib.lib()
    assert L.cheb_adjoint_workspace_bytes(0, 0, 8) == 0
    assert L.cheb_adjoint_workspace_bytes(22, 0, -1) == 0
    assert L.cheb_adjoint_workspace_bytes(22, 2, 8) == 0
    vb = (1 << 22) * 8
    w0 = L.cheb_adjoint_workspace_bytes(22, 0, 0)
    assert w0 >= 6 * vb + 2 * (1 << 22) * 8
    assert w0 < (6 * vb + 2 * (1 << 22) * 8) * 1.05
    assert L.cheb_adjoint_workspace_bytes(22, 0, 60) - w0 == 60 * vb
    assert L.cheb_adjoint_workspace_bytes(22, 1, 8) - L.cheb_adjoint_workspace_bytes(22, 1, 0) == 8 * 2 * vb


@pytest.mark.parametrize("a,tol,method", [(0.0, 1e-12, "chebyshev"), (19.83, 1e-12, "chebyshev"),
                                          (430.0, 2.0 ** -23, "chebyshev"), (1300.0, 2.0 ** -23, "chebyshev"),
                                          (30.0, 1e-9, "cf"), (430.0, 2.0 ** -23, "cf")])
def test_coefficients_match_oracle(oracle, a, tol, method):
    """The product's generator (sum-of-squares Miller normalisation, its own
    eigensolver for CF) and the oracle's agree coefficient by coefficient."""
    phase = np.exp(-0.25j)
    c, err = api.coefficients(a, tol, method, phase)
    if method == "chebyshev":
        ref, K, tb = oracle.cheb_coeffs(a, tol, phase)
    else:
        ref, K, tb = oracle.cf_coeffs(a, tol, phase)
    assert len(c) == K + 1
    assert np.max(np.abs(c - ref)) < 1e-14
    assert abs(err - tb) <= 1e-3 * tb + 1e-30


def test_coefficients_paper_term_count():
    """Sec. II.B.2: 151 terms for exp(ix) on [-99, 99] at u = 2^-53."""
    c, _ = api.coefficients(99.0, 2.0 ** -53)
    assert len(c) == 151


def test_coefficients_reject_bad_arguments():
    L = _lib.lib()
    buf = np.zeros(16)
    K = ctypes.c_int()
    dp = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.cheb_coefficients(float("nan"), 1, 0, 1e-6, 0, 7, dp, ctypes.byref(K), None) == 1
    assert L.cheb_coefficients(1.0, 1, 0, 0.0, 0, 7, dp, ctypes.byref(K), None) == 1
    assert L.cheb_coefficients(1.0, 1, 0, 1e-6, 5, 7, dp, ctypes.byref(K), None) == 1
    # degree would exceed the buffer
    assert L.cheb_coefficients(100.0, 1, 0, 1e-6, 0, 7, dp, ctypes.byref(K), None) == 6


def test_fused_split_table():
    """Every default split covers exactly the n bits; invalid overrides are refused."""
    for n in range(11, 34):
        l, h = api.get_fused_split(n)
        assert 11 + l + h == n and 0 <= l <= 4 and (h == 0 or h >= 3), (n, l, h)
    with pytest.raises(_lib.ChebError):
        api.set_fused_split(20, 3, 3)  # 11 + 3 + 3 != 20
    with pytest.raises(_lib.ChebError):
        api.set_fused_split(20, 7, 2)  # h = 2 is not a strided pass
    with pytest.raises(_lib.ChebError):
        api.set_fused_split(10, 0, 0)
    with pytest.raises(_lib.ChebError):
        api.set_fused_split(33, 7, 15)  # more L2 partner bits than allowed
    api.set_fused_split(20, 3, 6)
    assert api.get_fused_split(20) == (3, 6)
    api.set_fused_split(20, -1)
    assert api.get_fused_split(20) == (0, 9)


def test_fp64_fused_split_table():
    """The float-float FP64 step: 10 tile bits + l partner bits + h strided bits; each pass
    6..9 bits (5 allowed on 256-byte rows, i.e. starting at bit 17 or above); n = 30 runs
    three partner bits and passes of 9 + 8 bits (the top one on wide rows)."""
    for n in range(11, 34):
        l, h = api.get_fused_split_fp64(n)
        assert 10 + l + h == n and 0 <= l <= 5 and (h == 0 or h >= 5), (n, l, h)
        for lo, hb in _passes(10 + l, h):
            assert 6 <= hb <= 9 or (hb == 5 and lo >= 17), (n, lo, hb)
    assert api.get_fused_split_fp64(30) == (3, 17)
    assert api.get_fused_split_fp64(24) == (0, 14)
    with pytest.raises(_lib.ChebError):
        api.set_fused_split_fp64(20, 0, 10)  # 5 + 5 below bit 17 needs 6-bit passes
    with pytest.raises(_lib.ChebError):
        api.set_fused_split_fp64(20, 3, 6)  # 10 + 3 + 6 != 20
    with pytest.raises(_lib.ChebError):
        api.set_fused_split_fp64(10, 0, 0)
    api.set_fused_split_fp64(20, 4, 6)
    assert api.get_fused_split_fp64(20) == (4, 6)
    api.set_fused_split_fp64(20, -1)
    assert api.get_fused_split_fp64(20) == (1, 9)


def test_autotune_cache_file(tmp_path):
    """cheb_autotune_load applies the cache lines recorded for the named device (later
    lines win) and skips other devices and invalid entries; cheb_autotune_reset drops
    every choice."""
    f = tmp_path / "tune.txt"
    f.write_text("\n".join([
        "cheb-tune-1 TestDev 0 26 2 2 13 0 0.9",
        "cheb-tune-1 TestDev 0 26 2 1 14 1 0.8",     # later line for the same n wins
        "cheb-tune-1 OtherDev 0 27 2 3 13 0 0.1",    # another device
        "cheb-tune-1 TestDev 0 28 2 9 8 0 0.1",      # impossible split: skipped
        "cheb-tune-1 TestDev 1 24 2 5 9 0 2.0",      # float-float split
        "garbage line",
    ]) + "\n")
    try:
        assert api.autotune_load(str(f), "TestDev") == 3
        assert api.get_fused_split(26) == (1, 14)
        assert api.get_fused_split(27) == (0, 16)
        assert api.get_fused_split(28) == (1, 16)
        assert api.get_fused_split_fp64(24) == (5, 9)
    finally:
        api.autotune_reset()
    assert api.get_fused_split(26) == (0, 15)
    assert api.get_fused_split_fp64(24) == (0, 14)
    with pytest.raises(_lib.ChebError):
        api.autotune_load(str(tmp_path / "missing.txt"), "TestDev")


def _passes(lo, h):
    """Near-equal strided passes of at most 9 bits above bit lo (largest first)."""
    if h == 0:
        return []
    np_ = -(-h // 9)
    out = []
    for k in range(np_):
        hb = h // np_ + (1 if k < h % np_ else 0)
        out.append((lo, hb))
        lo += hb
    return out


def test_default_split_gives_the_top_range_wide_rows():
    """Past n = 28 the default split moves one bit to the L2 partner tiles when the top
    strided pass would otherwise be 9 bits at bit 18 or above. An 8-bit top pass there
    runs on 256-byte rows (n = 30: 9 + 8 bits, the benchmarked split). At n = 28 the
    9 + 8 ranges over a low pass without partner bits become 8 + 8 with one partner bit."""
    assert api.get_fused_split(30) == (2, 17)
    expect = {25: (0, 14), 26: (0, 15), 27: (0, 16), 28: (1, 16), 29: (1, 17), 30: (2, 17),
              31: (3, 17), 32: (4, 17), 33: (4, 18)}
    for n, lh in expect.items():
        assert api.get_fused_split(n) == lh, n
    for n in range(25, 33):
        l, h = api.get_fused_split(n)
        lo, hb = _passes(11 + l, h)[-1]
        assert lo + hb == n and not (hb == 9 and lo >= 18), (n, lo, hb)


def test_fused_blocking_switch():
    """The L2-blocked launches are automatic by default (-1), take 0 (off), 1 (step tail)
    or 2 (strided pair), and report the setting."""
    assert api.get_fused_blocking() == -1
    assert _lib.lib().cheb_set_fused_blocking(3) == 1  # CHEB_ERR_INVALID_ARG
    assert _lib.lib().cheb_set_fused_blocking(-2) == 1
    try:
        api.set_fused_blocking(True)
        assert api.get_fused_blocking() == 1
        api.set_fused_blocking(2)
        assert api.get_fused_blocking() == 2
        api.set_fused_blocking(False)
        assert api.get_fused_blocking() == 0
    finally:
        api.set_fused_blocking(None)
    assert api.get_fused_blocking() == -1


def test_fused_compensated_switch():
    """Compensated flip sums are off by default, take 0 or 1, and report their setting."""
    assert api.get_fused_compensated() is False
    assert _lib.lib().cheb_set_fused_compensated(3) == 1  # CHEB_ERR_INVALID_ARG
    api.set_fused_compensated(True)
    try:
        assert api.get_fused_compensated() is True
    finally:
        api.set_fused_compensated(False)
    assert api.get_fused_compensated() is False


def test_magnus4_nodes_match_the_oracle_sampler(oracle):
    """cheb_magnus4_nodes (host only) samples A, B at the Gauss-Legendre points of each
    step exactly as the oracle's sampler does; a failing schedule aborts the call."""
    T, steps = 2.0, 7
    A = lambda t: 1.5 * (1 - t / T) + 0.3 * np.sin(3 * t)
    B = lambda t: t / T + 0.2 * np.cos(2 * t)
    dt, nodes = api.magnus4_nodes(A, B, T, steps)
    dto, nodeso = oracle.magnus4_nodes(A, B, T, steps)
    np.testing.assert_allclose(dt, dto, rtol=0, atol=1e-15)
    np.testing.assert_allclose(nodes, np.asarray(nodeso).reshape(steps, 4), rtol=0, atol=1e-14)

    def bad(t):
        raise ValueError("schedule failure")

    with pytest.raises(_lib.ChebError):
        api.magnus4_nodes(bad, B, T, steps)
    with pytest.raises(_lib.ChebError):
        api.magnus4_nodes(A, lambda t: float("nan"), T, steps)


def test_expmv_rejects_bad_arguments_before_touching_the_device():
    L = _lib.lib()
    n = 4
    h = np.zeros(n)
    J = np.zeros((n, n))
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the checks come first
    ws = L.cheb_workspace_bytes(n, 0)
    # n out of range
    assert L.cheb_expmv(0, dp(h), dp(J), 1.0, 1.0, fake, 0, 1e-6, 0, 0, fake, ws, None, None) == 1
    # null couplings
    assert L.cheb_expmv(n, None, dp(J), 1.0, 1.0, fake, 0, 1e-6, 0, 0, fake, ws, None, None) == 1
    # non-finite coupling
    hb = h.copy()
    hb[1] = np.inf
    assert L.cheb_expmv(n, dp(hb), dp(J), 1.0, 1.0, fake, 0, 1e-6, 0, 0, fake, ws, None, None) == 1
    # workspace too small / misaligned / missing
    assert L.cheb_expmv(n, dp(h), dp(J), 1.0, 1.0, fake, 0, 1e-6, 0, 0, fake, ws - 1, None, None) == 2
    assert L.cheb_expmv(n, dp(h), dp(J), 1.0, 1.0, fake, 0, 1e-6, 0, 0, ctypes.c_void_p((1 << 20) + 8), ws,
                        None, None) == 2
    assert L.cheb_expmv(n, dp(h), dp(J), 1.0, 1.0, fake, 0, 1e-6, 0, 0, None, ws, None, None) == 2
    # bad precision enum, bad method, bad tolerance, misaligned psi, non-finite t
    assert L.cheb_expmv(n, dp(h), dp(J), 1.0, 1.0, fake, 7, 1e-6, 0, 0, fake, ws, None, None) == 1
    assert L.cheb_expmv(n, dp(h), dp(J), 1.0, 1.0, fake, 0, 1e-6, 9, 0, fake, ws, None, None) == 1
    assert L.cheb_expmv(n, dp(h), dp(J), 1.0, 1.0, fake, 0, -1.0, 0, 0, fake, ws, None, None) == 1
    assert L.cheb_expmv(n, dp(h), dp(J), 1.0, 1.0, ctypes.c_void_p((1 << 20) + 4), 0, 1e-6, 0, 0, fake, ws,
                        None, None) == 1
    assert L.cheb_expmv(n, dp(h), dp(J), 1.0, float("inf"), fake, 0, 1e-6, 0, 0, fake, ws, None, None) == 1
    assert L.cheb_expmv(n, dp(h), dp(J), 1.0, 1.0, fake, 0, 1e-6, 0, -1, fake, ws, None, None) == 1
    # the evaluation bound is written into info, so it needs one
    assert L.cheb_expmv_path(n, dp(h), dp(J), 1.0, 1.0, fake, 0, 1e-6, 0, 0, api.EVAL_BOUND_FLAG, fake, ws, None,
                             None) == 1
    # unknown path bits
    assert L.cheb_expmv_path(n, dp(h), dp(J), 1.0, 1.0, fake, 0, 1e-6, 0, 0, 0x40, fake, ws, None, None) == 1


@pytest.mark.parametrize("K,seed", [(0, 0), (1, 1), (7, 2), (50, 3), (120, 4)])
def test_monomial_to_chebyshev(K, seed):
    """The host basis change agrees with numpy's poly2cheb and gives the same values
    as the monomial form on [-1, 1] (Chebyshev series summed by numpy's chebval)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(K + 1) + 1j * rng.standard_normal(K + 1)
    c = api.monomial_to_chebyshev(a)
    ref = np.polynomial.chebyshev.poly2cheb(a.real) + 1j * np.polynomial.chebyshev.poly2cheb(a.imag)
    assert np.max(np.abs(c - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    x = np.linspace(-1, 1, 97)
    pv = np.polynomial.polynomial.polyval(x, a)
    cv = np.polynomial.chebyshev.chebval(x, c)
    assert np.max(np.abs(pv - cv)) <= 1e-12 * max(1.0, np.max(np.abs(pv)))


def test_monomial_to_chebyshev_rejects_bad_input():
    L = _lib.lib()
    buf = np.zeros(4)
    out = np.zeros(4)
    dp = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.cheb_monomial_to_chebyshev(-1, dp(buf), dp(out)) == 1
    assert L.cheb_monomial_to_chebyshev(1, None, dp(out)) == 1
    buf[1] = np.nan
    assert L.cheb_monomial_to_chebyshev(1, dp(buf), dp(out)) == 1


def test_graph_and_checkpoint_entry_points_reject_bad_arguments():
    """The graph capture and checkpointed forward check their arguments on the host
    before any device work; the graph workspace grows with the segment count."""
    L = _lib.lib()
    n, S = 4, 3
    h = np.zeros(n)
    J = np.zeros((n, n))
    g = np.full(S, 0.5)
    t = np.full(S, 0.3)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the checks come first
    gw = L.cheb_anneal_graph_workspace_bytes(n, 0, S)
    assert gw > L.cheb_workspace_bytes(n, 0)
    assert L.cheb_anneal_graph_workspace_bytes(n, 0, 2 * S) > gw
    assert L.cheb_anneal_graph_workspace_bytes(n, 0, 0) == 0
    assert L.cheb_anneal_graph_workspace_bytes(0, 0, S) == 0
    handle = ctypes.c_void_p()
    # no output handle; null schedule; a workspace one byte short; bad method
    assert L.cheb_anneal_graph_create(n, dp(h), dp(J), S, dp(g), None, dp(t), fake, 0, 1e-6, 0, None, fake, gw,
                                      None, None) == 1
    assert L.cheb_anneal_graph_create(n, dp(h), dp(J), S, None, None, dp(t), fake, 0, 1e-6, 0, None, fake, gw,
                                      None, ctypes.byref(handle)) == 1
    assert L.cheb_anneal_graph_create(n, dp(h), dp(J), S, dp(g), None, dp(t), fake, 0, 1e-6, 0, None, fake,
                                      gw - 1, None, ctypes.byref(handle)) == 2
    assert L.cheb_anneal_graph_create(n, dp(h), dp(J), S, dp(g), None, dp(t), fake, 0, 1e-6, 9, None, fake, gw,
                                      None, ctypes.byref(handle)) == 1
    assert not handle.value
    assert L.cheb_anneal_graph_launch(None, None) == 1
    L.cheb_anneal_graph_destroy(None)
    # the checkpointed forward needs the boundaries buffer and an adjoint workspace
    aw = L.cheb_adjoint_workspace_bytes(n, 0, 8)
    assert L.cheb_anneal_checkpointed(n, dp(h), dp(J), S, dp(g), dp(t), fake, 0, 1e-6, 0, None, fake, aw,
                                      None) == 1
    assert L.cheb_anneal_checkpointed(n, dp(h), dp(J), S, dp(g), dp(t), fake, 0, 1e-6, 0, fake, fake, 16,
                                      None) == 2
    assert L.cheb_anneal_general_checkpointed(n, dp(h), dp(J), S, dp(g), None, dp(t), fake, 0, 1e-6, 0, fake,
                                              fake, aw, None) == 1


def test_traffic_profile_covers_the_default_splits():
    """The committed per-launch DRAM bytes (profiles/fused_dram_traffic.json, which
    bench.py scales to the n=30 run) hold the low pass for every number of partner bits
    and the pair for every range shape that the default FP32 splits use at n = 26..30."""
    import json
    import os

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles",
                        "fused_dram_traffic.json")
    with open(path) as f:
        per = json.load(f)["dram_bytes_per_amplitude"]
    for n in range(26, 31):
        l, h = api.get_fused_split(n)
        shape = f"{(h + 1) // 2}+{h // 2}"  # two strided ranges, the first takes the extra bit
        assert str(l) in per["k_low"], (n, l)
        assert shape in per["k_pair"], (n, shape)
        assert 24.0 <= per["k_pair"][shape] <= 48.0 and 32.0 * 0.99 <= per["k_low"][str(l)] <= 40.0


@pytest.mark.parametrize("HA,HB", [(6, 6), (7, 6), (7, 7), (8, 7), (8, 8), (9, 8), (9, 9)])
@pytest.mark.parametrize("gbits", [0, 1, 3, 6])
def test_pair_schedule_is_a_complete_ordered_work_list(HA, HB, gbits):
    """The blocked pair's item order (cheb_pair_schedule_check, the device decode run on
    the host): every A- and B-tile once, then the end marker, and every B-tile of a group
    after all of its A-tiles, for lags from one group to all of them."""
    import ctypes

    lib = _lib.lib()
    for lag in sorted({1, 2, 3, 1 << gbits}):
        if lag > (1 << gbits):
            continue
        gap = ctypes.c_longlong(0)
        assert lib.cheb_pair_schedule_check(gbits, HA, HB, lag, ctypes.byref(gap)) == 0, (gbits, lag)
        assert gap.value >= 1


def test_pair_schedule_at_the_benchmarked_sizes():
    """The work lists of the n=30 split (2, 17) (512 groups, ranges 9 + 8, lag 1) and the
    n=28 split (1, 16) (256 groups, 8 + 8, lag 2): complete and ordered, with at least
    one group's A-tiles between a group's last A-tile and its first B-tile."""
    import ctypes

    lib = _lib.lib()
    for gbits, HA, HB, lag in [(9, 9, 8, 1), (8, 8, 8, 2)]:
        gap = ctypes.c_longlong(0)
        assert lib.cheb_pair_schedule_check(gbits, HA, HB, lag, ctypes.byref(gap)) == 0
        assert gap.value > (1 << HB) * lag - 1, (gbits, gap.value)
    assert lib.cheb_pair_schedule_check(3, 9, 8, 9, None) == -1  # lag above the group count
    assert lib.cheb_pair_schedule_check(3, 10, 8, 1, None) == -1
