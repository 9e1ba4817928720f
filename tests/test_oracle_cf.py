"""Pins of the oracle's Caratheodory-Fejer coefficients (Sec. II.C).

A near-best approximation is pinned by what characterises best approximation:
the error curve equioscillates at K+2 points with magnitude ~|lambda| (the
equioscillation theorem quoted in Sec. II.C), and its maximum is below the
error of the Chebyshev truncation of the same degree.
"""
import numpy as np
import pytest


def _real_series(oracle, a, part):
    M = int(a + 25 * np.cbrt(a + 1) + 60)
    j = oracle.bessel_j(a, M)
    m = np.arange(M + 1)
    w = np.where(m == 0, 1.0, 2.0)
    sgn = np.where((m // 2) % 2 == 1, -1.0, 1.0)
    coef = w * sgn * j
    if part == "cos":
        coef[m % 2 == 1] = 0.0
        f = lambda x: np.cos(a * x)
    else:
        coef[m % 2 == 0] = 0.0
        f = lambda x: np.sin(a * x)
    return coef, f


def _alternations(err, level):
    """Number of sign alternations among the extrema of err with |err| >= level."""
    idx = np.where(np.abs(err) >= level)[0]
    signs = np.sign(err[idx])
    count = 1
    for k in range(1, len(signs)):
        if signs[k] != signs[k - 1]:
            count += 1
    return count


@pytest.mark.parametrize("a,K,part", [(10.0, 12, "cos"), (10.0, 13, "sin"), (30.0, 36, "cos"),
                                      (30.0, 35, "sin"), (60.0, 70, "cos")])
def test_cf_equioscillates(oracle, a, K, part):
    coef, f = _real_series(oracle, a, part)
    p, lam = oracle.cf_real(coef, K)
    x = np.cos(np.linspace(0, np.pi, 200001))
    err = f(x) - np.polynomial.chebyshev.chebval(x, p)
    emax = np.max(np.abs(err))
    # |lambda| estimates the error to a few digits
    assert abs(emax - abs(lam)) <= 2e-3 * abs(lam)
    # K+2 alternation points at (nearly) the maximal level; the cos/sin parts have
    # parity, so their effective degree is the largest even/odd number <= K
    deg = K if (K % 2 == 0) == (part == "cos") else K - 1
    assert _alternations(err, 0.98 * emax) >= deg + 2
    # better than the Chebyshev truncation of the same degree
    cheb_err = np.max(np.abs(f(x) - np.polynomial.chebyshev.chebval(x, coef[: K + 1])))
    assert emax < cheb_err
    # and the truncation is near-best (Sec. II.C: Chebyshev approximations lose at most a
    # logarithmic Lebesgue factor against the minimax polynomial; for a truncated series
    # ||f - S_K f|| <= (4 + 4 ln(K) / pi^2) E_K(f), and E_K(f) <= the CF error)
    assert cheb_err <= (4.0 + 4.0 * np.log(K) / np.pi ** 2) * emax


@pytest.mark.parametrize("a,tol", [(10.0, 1e-8), (30.0, 2.0 ** -23), (100.0, 1e-12), (430.0, 2.0 ** -23)])
def test_cf_complex_coefficients(oracle, a, tol):
    """The combined CF polynomial for exp(-i a x) meets tol, never needs more terms
    than Chebyshev, and its error is below the Chebyshev error at equal degree."""
    phase = np.exp(0.6j)
    cf, Kf, est = oracle.cf_coeffs(a, tol, phase)
    ch, Kc, _ = oracle.cheb_coeffs(a, tol, phase)
    assert Kf <= Kc
    x = np.cos(np.linspace(0, np.pi, 40001))
    f = phase * np.exp(-1j * a * x)
    e_cf = np.max(np.abs(f - np.polynomial.chebyshev.chebval(x, cf)))
    e_ch = np.max(np.abs(f - np.polynomial.chebyshev.chebval(x, ch[: Kf + 1])))
    assert e_cf <= tol * 1.01
    assert e_cf <= e_ch
    assert e_cf <= est * 1.01 + 64 * Kf * 2.0 ** -53  # plus chebval rounding


def test_cf_expmv_matches_dense(oracle):
    """The CF path through the full pipeline agrees with the dense reference."""
    from paper_2608_12058_b300 import inputs as I

    n = 8
    h, J = I.sk_instance(n, 7)
    psi = I.random_state(n, 8)
    y, info = oracle.expmv(h, J, 0.9, 4.0, psi, 1e-10, method="cf")
    ref = oracle.dense_expmv(h, J, 0.9, 4.0, psi)
    assert np.linalg.norm(y - ref) <= 1e-10 + info["eval_bound"]


# Remez exchange (Sec. II.C): the product's host generator, pinned by the
# alternation theorem (a certificate of optimality) and against the oracle's CF.

def _alternation_count(e, level):
    """Number of alternating-sign extrema of the sampled error e (increasing abscissae)
    whose size is at least `level` (one per run of constant sign; qualifying runs of
    the same sign in a row count once)."""
    count, last = 0, 0
    run_sign, run_max = None, 0.0
    for v in np.append(e, 0.0):
        s = 1 if v > 0 else (-1 if v < 0 else 0)
        if s != run_sign:
            if run_sign and run_max >= level and run_sign != last:
                count += 1
                last = run_sign
            run_sign, run_max = s, 0.0
        run_max = max(run_max, abs(v))
    return count


@pytest.mark.parametrize("a,tol", [(3.0, 1e-8), (20.0, 1e-10), (30.5, 1e-9), (100.0, 1e-9), (430.0, 2.0 ** -23)])
def test_remez_equioscillates(a, tol):
    """cos(ax) and sin(ax) parts each equioscillate: at least J+2 alternating extrema
    of equal size on [0, 1] (J+1 = dimension of the even/odd subspace of degree <= K),
    which by the alternation theorem makes each the unique minimax polynomial."""
    from paper_2608_12058_b300 import api

    c, err = api.coefficients(a, tol, "remez")
    K = c.shape[0] - 1
    ld = np.longdouble  # the error curves are evaluated in extended precision
    pc, ps = c.real.astype(ld), (-c.imag).astype(ld)
    x = np.cos(np.linspace(ld(np.pi) / 2, ld(0.0), 400001, dtype=ld))  # [0, 1], increasing
    ec = np.cos(ld(a) * x) - np.polynomial.chebyshev.chebval(x, pc)
    es = np.sin(ld(a) * x) - np.polynomial.chebyshev.chebval(x, ps)
    Jc, Js = K // 2, (K - 1) // 2
    # the odd error vanishes at x = 0, which is not an extremum. The margin covers the
    # rounding of the coefficients to FP64 (de la Vallee Poussin: alternation at level
    # (1 - d) E puts the minimax error within a factor 1 - d of E)
    for e, J, q in ((ec, Jc, pc), (es[1:], Js, ps)):
        E = np.max(np.abs(e))
        d = max(1e-3, 10 * np.finfo(np.float64).eps * float(np.sum(np.abs(q))) / float(E))
        assert d < 0.05
        assert _alternation_count(e, E * (1 - d)) >= J + 2
    Ec, Es = float(np.max(np.abs(ec))), float(np.max(np.abs(es)))
    assert np.hypot(Ec, Es) <= tol * (1 + 1e-6)
    assert abs(np.hypot(Ec, Es) - err) <= 1e-5 * err


@pytest.mark.parametrize("a,tol", [(20.0, 1e-10), (60.0, 1e-9), (430.0, 2.0 ** -23)])
def test_remez_agrees_with_oracle_cf_and_beats_chebyshev(oracle, a, tol):
    """The Remez degree equals the oracle's CF degree and its minimax error matches the
    CF estimate |lambda| (CF is near-best) while staying below the truncation bound of
    the Chebyshev series of the same degree."""
    from paper_2608_12058_b300 import api

    cr, er = api.coefficients(a, tol, "remez")
    cf, Kcf, ecf = oracle.cf_coeffs(a, tol)
    K = cr.shape[0] - 1
    assert K == Kcf
    assert abs(er - ecf) <= 1e-3 * ecf
    # Chebyshev series of the same degree: sup error <= its tail sum_{m>K} 2|J_m(a)|
    J = oracle.bessel_j(a, int(a) + 200)
    tail = 2.0 * np.sum(np.abs(J[K + 1:]))
    assert er <= tail
