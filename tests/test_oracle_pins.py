"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with a retyping of itself: every check is a
library routine used as a single step (numpy eigh/norm, scipy/mpmath Bessel,
scipy Hadamard), a closed form, an invariant, or a value printed in the paper.
"""
import os

import numpy as np
import pytest

from paper_2608_12058_b300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Ising diagonal (Sec. I)

@pytest.mark.parametrize("n,seed", [(3, 1), (7, 2), (11, 3)])
def test_energy_invariants(oracle, n, seed):
    """Walsh-function orthogonality fixes the first two moments of E over all z:
    sum_z E(z) = 0 and sum_z E(z)^2 = N (sum_{i<j} J_ij^2 + sum_i h_i^2).
    Flipping every spin leaves the J part unchanged and negates the h part."""
    h, J = I.sk_instance(n, seed)
    E = oracle.energies(h, J)
    N = 1 << n
    assert abs(E.sum()) < 1e-9 * N
    np.testing.assert_allclose((E ** 2).sum(), N * (np.sum(np.triu(J, 1) ** 2) + np.sum(h ** 2)),
                               rtol=1e-12)
    Eh = oracle.energies(h, np.zeros_like(J))
    EJ = oracle.energies(np.zeros_like(h), J)
    z = np.arange(N)
    zc = z ^ (N - 1)
    np.testing.assert_allclose(EJ[zc], EJ[z], atol=1e-12)
    np.testing.assert_allclose(Eh[zc], -Eh[z], atol=1e-12)
    np.testing.assert_allclose(Eh + EJ, E, atol=1e-12)
    # single-spin fields: E for h = e_i is s_i(z) = 1 - 2 bit_i(z)
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        np.testing.assert_array_equal(oracle.energies(e, np.zeros_like(J)), 1.0 - 2.0 * ((z >> i) & 1))
    # a single coupling J_ij reads only i<j and gives s_i s_j
    Jt = np.zeros((n, n))
    Jt[0, n - 1] = 1.0
    np.testing.assert_array_equal(oracle.energies(np.zeros(n), Jt),
                                  (1.0 - 2.0 * (z & 1)) * (1.0 - 2.0 * ((z >> (n - 1)) & 1)))
    np.testing.assert_array_equal(oracle.energies(np.zeros(n), Jt.T), np.zeros(N))


@pytest.mark.parametrize("n,gamma", [(4, 0.7), (8, 1.3), (9, 0.0)])
def test_bounds_are_induced_l1_norm(oracle, n, gamma):
    """Sec. II.A: r equals the induced 1-norm of H - c (numpy's matrix 1-norm) and
    bounds the spectral radius of H - c (numpy eigvalsh)."""
    h, J = I.sk_instance(n, 5)
    emin, emax, c, r = oracle.bounds(h, J, gamma)
    H = oracle.dense_hamiltonian(h, J, gamma)
    Hs = H - c * np.eye(1 << n)
    np.testing.assert_allclose(r, np.linalg.norm(Hs, 1), rtol=1e-13)
    w = np.linalg.eigvalsh(Hs)
    assert np.max(np.abs(w)) <= r * (1 + 1e-13)
    np.testing.assert_allclose([emin, emax], [np.min(np.diag(H)), np.max(np.diag(H))], rtol=1e-13)


# --------------------------------------------------------------------------
# Bessel values by Miller's algorithm (Sec. II.B.1)

@pytest.mark.parametrize("a", [1e-10, 0.3, 1.0, 7.5, 30.0, 99.0, 430.0, 1300.0])
def test_bessel_against_scipy(oracle, a):
    from scipy.special import jv

    mmax = int(a + 40 + 10 * np.cbrt(a))
    j = oracle.bessel_j(a, mmax)
    m = np.arange(mmax + 1)
    ref = jv(m, a)
    big = np.abs(ref) > 1e-250
    # scipy's jv is good to ~1e-14 absolute in the oscillatory region (the tight
    # check against 40-digit mpmath is below); relative accuracy in the decaying tail
    err = np.abs(j - ref)
    assert np.all(err[big] <= 3e-14)
    tail = big & (m > a + 5)
    if np.any(tail):
        np.testing.assert_allclose(j[tail], ref[tail], rtol=1e-11)


@pytest.mark.parametrize("a", [0.5, 12.25, 99.0, 250.0, 1300.0])
def test_bessel_against_mpmath(oracle, a):
    import mpmath

    mpmath.mp.dps = 40
    j = oracle.bessel_j(a, int(a) + 30)
    for m in sorted({0, 1, 2, 15, 16, int(a) // 2, max(int(a) - 1, 0), int(a), int(a) + 10, int(a) + 25}):
        ref = float(mpmath.besselj(m, a))
        assert abs(j[m] - ref) <= 1e-16 + 1e-14 * abs(ref), (m, j[m], ref)


@pytest.mark.parametrize("a", [0.1, 3.0, 77.7, 800.0])
def test_bessel_identities(oracle, a):
    """J_0^2 + 2 sum J_m^2 = 1 (Parseval of Eq. cheb), three-term recurrence, J_m(-a)."""
    mmax = int(a + 60 + 20 * np.cbrt(a))
    j = oracle.bessel_j(a, mmax)
    assert abs(j[0] ** 2 + 2 * np.sum(j[1:] ** 2) - 1.0) < 1e-14
    m = np.arange(1, mmax - 1)
    resid = j[m - 1] + j[m + 1] - (2 * m / a) * j[m]
    assert np.max(np.abs(resid)) < 1e-13 * max(1.0, 2 * mmax / a)
    jn = oracle.bessel_j(-a, mmax)
    np.testing.assert_allclose(jn, j * (-1.0) ** np.arange(mmax + 1), rtol=0, atol=0)


# --------------------------------------------------------------------------
# Chebyshev coefficients (Eq. cheb) and the truncation rule (Eq. TruncError)

@pytest.mark.parametrize("a,tol", [(0.0, 1e-12), (0.01, 1e-14), (5.0, 1e-10), (99.0, 2.0 ** -24),
                                   (430.0, 1e-12), (1300.0, 2.0 ** -23)])
def test_series_reproduces_exponential(oracle, a, tol):
    """The truncated series evaluated by numpy's chebval at x = cos(theta) is
    exp(-i a x) within the stated tail bound (Eq. cheb is exact)."""
    phase = np.exp(-0.37j)
    c, K, tb = oracle.cheb_coeffs(a, tol, phase)
    assert tb <= tol
    x = np.cos(np.linspace(0, np.pi, 4001))
    p = np.polynomial.chebyshev.chebval(x, c)
    err = np.max(np.abs(p - phase * np.exp(-1j * a * x)))
    assert err <= tb + 64 * K * 2.0 ** -53 + 1e-15
    # dropping the last kept coefficient must violate the tolerance (K is minimal)
    if K > 0:
        assert tb + abs(c[K]) > tol


def test_paper_term_count(oracle):
    """Sec. II.B.2: 151 Chebyshev terms for exp(ix) on [-99, 99] at double precision."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_term_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for a, tol, terms, _ in rows:
        _, K, _ = oracle.cheb_coeffs(float(a), float(tol))
        assert K + 1 == int(terms)


def test_term_count_growth(oracle):
    """Fig. 1 / Sec. II.B.2: Chebyshev needs r + o(r) terms, far fewer than the
    Taylor count ~ e r; the excess over r shrinks relative to r."""
    prev = None
    for a in [50.0, 200.0, 800.0, 3200.0]:
        _, K, _ = oracle.cheb_coeffs(a, 2.0 ** -23)
        assert a < K < a + 12 * a ** (1 / 3) + 30
        assert K < np.e * a
        excess = (K - a) / a
        if prev is not None:
            assert excess < prev
        prev = excess


def test_term_count_excess_scales_as_cube_root(oracle):
    """The o(r) of Sec. II.B.2 at large radii: J_m(a) leaves its oscillating range through a
    transition layer around m = a whose width grows as a^(1/3) (the Airy scaling of Bessel
    functions of large order, J_{a + tau a^(1/3)}(a) ~ (2/a)^(1/3) Ai(2^(1/3) tau)), so at a
    fixed tolerance K - a is proportional to a^(1/3): the same constant at a = 1e3 .. 3e4."""
    ratios = []
    for a in [1000.0, 10000.0, 30000.0]:
        _, K, _ = oracle.cheb_coeffs(a, 2.0 ** -23)
        ratios.append((K - a) / a ** (1 / 3))
    assert max(ratios) <= 1.1 * min(ratios), ratios
    assert 3.0 < min(ratios) and max(ratios) < 10.0, ratios


# --------------------------------------------------------------------------
# Matrix-free operator (Sec. II.D) and Clenshaw (Algorithm 2)

def test_hypercube_operator_is_walsh_hadamard_diagonal(oracle):
    """H_G = W diag(n - 2|w|) W / N with W the Sylvester-Hadamard matrix (scipy):
    one Clenshaw run with coefficients (0, 1) applies Ht once."""
    from scipy.linalg import hadamard

    n = 6
    N = 1 << n
    psi = I.random_state(n, 3)
    y = oracle.clenshaw(np.zeros(N), 1.0, np.array([0.0, 1.0], dtype=complex), psi)
    W = hadamard(N)
    pop = np.array([bin(w).count("1") for w in range(N)])
    ref = W @ (np.diag(n - 2.0 * pop) @ (W @ psi)) / N
    np.testing.assert_allclose(y, ref, atol=1e-13)
    # and a pure diagonal
    D = np.linspace(-1, 1, N)
    y = oracle.clenshaw(D, 0.0, np.array([0.0, 1.0], dtype=complex), psi)
    np.testing.assert_allclose(y, D * psi, atol=1e-15)


def test_clenshaw_polynomial_degrees(oracle):
    """Clenshaw with arbitrary coefficients equals sum_m c_m T_m(Ht) psi built from
    numpy's Chebyshev-to-power conversion and explicit dense matrix powers;
    covers the degree-0 and degree-1 special cases."""
    n = 5
    N = 1 << n
    rng = np.random.default_rng(11)
    D = rng.uniform(-0.5, 0.5, N)
    g = 0.09
    Ht = np.diag(D) + g * (oracle.dense_hamiltonian(np.zeros(n), np.zeros((n, n)), 1.0))
    psi = I.random_state(n, 4)
    for K in [0, 1, 2, 7]:
        c = rng.standard_normal(K + 1) + 1j * rng.standard_normal(K + 1)
        y = oracle.clenshaw(D, g, c, psi)
        mono = np.polynomial.chebyshev.cheb2poly(c)
        ref = np.zeros(N, dtype=complex)
        P = np.eye(N)
        for k in range(K + 1):
            ref += mono[k] * (P @ psi)
            P = P @ Ht
        np.testing.assert_allclose(y, ref, atol=1e-12)


@pytest.mark.parametrize("n,seed,gamma,t,tol,psi_kind", [
    (10, 0, 1.0, 1.0, 1e-12, "uniform"),
    (8, 3, 0.4, 3.0, 1e-12, "random"),
    (9, 4, 2.0, 7.5, 1e-10, "random"),
    (6, 5, 1.1, 0.0, 1e-12, "random"),
    (7, 6, 0.8, -2.0, 1e-12, "random"),
])
def test_expmv_matches_dense_eigh(oracle, n, seed, gamma, t, tol, psi_kind):
    """Pin (i): exp(-itH) psi through numpy eigh of the explicit matrix."""
    h, J = I.sk_instance(n, seed)
    psi = I.uniform_state(n) if psi_kind == "uniform" else I.random_state(n, seed + 100)
    y, info = oracle.expmv(h, J, gamma, t, psi, tol)
    ref = oracle.dense_expmv(h, J, gamma, t, psi)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err <= tol + info["eval_bound"] + 1e-13
    assert abs(info["norm"] - 1.0) < tol + 1e-12


def test_config_n10_radius(oracle):
    """The n=10 SK workload has r = (Emax-Emin)/2 + gamma n ~ 19.83 and K ~ 46."""
    c = I.config_n10()
    _, info = oracle.expmv(c.h, c.J, c.gamma, c.t, I.uniform_state(10), 1e-12)
    assert abs(info["radius"] - 19.8312) < 1e-3
    assert 40 <= info["K"] <= 50


@pytest.mark.parametrize("n,gamma,t", [(5, 0.9, 1.7), (12, 0.35, 4.0), (16, 1.0, 2.5)])
def test_expmv_transverse_field_closed_form(oracle, n, gamma, t):
    """Pin (ii): with H_P = 0, exp(-it gamma sum X_j) is the product over qubits of
    cos(gamma t) I - i sin(gamma t) X, so from |0...0>:
    y(z) = cos(gamma t)^(n-|z|) (-i sin(gamma t))^|z|."""
    h = np.zeros(n)
    J = np.zeros((n, n))
    psi = I.basis_state(n, 0)
    y, info = oracle.expmv(h, J, gamma, t, psi, 1e-13)
    z = np.arange(1 << n)
    w = np.array([bin(v).count("1") for v in z])
    ref = np.cos(gamma * t) ** (n - w) * (-1j * np.sin(gamma * t)) ** w
    assert np.linalg.norm(y - ref) <= 1e-13 + info["eval_bound"] + 1e-12


@pytest.mark.parametrize("n,t", [(6, 3.3), (13, 10.0)])
def test_expmv_zero_field_pure_phase(oracle, n, t):
    """Pin (iii): gamma = 0 gives y(z) = exp(-i t E(z)) psi(z); E from the independent
    single-field/single-coupling decomposition checked above."""
    h, J = I.sk_instance(n, 8)
    psi = I.random_state(n, 9)
    y, info = oracle.expmv(h, J, 0.0, t, psi, 1e-13)
    E = oracle.energies(h, J)
    ref = np.exp(-1j * t * E) * psi
    assert np.linalg.norm(y - ref) <= 2e-13 + info["eval_bound"]


def test_expmv_group_property_and_splitting(oracle):
    """Pin (vi): exp(-i t1 H) exp(-i t2 H) = exp(-i (t1+t2) H), and time slicing gives
    the same map; pin (vii): <phi, U psi> = <U(-t) phi, psi>."""
    n = 9
    h, J = I.sk_instance(n, 12)
    psi = I.random_state(n, 13)
    phi = I.random_state(n, 14)
    y1, _ = oracle.expmv(h, J, 0.7, 1.25, psi, 1e-13)
    y12, _ = oracle.expmv(h, J, 0.7, 2.0, y1, 1e-13)
    y3, _ = oracle.expmv(h, J, 0.7, 3.25, psi, 1e-13)
    y3s, info = oracle.expmv(h, J, 0.7, 3.25, psi, 1e-13, splits=4)
    assert np.linalg.norm(y12 - y3) < 1e-11
    assert np.linalg.norm(y3s - y3) < 1e-11
    assert info["splits"] == 4
    u_psi, _ = oracle.expmv(h, J, 0.7, 2.0, psi, 1e-13)
    u_phi, _ = oracle.expmv(h, J, 0.7, -2.0, phi, 1e-13)
    assert abs(np.vdot(phi, u_psi) - np.vdot(u_phi, psi)) < 1e-12


def test_expmv_energy_conservation(oracle):
    """Pin (v): <y|H|y> = <psi|H|psi> (H from the dense matrix)."""
    n = 8
    h, J = I.sk_instance(n, 21)
    psi = I.random_state(n, 22)
    y, _ = oracle.expmv(h, J, 1.4, 6.0, psi, 1e-13)
    H = oracle.dense_hamiltonian(h, J, 1.4)
    assert abs(np.vdot(y, H @ y) - np.vdot(psi, H @ psi)) < 1e-11


def test_truncation_bound_holds(oracle):
    """Pin (viii): the degree-K result differs from a much longer series by no more
    than the tail bound of Eq. TruncError (||T_m(Ht)|| <= 1)."""
    n = 9
    h, J = I.sk_instance(n, 31)
    psi = I.random_state(n, 32)
    _, _, c, r = oracle.bounds(h, J, 1.0)
    E = oracle.energies(h, J)
    D = (E - c) / r
    t = 4.0
    a = t * r
    phase = np.exp(-1j * t * c)
    for tol in [1e-3, 1e-6, 1e-9]:
        ck, K, tb = oracle.cheb_coeffs(a, tol, phase)
        cl, _, _ = oracle.cheb_coeffs(a, 1e-15, phase)
        y = oracle.clenshaw(D, 1.0 / r, ck, psi)
        yl = oracle.clenshaw(D, 1.0 / r, cl, psi)
        d = np.linalg.norm(y - yl)
        assert d <= tb + 1e-13
        assert d > 1e-3 * tb  # the bound is not vacuous


def test_eval_bound_dominates_fp64_error(oracle):
    """Sec. II.B.3: the a-posteriori evaluation bound exceeds the observed error of
    the FP64 recurrence against the dense reference (minus truncation)."""
    n = 10
    h, J = I.sk_instance(n, 41)
    psi = I.random_state(n, 42)
    y, info = oracle.expmv(h, J, 1.0, 5.0, psi, 1e-14)
    ref = oracle.dense_expmv(h, J, 1.0, 5.0, psi)
    err = np.linalg.norm(y - ref)
    assert err <= info["eval_bound"] + info["trunc_bound"] + 1e-13
    assert info["eval_bound"] < 1e-11


# --------------------------------------------------------------------------
# Gradient oracle (dense, Frechet derivative)

def test_dense_gradients_vs_finite_differences(oracle):
    """The expm_frechet gradients agree with central differences of the dense map,
    and dL/dt with the closed form 2 Re <y|H_P (-i H) y>."""
    n = 4
    h, J = I.sk_instance(n, 51)
    psi = I.random_state(n, 52)
    gam, t = 0.8, 1.3
    g = oracle.dense_energy_gradients(h, J, gam, t, psi)

    def loss(h_, J_, gam_, t_, psi_):
        y = oracle.dense_expmv(h_, J_, gam_, t_, psi_)
        E = oracle.energies(h_, J_)
        return float(np.sum(E * np.abs(y) ** 2))

    eps = 1e-6
    fd = (loss(h, J, gam + eps, t, psi) - loss(h, J, gam - eps, t, psi)) / (2 * eps)
    assert abs(fd - g["gamma"]) < 1e-7
    fd = (loss(h, J, gam, t + eps, psi) - loss(h, J, gam, t - eps, psi)) / (2 * eps)
    assert abs(fd - g["t"]) < 1e-7
    for i in range(n):
        e = np.zeros(n)
        e[i] = eps
        fd = (loss(h + e, J, gam, t, psi) - loss(h - e, J, gam, t, psi)) / (2 * eps)
        assert abs(fd - g["h"][i]) < 1e-7
    for (i, j) in [(0, 1), (1, 3), (2, 3)]:
        E_ = np.zeros((n, n))
        E_[i, j] = eps
        fd = (loss(h, J + E_, gam, t, psi) - loss(h, J - E_, gam, t, psi)) / (2 * eps)
        assert abs(fd - g["J"][i, j]) < 1e-7
    # closed form dL/dt = 2 Re <y| H_P (-i H) |y> for L = <y|H_P|y>
    y = oracle.dense_expmv(h, J, gam, t, psi)
    H = oracle.dense_hamiltonian(h, J, gam)
    E = oracle.energies(h, J)
    assert abs(2.0 * np.real(np.vdot(y, E * (-1j * (H @ y)))) - g["t"]) < 1e-10
    # psi0 gradient (PyTorch convention: 2 dL/d conj(psi)) along a random direction
    d = I.random_state(n, 53)
    fd = (loss(h, J, gam, t, psi + eps * d) - loss(h, J, gam, t, psi - eps * d)) / (2 * eps)
    assert abs(fd - np.real(np.vdot(g["psi0"], d))) < 1e-7


def test_dense_gradients_small_t_series(oracle):
    """Gradient pins independent of finite differences. L(t) = <psi| e^{iHt} H_P e^{-iHt} |psi>
    with H = H_P + gamma H_G expands as <H_P> + i t gamma <C> + O(t^2), C = [H_G, H_P].
    So dL/dgamma = i t <C> - (t^2 / 2)(<[H_P, C]> + 2 gamma <[H_G, C]>) + O(t^3).
    At t = 0 the gradients in h and J are the spin moments <s_i>, <s_i s_j> under |psi|^2."""
    n = 4
    h, J = I.sk_instance(n, 61)
    psi = I.random_state(n, 62)
    gam = 0.9
    HP = np.diag(oracle.energies(h, J)).astype(np.complex128)
    HG = oracle.dense_hamiltonian(np.zeros(n), np.zeros((n, n)), 1.0)
    C = HG @ HP - HP @ HG

    def ev(A):
        return np.vdot(psi, A @ psi)

    c1 = 1j * ev(C)
    c2 = -0.5 * (ev(HP @ C - C @ HP) + 2.0 * gam * ev(HG @ C - C @ HG))
    assert abs(c1.imag) < 1e-12 and abs(c2.imag) < 1e-12
    for t in (1e-2, 3e-3, 1e-3):
        g = oracle.dense_energy_gradients(h, J, gam, t, psi)
        series = c1.real * t + c2.real * t * t
        assert abs(g["gamma"] - series) < 50.0 * t ** 3, (t, g["gamma"], series)
    g0 = oracle.dense_energy_gradients(h, J, gam, 0.0, psi)
    z = np.arange(1 << n)
    s = 1.0 - 2.0 * ((z[:, None] >> np.arange(n)[None, :]) & 1)
    w = np.abs(psi) ** 2
    assert np.allclose(g0["h"], s.T @ w, atol=1e-12)
    for i in range(n):
        for j in range(i + 1, n):
            assert abs(g0["J"][i, j] - np.sum(w * s[:, i] * s[:, j])) < 1e-12
    assert abs(g0["gamma"]) < 1e-12


def test_anneal_matches_dense_product(oracle):
    """A piecewise-constant schedule is the ordered product of the segments' dense
    exponentials (eigh of each explicit H_s)."""
    n = 7
    h, J = I.sk_instance(n, 61)
    psi = I.random_state(n, 62)
    gammas = np.array([1.5, 0.9, 0.4, 0.1])
    ts = np.array([0.5, 0.7, 0.3, 1.1])
    y, starts = oracle.anneal(h, J, gammas, ts, psi, 1e-13)
    ref = psi.copy()
    for g, t, st in zip(gammas, ts, starts):
        np.testing.assert_allclose(st, ref, atol=1e-12)
        ref = oracle.dense_expmv(h, J, g, t, ref)
    assert np.linalg.norm(y - ref) < 1e-12


# Polynomials in the monomial basis (Sec. II.B; the Fig. 4 / Fig. 6 workloads)

@pytest.mark.parametrize("n,seed", [(4, 0), (6, 3)])
def test_monomial_apply_matches_dense_matrix_powers(oracle, n, seed):
    """sum_m a_m Ht^m psi by repeated matvecs equals the dense matrix polynomial
    (numpy matrix powers of the explicit Ht), degree 50, N(0,1) coefficients."""
    h, J = I.sk_instance(n, seed)
    gam = 0.7
    E = oracle.energies(h, J)
    c = 0.5 * (E.max() + E.min())
    r = 0.5 * (E.max() - E.min()) + gam * n
    a = I.monomial_polynomial(50, seed) * (1.0 + 0.5j)
    psi = I.random_state(n, seed + 1)
    y = oracle.monomial_apply((E - c) / r, gam / r, a, psi)
    Ht = (oracle.dense_hamiltonian(h, J, gam) - c * np.eye(1 << n)) / r
    ref = sum(a[m] * (np.linalg.matrix_power(Ht, m) @ psi) for m in range(a.shape[0]))
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)


# Time-dependent H (Sec. III.B): general segments and the fourth-order
# commutator-free Magnus integrator

def test_anneal_general_matches_dense_product(oracle):
    """Segments b_s H_P + a_s sum_j X_j, including b_s < 0 and b_s = 0, are the ordered
    product of dense exponentials of the explicit segment matrices."""
    n = 6
    h, J = I.sk_instance(n, 71)
    psi = I.random_state(n, 72)
    a_s = np.array([1.2, 0.0, -0.4, 0.8])
    b_s = np.array([0.3, 1.1, -0.7, 0.0])
    ts = np.array([0.6, 0.4, 0.9, 0.5])
    y = oracle.anneal_general(h, J, a_s, b_s, ts, psi, 1e-13)
    HP = np.diag(oracle.energies(h, J))
    HX = oracle.dense_hamiltonian(np.zeros(n), np.zeros((n, n)), 1.0)
    ref = psi.copy()
    for a, b, t in zip(a_s, b_s, ts):
        w, V = np.linalg.eigh(b * HP + a * HX)
        ref = V @ (np.exp(-1j * t * w) * (V.conj().T @ ref))
    assert np.linalg.norm(y - ref) < 1e-12


def _schedule(T):
    A = lambda t: 1.5 * (1 - t / T) + 0.3 * np.sin(3 * t)
    B = lambda t: t / T + 0.2 * np.cos(2 * t)
    return A, B


def test_magnus4_is_fourth_order(oracle):
    """Halving the step divides the error by ~16 against an adaptive ODE solution of
    i dpsi/dt = (A(t) sum_j X_j + B(t) H_P) psi (a wrong weight, node or factor order
    gives order 2 or less)."""
    from scipy.integrate import solve_ivp

    n, T = 4, 2.0
    h, J = I.sk_instance(n, 3)
    A, B = _schedule(T)
    psi = I.random_state(n, 4)
    HP = np.diag(oracle.energies(h, J))
    HX = oracle.dense_hamiltonian(np.zeros(n), np.zeros((n, n)), 1.0)
    sol = solve_ivp(lambda t, y: -1j * (A(t) * HX + B(t) * HP) @ y, (0, T), psi, method="DOP853",
                    rtol=1e-13, atol=1e-13)
    ref = sol.y[:, -1]
    errs = []
    for M in (8, 16, 32):
        dt, nodes = oracle.magnus4_nodes(A, B, T, M)
        errs.append(np.linalg.norm(oracle.magnus4(h, J, dt, nodes, psi, 1e-14) - ref))
    for e0, e1 in zip(errs, errs[1:]):
        assert 13.0 < e0 / e1 < 19.0


def test_magnus4_constant_schedule_is_exact(oracle):
    """With constant A and B both factors commute and the product is exp(-i T H)."""
    n, T = 5, 1.7
    h, J = I.sk_instance(n, 5)
    psi = I.random_state(n, 6)
    dt, nodes = oracle.magnus4_nodes(lambda t: 0.9, lambda t: 1.0, T, 3)
    y = oracle.magnus4(h, J, dt, nodes, psi, 1e-14)
    assert np.linalg.norm(y - oracle.dense_expmv(h, J, 0.9, T, psi)) < 1e-12
