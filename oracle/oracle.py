"""Python front end of the FP64 oracle (test infrastructure only).

The arithmetic lives in ``oracle.cpp`` (plain C++, FP64, Bessel values in 80-bit
long double); this module compiles it on demand with g++ and calls it through
ctypes with numpy arrays. It also holds the dense-matrix references used to pin
the oracle itself at small n (``dense_hamiltonian``, ``dense_expmv``,
``dense_energy_gradients``): they use numpy / scipy library routines as single
steps (eigh, expm, expm_frechet) and nothing else.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. The CUDA library never does.

What pins each function (tests/test_oracle_pins.py, tests/test_oracle_cf.py):
  energies/bounds      brute force vs a numpy-vectorised restatement at n<=12;
                       symmetric-spectrum shift (Sec. II.A) vs dense eigvalsh
  bessel_j             scipy.special.jv and 40-digit mpmath; J_0^2 + 2 sum J_m^2 = 1;
                       three-term recurrence
  cheb_coeffs          scalar series vs exp(-i a cos theta) (Eq. cheb is exact);
                       tail rule vs brute-force error; K(a) growth (Fig. 1 shape);
                       the paper's 151-term count (tests/golden/paper_term_counts.txt)
  cf_coeffs            equioscillation at >= K+2 points with |error| ~ |lambda|;
                       error below the Chebyshev error of the same degree
  clenshaw / expmv     dense eigh exp(-itH) at n<=10; H_P = 0 closed form
                       (product of cos(gt) I - i sin(gt) X); gamma = 0 pure
                       phases; norm preservation; group property; truncation
                       bound; Walsh-Hadamard check of H_G
  eval_bound           bound >= observed FP64 error (Sec. II.B.3)
  monomial_apply       dense matrix polynomial (numpy matrix powers) at n <= 6
  anneal               ordered product of dense segment exponentials (eigh)
  anneal_general       the same with b_s H_P (dense product)
  magnus4              fourth-order convergence against an adaptive ODE solution
                       (scipy DOP853); a constant schedule gives the exact exponential
  dense gradients      central finite differences; closed form dL/dt
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++ -O2 -fopenmp, no intrinsics)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-fopenmp", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", _LIB_PATH]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.oracle_energies.argtypes = [ctypes.c_int, _dp, _dp, _dp]
            L.oracle_bounds.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, _dp]
            L.oracle_bessel_j.argtypes = [ctypes.c_double, ctypes.c_int, _dp]
            L.oracle_cheb_coeffs.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, _dp, _dp]
            L.oracle_cheb_coeffs.restype = ctypes.c_int
            L.oracle_cf_real.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp]
            L.oracle_cf_real.restype = ctypes.c_double
            L.oracle_cf_coeffs.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, _dp, _dp]
            L.oracle_cf_coeffs.restype = ctypes.c_int
            L.oracle_clenshaw.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int, _dp,
                                          _dp, _dp, _dp]
            L.oracle_monomial_apply.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
            L.oracle_monomial_apply.restype = None
            L.oracle_eval_bound.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double]
            L.oracle_eval_bound.restype = ctypes.c_double
            L.oracle_expmv.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.oracle_expmv.restype = ctypes.c_int
            L.oracle_energy_norm.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _c128_view(psi) -> np.ndarray:
    psi = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128))
    return psi.view(np.float64)


METHODS = {"chebyshev": 0, "cf": 1}


def energies(h, J) -> np.ndarray:
    """E(z) for every basis state z (brute force)."""
    h, J = _f64(h), _f64(J)
    n = h.shape[0]
    E = np.empty(1 << n)
    lib().oracle_energies(n, _p(h), _p(J), _p(E))
    return E


def bounds(h, J, gamma: float):
    """(Emin, Emax, c, r) of Sec. II.A."""
    h, J = _f64(h), _f64(J)
    out = np.empty(4)
    lib().oracle_bounds(h.shape[0], _p(h), _p(J), float(gamma), _p(out))
    return tuple(float(x) for x in out)


def bessel_j(a: float, mmax: int) -> np.ndarray:
    out = np.empty(mmax + 1)
    lib().oracle_bessel_j(float(a), int(mmax), _p(out))
    return out


def _maxk(a: float) -> int:
    a = abs(a)
    return int(np.ceil(a + 25.0 * np.cbrt(a + 1.0) + 60.0))


def cheb_coeffs(a: float, tol: float, phase: complex = 1.0 + 0.0j):
    """Chebyshev coefficients c_0..c_K of exp(-i a x) * phase; returns (coeffs, K, tail_bound)."""
    maxk = _maxk(a)
    buf = np.empty(2 * (maxk + 1))
    tb = np.zeros(1)
    K = lib().oracle_cheb_coeffs(float(a), float(np.real(phase)), float(np.imag(phase)),
                                 float(tol), maxk, _p(buf), _p(tb))
    if K < 0:
        raise ValueError("degree exceeds the coefficient table")
    return buf[: 2 * (K + 1)].view(np.complex128).copy(), K, float(tb[0])


def cf_coeffs(a: float, tol: float, phase: complex = 1.0 + 0.0j):
    """CF near-minimax coefficients of exp(-i a x) * phase; returns (coeffs, K, err_estimate)."""
    maxk = _maxk(a)
    buf = np.empty(2 * (maxk + 1))
    tb = np.zeros(1)
    K = lib().oracle_cf_coeffs(float(a), float(np.real(phase)), float(np.imag(phase)),
                               float(tol), maxk, _p(buf), _p(tb))
    if K < 0:
        raise ValueError("degree exceeds the coefficient table")
    return buf[: 2 * (K + 1)].view(np.complex128).copy(), K, float(tb[0])


def cf_real(a_cheb, K: int):
    """CF correction of a real Chebyshev series a[0..M] to degree K; returns (p, lambda)."""
    a_cheb = _f64(a_cheb)
    M = a_cheb.shape[0] - 1
    p = np.empty(K + 1)
    lam = lib().oracle_cf_real(M, _p(a_cheb), int(K), _p(p))
    return p, float(lam)


def clenshaw(D, g: float, coeffs, psi, with_norms: bool = False):
    """Algorithm 2 with Ht = diag(D) + g * sum_j X_j; returns y (and per-step norms)."""
    D = _f64(D)
    n = int(np.log2(D.shape[0]))
    assert D.shape[0] == 1 << n
    c = _c128_view(coeffs)
    K = c.shape[0] // 2 - 1
    x = _c128_view(psi)
    y = np.empty(2 << n)
    norms = np.empty(3 * (K + 1))
    lib().oracle_clenshaw(n, _p(D), float(g), K, _p(c), _p(x), _p(y), _p(norms))
    out = y.view(np.complex128)
    return (out, norms) if with_norms else out


def monomial_apply(D, g: float, a, psi):
    """y = sum_m a_m Ht^m psi by repeated matvecs (the definition), Ht = diag(D) + g sum_j X_j."""
    D = _f64(D)
    n = int(np.log2(D.shape[0]))
    assert D.shape[0] == 1 << n
    c = _c128_view(a)
    K = c.shape[0] // 2 - 1
    x = _c128_view(psi)
    y = np.empty(2 << n)
    lib().oracle_monomial_apply(n, _p(D), float(g), K, _p(c), _p(x), _p(y))
    return y.view(np.complex128)


def eval_bound(n: int, norms, u: float) -> float:
    norms = _f64(norms)
    K = norms.shape[0] // 3 - 1
    return float(lib().oracle_eval_bound(int(n), K, _p(norms), float(u)))


def expmv(h, J, gamma: float, t: float, psi, tol: float = 1e-12, method: str = "chebyshev",
          splits: int = 1):
    """psi(t) = exp(-i t H) psi by the oracle pipeline. Returns (y, info dict)."""
    h, J = _f64(h), _f64(J)
    n = h.shape[0]
    x = _c128_view(psi)
    assert x.shape[0] == 2 << n
    y = np.empty(2 << n)
    info = np.zeros(12)
    rc = lib().oracle_expmv(n, _p(h), _p(J), float(gamma), float(t), float(tol), METHODS[method],
                            int(splits), _p(x), _p(y), _p(info))
    if rc != 0:
        raise ValueError("oracle_expmv rejected its arguments")
    keys = ["K", "emin", "emax", "center", "radius", "a", "trunc_bound", "eval_bound", "norm",
            "energy", "splits"]
    d = {k: float(info[i]) for i, k in enumerate(keys)}
    d["K"] = int(d["K"])
    return y.view(np.complex128), d


def anneal(h, J, gammas, ts, psi, tol: float = 1e-12, method: str = "chebyshev"):
    """Piecewise-constant schedule: psi <- exp(-i t_s H(gamma_s)) psi for each segment,
    each segment with tolerance tol / S. Returns (final state, list of segment starts)."""
    S = len(gammas)
    cur = np.asarray(psi, dtype=np.complex128).copy()
    starts = []
    for g, t in zip(gammas, ts):
        starts.append(cur.copy())
        cur, _ = expmv(h, J, float(g), float(t), cur, tol / S, method)
    return cur, starts


def anneal_general(h, J, a_s, b_s, ts, psi, tol: float = 1e-12, method: str = "chebyshev"):
    """Segments H_s = b_s H_P + a_s sum_j X_j: psi <- exp(-i t_s H_s) psi in order, each
    with tolerance tol / S (b_s H_P is the energy function of the couplings b_s h, b_s J)."""
    h, J = _f64(h), _f64(J)
    S = len(a_s)
    cur = np.asarray(psi, dtype=np.complex128).copy()
    for a, b, t in zip(a_s, b_s, ts):
        cur, _ = expmv(float(b) * h, float(b) * J, float(a), float(t), cur, tol / S, method)
    return cur


def magnus4_nodes(A, B, T: float, steps: int):
    """Equal steps dt = T/steps of [0, T]; per step (A(t1), B(t1), A(t2), B(t2)) at the
    Gauss-Legendre nodes t1,2 = t + (1/2 -+ sqrt(3)/6) dt."""
    dt = T / steps
    nodes = np.empty((steps, 4))
    for m in range(steps):
        t1 = m * dt + (0.5 - np.sqrt(3.0) / 6.0) * dt
        t2 = m * dt + (0.5 + np.sqrt(3.0) / 6.0) * dt
        nodes[m] = (A(t1), B(t1), A(t2), B(t2))
    return np.full(steps, dt), nodes


def magnus4(h, J, dt, nodes, psi, tol: float = 1e-12, method: str = "chebyshev"):
    """Fourth-order commutator-free Magnus integration of i dpsi/dt = H(t) psi with
    H(t) = A(t) sum_j X_j + B(t) H_P (Sec. III.B and the integrator it cites): per step
    psi <- exp(-i dt (w1 H(t1) + w2 H(t2))) exp(-i dt (w2 H(t1) + w1 H(t2))) psi,
    w1 = 1/4 - sqrt(3)/6, w2 = 1/4 + sqrt(3)/6, each exponential by the oracle's expmv."""
    w1, w2 = 0.25 - np.sqrt(3.0) / 6.0, 0.25 + np.sqrt(3.0) / 6.0
    a_s, b_s, ts = [], [], []
    for d, (A1, B1, A2, B2) in zip(dt, nodes):
        a_s += [w2 * A1 + w1 * A2, w1 * A1 + w2 * A2]
        b_s += [w2 * B1 + w1 * B2, w1 * B1 + w2 * B2]
        ts += [d, d]
    return anneal_general(h, J, a_s, b_s, ts, psi, tol, method)


def energy_norm(h, J, psi):
    h, J = _f64(h), _f64(J)
    x = _c128_view(psi)
    out = np.empty(2)
    lib().oracle_energy_norm(h.shape[0], _p(h), _p(J), _p(x), _p(out))
    return float(out[0]), float(out[1])


# ---------------------------------------------------------------------------
# Dense references (small n only). Library routines serve as single steps.

def dense_hamiltonian(h, J, gamma: float) -> np.ndarray:
    """Explicit 2^n x 2^n H = diag(E) + gamma * sum_j X_j (Sec. I), built entry by entry."""
    h, J = _f64(h), _f64(J)
    n = h.shape[0]
    N = 1 << n
    E = energies(h, J)
    H = np.zeros((N, N))
    for z in range(N):
        H[z, z] = E[z]
        for j in range(n):
            H[z, z ^ (1 << j)] += gamma
    return H


def dense_expmv(h, J, gamma: float, t: float, psi) -> np.ndarray:
    """exp(-i t H) psi through the eigendecomposition of the dense H (Sec. II.A)."""
    H = dense_hamiltonian(h, J, gamma)
    w, V = np.linalg.eigh(H)
    psi = np.asarray(psi, dtype=np.complex128)
    return V @ (np.exp(-1j * t * w) * (V.conj().T @ psi))


def dense_energy_gradients(h, J, gamma: float, t: float, psi0):
    """Exact gradients of L = <y|H_P|y>, y = exp(-i t H) psi0, at small n.

    The directional derivative of exp(A) along E is taken from scipy's
    expm_frechet (the augmented 2N block-matrix exponential), with A = -i t H.
    Returns dict with dL/dgamma, dL/dt, dL/dh (n), dL/dJ (n x n, upper triangle),
    and dL/dpsi0 in PyTorch's convention for a real loss of a complex input
    (conjugate Wirtinger derivative times 2).
    """
    from scipy.linalg import expm, expm_frechet

    h, J = _f64(h), _f64(J)
    n = h.shape[0]
    N = 1 << n
    psi0 = np.asarray(psi0, dtype=np.complex128)
    H = dense_hamiltonian(h, J, gamma).astype(np.complex128)
    E = energies(h, J)
    HP = np.diag(E).astype(np.complex128)
    A = -1j * t * H
    U = expm(A)
    y = U @ psi0
    L = float(np.real(np.vdot(y, HP @ y)))

    def dL_along(dH, dHP):
        # y depends on H through U; the observable depends on H_P directly.
        _, dU = expm_frechet(A, -1j * t * dH, compute_expm=True)
        dy = dU @ psi0
        return float(2.0 * np.real(np.vdot(y, HP @ dy)) + np.real(np.vdot(y, dHP @ y)))

    Z = np.zeros((N, N), dtype=np.complex128)
    HG = (dense_hamiltonian(np.zeros(n), np.zeros((n, n)), 1.0)).astype(np.complex128)
    d_gamma = dL_along(HG, Z)
    d_t = float(2.0 * np.real(np.vdot(y, HP @ (-1j * H @ y))))
    z = np.arange(N)
    s = 1.0 - 2.0 * ((z[:, None] >> np.arange(n)[None, :]) & 1)
    d_h = np.zeros(n)
    for i in range(n):
        dD = np.diag(s[:, i]).astype(np.complex128)
        d_h[i] = dL_along(dD, dD)
    d_J = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            dD = np.diag(s[:, i] * s[:, j]).astype(np.complex128)
            d_J[i, j] = dL_along(dD, dD)
    # dL/dpsi0: L = psi0^H U^H HP U psi0 -> grad (PyTorch convention) = 2 U^H HP U psi0
    g_psi = 2.0 * (U.conj().T @ (HP @ y))
    return {"loss": L, "gamma": d_gamma, "t": d_t, "h": d_h, "J": d_J, "psi0": g_psi, "y": y}
