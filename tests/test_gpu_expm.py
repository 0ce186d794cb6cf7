"""The small exponential of the Lanczos step (row a5) on its own: the GPU's
c = exp(-i T dt) e_1 (tdse_lanczos_expm, the kernel body every Lanczos step
runs) against a 40-digit eigendecomposition of T (mpmath), for the
tridiagonal matrices the oracle's Lanczos recurrence produces on the
configurations' grids, and for synthetic matrices built to be hard: stiff
(eigenvalues from ~1 to ~1e6), clustered eigenvalues, couplings just above the
breakdown threshold, the largest Krylov dimension.

Bounds: each coefficient within 1e-13 + 4e-16 ||T|| dt (the FP64 rounding of
the phases lambda dt), and |c| = 1 within 1e-14 (the step is unitary)."""
import numpy as np
import pytest

import oracle
import tdse_workloads as W
from gpu_helpers import grid_of

pytestmark = pytest.mark.gpu

mpmath = pytest.importorskip("mpmath")


def _reference(alpha, beta, dt, imag=False):
    """c = V f(Lambda) V^T e_1 in 40 digits, with the breakdown rule of the
    library (beta_j <= 1e-13 max(1, max_{i<=j} |alpha_i|) cuts the space)."""
    m = len(alpha)
    k = m
    amax = 0.0
    for j in range(m - 1):
        amax = max(amax, abs(alpha[j]))
        if beta[j] <= 1e-13 * max(1.0, amax):
            k = j + 1
            break
    mpmath.mp.dps = 40
    T = mpmath.matrix(k, k)
    for i in range(k):
        T[i, i] = mpmath.mpf(float(alpha[i]))
        if i + 1 < k:
            T[i, i + 1] = T[i + 1, i] = mpmath.mpf(float(beta[i]))
    lam, V = mpmath.eigsy(T)
    c = np.zeros(m, dtype=np.complex128)
    for i in range(k):
        s = mpmath.mpc(0)
        for e in range(k):
            ph = mpmath.exp(-lam[e] * dt) if imag else mpmath.exp(-1j * lam[e] * dt)
            s += V[i, e] * V[0, e] * ph
        c[i] = complex(s)
    return c, k


def _check(alpha, beta, dt, imag=False):
    from paper_1308_1856_gb300 import lanczos_expm
    got, k = lanczos_expm(alpha, beta, dt, imag)
    want, kw = _reference(alpha, beta, dt, imag)
    assert k == kw
    tnorm = max(abs(np.asarray(alpha, dtype=float)).max(), abs(np.asarray(beta, dtype=float)).max() if len(beta) else 0)
    tol = 1e-13 + 4e-16 * 3 * tnorm * dt
    err = np.abs(got - want).max()
    assert err <= tol, (err, tol)
    if not imag:
        assert abs(np.linalg.norm(got) - 1.0) <= 1e-14, np.linalg.norm(got) - 1.0
    return err


def _oracle_T(grid, E, m, psi):
    a, b = oracle.lanczos_coefficients(grid, E, m, psi)
    return a, b


def _stiff_cases():
    """(alpha, beta, dt) of Lanczos steps on the configurations' grids."""
    out = []
    c = W.SMALL
    g = grid_of(c.N, c.dr, c.lmax, c.stencil)
    psi = W.smooth_state(c.N, c.dr, c.lmax, seed=1)
    a, b = _oracle_T(g, 0.05, 12, psi)
    out.append(("small dt 0.05", a, b, 0.05))
    # batched-like grids (dr 0.1, lmax up to 127) at a converging step and at dt = 0.02
    for N, L, m, seed in ((2000, 15, 8, 2), (3000, 63, 12, 3), (2500, 127, 16, 4)):
        g = grid_of(N, 0.1, L, 5)
        psi = W.smooth_state(N, 0.1, L, seed=seed, lmax_populated=20)
        a, b = _oracle_T(g, 0.04, m, psi)
        out.append((f"N{N} L{L} m{m} converging", a, b, W.converging_dt(N, 0.1, L, m, 5, 0.04)))
        out.append((f"N{N} L{L} m{m} dt 0.02", a, b, 0.02))
    # the velocity-gauge grid of the full-pulse test near the end of its pulse
    N, dr, L = 300, 0.1, 6
    g = grid_of(N, dr, L, 5, gauge=1)
    psi = W.smooth_state(N, dr, L, seed=5)
    for A in (0.0, 0.2, 20.0):
        a, b = _oracle_T(g, A, 10, psi)
        out.append((f"velocity A={A}", a, b, 0.005))
    return out


CASES = None


def _cases():
    global CASES
    if CASES is None:
        CASES = _stiff_cases()
    return CASES


@pytest.mark.parametrize("i", range(10))
def test_expm_on_lanczos_matrices(i):
    name, a, b, dt = _cases()[i]
    _check(a, b, dt)


def test_expm_on_hard_synthetic_matrices():
    rng = np.random.default_rng(17)
    cases = []
    # stiff: eigenvalues spread over six decades
    for m in (8, 12, 16, 32):
        a = 10.0 ** np.linspace(6, -1, m) * rng.choice([-1.0, 1.0], m)
        b = 10.0 ** rng.uniform(-2, 4, m - 1)
        cases.append((a, b, 5.0 / np.abs(a).max()))
    # clustered: many eigenvalues within 1e-9 of each other, weak couplings
    for m in (6, 12):
        a = 1.0 + 1e-9 * rng.standard_normal(m)
        b = 1e-8 * rng.uniform(0.5, 1.0, m - 1)
        cases.append((a, b, 0.7))
    # couplings just above the breakdown threshold, and at it
    a = np.array([-0.5, 200.0, 150.0, 140.0, 130.0, 120.0])
    b = np.array([4e-6, 50.0, 3e-11, 60.0, 65.0])
    cases.append((a, b, 0.02))
    b2 = b.copy()
    b2[2] = 0.9e-13 * 200.0
    cases.append((a, b2, 0.02))
    # m = 1, 2, 3
    cases.append((np.array([0.3]), np.array([]), 0.1))
    cases.append((np.array([0.3, -1.0]), np.array([0.7]), 0.1))
    cases.append((np.array([0.3, -1.0, 2.0]), np.array([0.7, 1e-3]), 0.1))
    for a, b, dt in cases:
        _check(a, b, dt)


def test_expm_imaginary_time():
    rng = np.random.default_rng(18)
    for m in (4, 12):
        a = rng.uniform(-1, 20, m)
        b = rng.uniform(0.1, 3, m - 1)
        _check(a, b, 0.1, imag=True)
