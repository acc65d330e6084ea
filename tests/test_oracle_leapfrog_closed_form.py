"""Closed-form pins of the oracle's leapfrog (App. B; the kick-drift-kick integrator of
Neal 2011).

On a quadratic potential U(q) = q^T A q / 2 one step with mass M is the linear map
T = K D K with the half kick K = [[I, 0], [-(eps/2) A, I]] and the drift
D = [[I, eps M^-1], [0, I]], so n steps are T^n applied to (q0, p0).  Here T is built from
these textbook blocks and a library inverse of M = L L^T, independently of the oracle's
triangular solves.  A dropped half kick, a drift by M instead of M^-1, a swapped order or a
wrong block offset in the mass matrix each move the end point by far more than rounding.
For one degree of freedom the map also conserves the quadratic form
p^2 / m + omega^2 (1 - eps^2 omega^2 / (4 m)) q^2 exactly, the integrator's own invariant.
"""
import numpy as np

import oracle


def _quadratic(A):
    def fn(q):
        g = A @ q
        return 0.5 * float(q @ g), g
    return fn


def _leapfrog_map(A, Minv, eps):
    n = A.shape[0]
    I, Z = np.eye(n), np.zeros((n, n))
    kick = np.block([[I, Z], [-0.5 * eps * A, I]])
    drift = np.block([[I, eps * Minv], [Z, I]])
    return kick @ drift @ kick


def test_scalar_oscillator_matches_textbook_map_and_invariant():
    omega2, m = 2.3, 0.7
    A = np.array([[omega2]])
    mass = oracle.BlockCholesky([(0, np.array([[np.sqrt(m)]]))])
    q0, p0 = np.array([0.8]), np.array([-0.35])
    for eps, n in ((0.1, 1), (0.1, 20), (0.37, 13)):
        # the one-step map written out: q' = (1 - e w^2/2m) q + (e/m) p, and so on
        c = 1.0 - eps * eps * omega2 / (2.0 * m)
        T = np.array([[c, eps / m], [-eps * omega2 * (1.0 - eps * eps * omega2 / (4.0 * m)), c]])
        assert abs(np.linalg.det(T) - 1.0) < 1e-12                      # symplectic
        want = np.linalg.matrix_power(T, n) @ np.array([q0[0], p0[0]])
        q, p, H0, H1, acc = oracle.leapfrog(_quadratic(A), q0, p0, eps, n, 0.0, mass)
        np.testing.assert_allclose([q[0], p[0]], want, rtol=1e-12, atol=1e-14)
        assert abs(H0 - (0.5 * omega2 * q0[0] ** 2 + 0.5 * p0[0] ** 2 / m)) < 1e-14
        assert abs(H1 - (0.5 * omega2 * q[0] ** 2 + 0.5 * p[0] ** 2 / m)) < 1e-14
        inv = lambda qq, pp: pp * pp / m + omega2 * (1.0 - eps * eps * omega2 / (4.0 * m)) * qq * qq
        assert abs(inv(q[0], p[0]) - inv(q0[0], p0[0])) < 1e-12 * inv(q0[0], p0[0])
        assert acc                                                      # u = 0 always accepts


def test_block_mass_quadratic_matches_matrix_power():
    rng = np.random.default_rng(21)
    n = 7
    B = rng.standard_normal((n, n))
    A = B @ B.T + n * np.eye(n)                                         # SPD potential
    # two mass blocks at offsets 0 and 4 (a wrong offset mixes the blocks)
    L1 = np.tril(rng.standard_normal((4, 4))) + 3.0 * np.eye(4)
    L2 = np.tril(rng.standard_normal((3, 3))) + 3.0 * np.eye(3)
    mass = oracle.BlockCholesky([(0, L1), (4, L2)])
    M = np.zeros((n, n))
    M[:4, :4] = L1 @ L1.T
    M[4:, 4:] = L2 @ L2.T
    Minv = np.linalg.inv(M)
    q0 = rng.standard_normal(n)
    p0 = mass.mul_lower(rng.standard_normal(n))
    for eps, steps in ((0.05, 1), (0.05, 20), (0.2, 9)):
        want = np.linalg.matrix_power(_leapfrog_map(A, Minv, eps), steps) @ np.concatenate([q0, p0])
        q, p, H0, H1, _ = oracle.leapfrog(_quadratic(A), q0, p0, eps, steps, 0.0, mass)
        scale = np.abs(want).max()
        np.testing.assert_allclose(np.concatenate([q, p]), want, rtol=0, atol=1e-11 * scale)
        # H = U + p^T M^-1 p / 2 at both ends
        assert abs(H0 - (0.5 * q0 @ A @ q0 + 0.5 * p0 @ Minv @ p0)) < 1e-11 * abs(H0)
        assert abs(H1 - (0.5 * q @ A @ q + 0.5 * p @ Minv @ p)) < 1e-11 * abs(H1)
