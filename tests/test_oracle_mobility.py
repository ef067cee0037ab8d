"""Pins for the oracle's single-layer matrix and mobility (Secs. 3.1-3.2, 4.2, 4.4.1)."""
import math

import numpy as np
import pytest

import fbim_synth
from oracle import saddle, singlelayer


def _mobility(Q, ref, L, xi, order=4):
    X = singlelayer.node_positions(Q, ref)
    M = singlelayer.single_layer(X, L, xi, order=order)
    K = saddle.k_matrix(X, Q)
    return saddle.mobility(M, K), M, K


def _dilute_theory(phi):
    # Sec. 4.2, Eq. DiluteTheory (Sangani & Acrivos): F/(eta U)
    return 4 * math.pi / (-math.log(math.sqrt(phi)) - 0.738 + phi - 0.887 * phi ** 2 + 2.039 * phi ** 3)


@pytest.mark.parametrize("phi,tol", [(0.05, 1e-3), (0.1, 2e-3)])
def test_square_array_drag_matches_dilute_theory(phi, tol):
    a = 1.0
    L = a * math.sqrt(math.pi / phi)
    ref = fbim_synth.disk_ref_nodes(64, a)
    N, _, _ = _mobility(np.array([[0.5 * L, 0.5 * L, 0.3]]), ref, L, 3.0)
    drag = 1.0 / N[0, 0]
    assert abs(drag / _dilute_theory(phi) - 1.0) < tol
    # isotropic lattice: N_xx = N_yy, no coupling
    assert abs(N[0, 0] - N[1, 1]) < 1e-8 * N[0, 0]
    assert abs(N[0, 1]) < 1e-10 * N[0, 0]


def test_starfish_self_mobility_matches_printed_diffusion_coefficients():
    # Sec. 4.4.1: four-fold starfish, b = 0.3, a = 1.3 r_s = 0.45, unit cell, N_p = 64;
    # <N_xx> ~ 2.47e-3 and <N_thth> ~ 2.081e-1 (kT = 1, eta = 1, uniform theta).
    ref = fbim_synth.starfish_ref_nodes(64, r_s=0.45 / 1.3, b=0.3, arms=4)
    th = np.linspace(0.0, math.pi / 4, 7)
    vals = []
    for t in th:
        N, _, _ = _mobility(np.array([[0.5, 0.5, t]]), ref, 1.0, 12.0, order=8)
        vals.append((N[0, 0], N[1, 1], N[2, 2]))
        # four-fold symmetry: diagonal with N_xx = N_yy
        assert abs(N[0, 0] - N[1, 1]) < 1e-6 * N[0, 0]
        assert abs(N[0, 2]) < 1e-6 * math.sqrt(N[0, 0] * N[2, 2])
    v = np.array(vals)
    w = np.ones(len(th))
    w[0] = w[-1] = 0.5
    w /= w.sum()
    nxx, nthth = w @ v[:, 0], w @ v[:, 2]
    assert abs(nxx / 2.47e-3 - 1.0) < 2.5e-3
    assert abs(nthth / 0.2081 - 1.0) < 5e-4


def test_alpert_block_is_rotation_covariant():
    ref = fbim_synth.starfish_ref_nodes(32)
    th = 0.83
    Q0 = np.array([[1.0, 1.0, 0.0]])
    Q1 = np.array([[2.0, 0.5, th]])
    A0 = singlelayer.alpert_body(singlelayer.node_positions(Q0, ref)[0], 5.0)
    A1 = singlelayer.alpert_body(singlelayer.node_positions(Q1, ref)[0], 5.0)
    c, s = math.cos(th), math.sin(th)
    R = np.kron(np.eye(32), np.array([[c, -s], [s, c]]))
    assert np.max(np.abs(R @ A0 @ R.T - A1)) < 1e-13 * np.max(np.abs(A0))


@pytest.fixture(scope="module")
def tiny_system(tiny_workload):
    w = tiny_workload
    X = singlelayer.node_positions(w.Q, w.ref_nodes)
    xi = 7.0
    M = singlelayer.single_layer(X, w.L, xi)
    K = saddle.k_matrix(X, w.Q)
    return w, X, M, K


def test_mobility_is_symmetric_positive_definite(tiny_system):
    w, X, M, K = tiny_system
    N = saddle.mobility(M, K)
    assert np.linalg.norm(N - N.T) <= 1e-10 * np.linalg.norm(N)
    assert np.linalg.eigvalsh(0.5 * (N + N.T)).min() > 0.0


def test_discrete_fluctuation_dissipation_identity(tiny_system):
    # Sec. 3.1, Eq. discreteFDB: N^1/2 (N^1/2)^T = N whenever M^1/2 (M^1/2)^T = M.
    w, X, M, K = tiny_system
    lam, V = np.linalg.eigh(M)
    # The Alpert correction leaves each body's near-null normal mode slightly
    # negative (about -2e-5 of the largest eigenvalue here).  For a positive
    # definite M (here M shifted by twice that) the identity is exact; on M
    # itself it holds to the size of those modes.
    Mp = M + 2.0 * abs(min(lam.min(), 0.0)) * np.eye(M.shape[0])
    N = saddle.mobility(Mp, K)
    Nh = saddle.n_half(Mp, K)
    assert np.linalg.norm(Nh @ Nh.T - N) <= 1e-9 * np.linalg.norm(N)
    N = saddle.mobility(M, K)
    Nh = saddle.n_half(M, K)
    assert np.linalg.norm(Nh @ Nh.T - N) <= 1e-6 * np.linalg.norm(N)
    assert lam.min() > -1e-4 * lam.max()


def test_mobility_does_not_depend_on_xi(tiny_workload):
    w = tiny_workload
    # only the Alpert quadrature error depends on xi (Sec. 4.1): about 1e-4
    # for the 4th-order rule and 1e-6 for the 8th-order rule on this case
    for order, tol in ((4, 5e-4), (8, 2e-6)):
        N1, _, _ = _mobility(w.Q, w.ref_nodes, w.L, 5.0, order)
        N2, _, _ = _mobility(w.Q, w.ref_nodes, w.L, 7.0, order)
        assert np.linalg.norm(N1 - N2) <= tol * np.linalg.norm(N1)


def test_gmres_agrees_with_direct_solve(tiny_system):
    w, X, M, K = tiny_system
    A = saddle.saddle_matrix(M, K)
    F = w.F.reshape(-1)
    mu, U = saddle.solve_saddle(M, K, F)
    b = -np.concatenate([np.zeros(M.shape[0]), F])
    x, it, res = saddle.gmres(lambda v: A @ v, b, tol=1e-11, restart=600, max_iter=600)
    assert res <= 1e-11
    assert np.linalg.norm(x[M.shape[0]:] - U) <= 1e-8 * np.linalg.norm(U)


def test_block_preconditioner_is_the_exact_inverse_for_one_unrotated_body():
    # Sec. 3.4: P neglects only inter-body interactions; one body at theta = 0 alone in
    # the box has M~ = M, so applying P^-1 to A x returns x
    ref = fbim_synth.starfish_ref_nodes(32)
    L = 3.0
    xi = math.sqrt(math.log(100.0 / 1e-12)) / (L / 4)
    Q = np.array([[1.1, 1.7, 0.0]])
    X = singlelayer.node_positions(Q, ref)
    M = singlelayer.single_layer(X, L, xi)
    K = saddle.k_matrix(X, Q)
    A = saddle.saddle_matrix(M, K)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(A.shape[0])
    r = A @ x
    mu, U = saddle.block_preconditioner(r[:64], r[64:], Q, ref, L, xi)
    got = A @ np.concatenate([mu.reshape(-1), U.reshape(-1)])
    assert np.max(np.abs(got - r)) < 1e-9 * np.max(np.abs(r))
    assert np.max(np.abs(U.reshape(-1) - x[64:])) < 1e-8 * np.max(np.abs(x[64:]))


def test_block_preconditioner_rotates_the_reference_block_exactly_by_a_quarter_turn():
    # the square periodic lattice is invariant under a quarter turn, so for one body at
    # theta = pi/2 the rotated reference block of Eq. M-block-inverse is its exact block
    # and P^-1 is again the exact inverse; a wrong rotation (R^T for R, or none) breaks it
    ref = fbim_synth.starfish_ref_nodes(32)
    L = 3.0
    xi = math.sqrt(math.log(100.0 / 1e-12)) / (L / 4)
    Q = np.array([[1.1, 1.7, 0.5 * math.pi]])
    X = singlelayer.node_positions(Q, ref)
    A = saddle.saddle_matrix(singlelayer.single_layer(X, L, xi), saddle.k_matrix(X, Q))
    x = np.random.default_rng(7).standard_normal(A.shape[0])
    r = A @ x
    mu, U = saddle.block_preconditioner(r[:64], r[64:], Q, ref, L, xi)
    got = A @ np.concatenate([mu.reshape(-1), U.reshape(-1)])
    assert np.max(np.abs(got - r)) < 1e-9 * np.max(np.abs(r))
    assert np.max(np.abs(U.reshape(-1) - x[64:])) < 1e-8 * np.max(np.abs(x[64:]))
