"""Close body pairs, two-body mobility corrections and the coarse level -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The learned coarse level (hot-path specification; the paper's preconditioner
is the block-diagonal one of Sec. 3.4, Eq. preconditionerGMRES) adds, for each
close pair of bodies (alpha, beta), a 6x6 correction C_ab to the per-body
mobilities N~_b = (K_b^T M_bb^+ K_b)^-1 that the block preconditioner uses:
C_ab approximates N_pair - blockdiag(N_a, N_b), with N_pair the mobility of the
two bodies alone (Sec. 3.1, Eq. discreteParticleVelocity, applied to the pair).

* ``pair_features``   close pairs (gap < g_c) of a configuration, alpha-major, with the
                      network inputs (dx, dy, |d|, cos phi, sin phi, gap): d = q_b - q_a
                      (minimum image) in alpha's frame, phi = theta_b - theta_a, gap =
                      smallest node-to-node distance between the two bodies
* ``two_body``        (N_pair, N_single) from dense solves: body a at the box centre with
                      theta = 0, body b at offset (dx, dy) with theta = phi, box side L
* ``pair_target``     C in alpha's frame: N_pair - blockdiag(N_single, T(phi) N_single T(phi)^T)
* ``to_lab``          T(theta_a) C T(theta_a)^T, T(t) = blockdiag(R(t) + 1, R(t) + 1)
* ``coarse_velocity`` U = N~ a + sum over pairs of C_lab a_pair, the coarse-level body
                      velocities for effective body forces a
* ``coarse_preconditioner`` one application of the block preconditioner of Sec. 3.4
                      with the coarse level: per body g = M~_b^+ r_mu,b and a_b = r_U,b +
                      K_b^T g_b, then U = -coarse_velocity(N~, pairs, C, a) and
                      mu_b = M~_b^+ (r_mu,b + K_b U_b), with M~_b^+ = R_b M_ref^+ R_b^T and
                      N~_b = R_b N~_ref R_b^T (the reference body alone in the box)

Parity: the pair list and features are plain definitions, checked by brute
force and by invariance under a common translation and a periodic shift; the
two-body target is pinned by the symmetry of N_pair and by the decay of C_ab
with separation (the bodies decouple); ``coarse_velocity`` with the exact pair
correction reproduces the mobility of the two bodies from an independent dense
solve.  The network's accuracy for C is unpinned (only the solve it
preconditions is checked).
"""
from __future__ import annotations

import numpy as np

from . import saddle, singlelayer


def _rot(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, -s], [s, c]])


def body_frame_T(theta: float) -> np.ndarray:
    """T(theta): rotates (u_x, u_y, omega) of two bodies by theta (6x6)."""
    T3 = np.eye(3)
    T3[:2, :2] = _rot(theta)
    T = np.zeros((6, 6))
    T[:3, :3] = T3
    T[3:, 3:] = T3
    return T


def pair_features(Q: np.ndarray, ref_nodes: np.ndarray, L: float, g_c: float):
    """Return (pairs [n, 2] int, features [n, 6]) of all pairs with gap < g_c, alpha < beta."""
    X = singlelayer.node_positions(Q, ref_nodes)  # [n_b, n_p, 2]
    n_b = Q.shape[0]
    pairs, feats = [], []
    for a in range(n_b):
        for b in range(a + 1, n_b):
            diff = X[b][None, :, :] - X[a][:, None, :]
            diff -= L * np.round(diff / L)
            gap = float(np.sqrt(np.min(np.sum(diff * diff, axis=2))))
            if gap >= g_c:
                continue
            d = Q[b, :2] - Q[a, :2]
            d -= L * np.round(d / L)
            dl = _rot(-Q[a, 2]) @ d
            phi = Q[b, 2] - Q[a, 2]
            pairs.append((a, b))
            feats.append((dl[0], dl[1], np.hypot(*d), np.cos(phi), np.sin(phi), gap))
    return np.array(pairs, dtype=np.int64).reshape(-1, 2), np.array(feats).reshape(-1, 6)


def _mobility(Q, ref_nodes, L, xi):
    X = singlelayer.node_positions(Q, ref_nodes)
    M = singlelayer.single_layer(X, L, xi)
    K = saddle.k_matrix(X, Q)
    return saddle.mobility(M, K)


def two_body(ref_nodes: np.ndarray, L: float, xi: float, dx: float, dy: float, phi: float):
    """(N_pair 6x6, N_single 3x3) in the frame of body a (theta_a = 0)."""
    c = L / 2.0
    Qp = np.array([[c, c, 0.0], [c + dx, c + dy, phi]])
    Np = _mobility(Qp, ref_nodes, L, xi)
    Ns = _mobility(np.array([[c, c, 0.0]]), ref_nodes, L, xi)
    return Np, Ns


def pair_target(N_pair: np.ndarray, N_single: np.ndarray, phi: float) -> np.ndarray:
    T3 = np.eye(3)
    T3[:2, :2] = _rot(phi)
    C = N_pair.copy()
    C[:3, :3] -= N_single
    C[3:, 3:] -= T3 @ N_single @ T3.T
    return 0.5 * (C + C.T)


def to_lab(C_frame: np.ndarray, theta_a: float) -> np.ndarray:
    T = body_frame_T(theta_a)
    return T @ C_frame @ T.T


def coarse_velocity(N_tilde: np.ndarray, pairs: np.ndarray, C_lab: np.ndarray, a: np.ndarray) -> np.ndarray:
    """U [n_b, 3] = N~_b a_b + sum_{pairs (p, q) containing b} (C_pq [a_p; a_q])_b."""
    U = np.einsum("bij,bj->bi", N_tilde, a)
    for (p, q), C in zip(pairs, C_lab):
        aa = np.concatenate([a[p], a[q]])
        du = C @ aa
        U[p] += du[:3]
        U[q] += du[3:]
    return U


def coarse_preconditioner(r_mu, r_U, Q, ref_nodes, L, xi, pairs, C_lab, eta=1.0, order=4):
    """P^-1 [r_mu; r_U] with the coarse level: returns (mu [N, 2], U [N_b, 3])."""
    n_b, n_p = Q.shape[0], ref_nodes.shape[0]
    Xr = singlelayer.node_positions(np.array([[0.5 * L, 0.5 * L, 0.0]]), ref_nodes)
    Mp_ref = saddle.pinv_sym(singlelayer.single_layer(Xr, L, xi, eta, order))
    K_ref = saddle.k_matrix(Xr, np.array([[0.5 * L, 0.5 * L, 0.0]]))
    N_ref = np.linalg.inv(K_ref.T @ Mp_ref @ K_ref)
    X = singlelayer.node_positions(Q, ref_nodes)
    r_mu = np.asarray(r_mu, dtype=np.float64).reshape(n_b, 2 * n_p)
    r_U = np.asarray(r_U, dtype=np.float64).reshape(n_b, 3)
    Mp, Kb, a, N_t = [], [], np.zeros((n_b, 3)), np.zeros((n_b, 3, 3))
    for b in range(n_b):
        c, s = np.cos(Q[b, 2]), np.sin(Q[b, 2])
        R = np.kron(np.eye(n_p), np.array([[c, -s], [s, c]]))
        T3 = np.eye(3)
        T3[:2, :2] = [[c, -s], [s, c]]
        Mp.append(R @ Mp_ref @ R.T)
        Kb.append(saddle.k_matrix(X[b:b + 1], Q[b:b + 1]))
        a[b] = r_U[b] + Kb[b].T @ Mp[b] @ r_mu[b]
        N_t[b] = T3 @ N_ref @ T3.T
    U = -coarse_velocity(N_t, pairs, C_lab, a)
    mu = np.stack([Mp[b] @ (r_mu[b] + Kb[b] @ U[b]) for b in range(n_b)])
    return mu.reshape(-1, 2), U
