"""Rigid-body coupling, the saddle-point system and the mobility -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``k_matrix``   K: (K_beta U_beta)_j = u_beta + omega_beta x (x_{beta,j} - q_beta), and K^T
                 sums node forces and torques                              (Sec. 3.1)
* ``saddle_matrix`` [[M, -K], [-K^T, 0]]                                   (Sec. 3.1, Eq. discreteSaddlePoint)
* ``solve_saddle`` dense LU solve of  [[M,-K],[-K^T,0]] [mu; U] = -[slip; F]
* ``mobility``   N = (K^T M^+ K)^-1, column by column from saddle solves with unit F
                                                                           (Sec. 3.1, Eq. discreteParticleVelocity)
* ``n_half``     N^1/2 = N K^T M^+ M^1/2                                   (Sec. 3.1, Eq. discreteParticleVelocity)
* ``gmres``      plain restarted GMRES (Arnoldi with modified Gram-Schmidt, Givens
                 rotations), unpreconditioned, for the iteration-count comparison
* ``block_preconditioner``  one application of the block-diagonal preconditioner P
                 (Sec. 3.4, Eqs. preconditionerGMRES, approximate-body-mobility,
                 M-block-inverse): per body, [[M~_bb, -K_b], [-K_b^T, 0]] [mu; U] = [r_mu; r_U]
                 with M~_bb^+ = R_b M_ref^+ R_b^T, solved through the Schur complement
                 N~_b = (K_b^T M~_bb^+ K_b)^-1 with K_b from the body's actual nodes

Parity: pinned by the symmetry and positive-definiteness of N (Sec. 2, the
mobility is SPD), by the exact identity N^1/2 (N^1/2)^T = N (Sec. 3.1,
Eq. discreteFDB) and by the disk-array drag (Sec. 4.2, Eq. DiluteTheory).
``block_preconditioner`` is pinned by the case where it is the exact inverse: one
body at theta = 0 alone in the box (then M~ = M and P^-1 = A^-1 exactly), and by
the same body turned by a quarter turn (the square lattice is invariant under it,
so Eq. M-block-inverse is exact and P^-1 = A^-1 again).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def k_matrix(X: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """K [2N, 3N_b] for nodes X [N_b, N_p, 2] and body coordinates Q [N_b, 3]."""
    n_b, n_p = X.shape[:2]
    K = np.zeros((n_b, n_p, 2, n_b, 3))
    r = X - Q[:, None, :2]
    for b in range(n_b):
        K[b, :, 0, b, 0] = 1.0
        K[b, :, 1, b, 1] = 1.0
        K[b, :, 0, b, 2] = -r[b, :, 1]
        K[b, :, 1, b, 2] = r[b, :, 0]
    return K.reshape(2 * n_b * n_p, 3 * n_b)


def saddle_matrix(M: np.ndarray, K: np.ndarray) -> np.ndarray:
    n, m = K.shape
    A = np.zeros((n + m, n + m))
    A[:n, :n] = M
    A[:n, n:] = -K
    A[n:, :n] = -K.T
    return A


def solve_saddle(M: np.ndarray, K: np.ndarray, F: np.ndarray, slip: np.ndarray | None = None):
    """Return (mu [2N], U [3N_b]) solving the saddle system for one or more right-hand sides."""
    n, m = K.shape
    A = saddle_matrix(M, K)
    F = np.asarray(F, dtype=np.float64)
    cols = F.ndim == 2
    Fm = F.reshape(m, -1)
    S = np.zeros((n, Fm.shape[1])) if slip is None else np.asarray(slip, dtype=np.float64).reshape(n, -1)
    rhs = -np.concatenate([S, Fm], axis=0)
    sol = sla.lu_solve(sla.lu_factor(A), rhs)
    mu, U = sol[:n], sol[n:]
    if not cols:
        mu, U = mu[:, 0], U[:, 0]
    return mu, U


def mobility(M: np.ndarray, K: np.ndarray) -> np.ndarray:
    """N [3N_b, 3N_b]: U = N F with no slip."""
    m = K.shape[1]
    _, U = solve_saddle(M, K, np.eye(m))
    return U


def pinv_sym(M: np.ndarray, rel: float = 1e-12) -> np.ndarray:
    """Pseudo-inverse of a symmetric matrix: eigenvalues with |lam| <= rel max|lam| dropped."""
    lam, V = np.linalg.eigh(M)
    keep = np.abs(lam) > rel * np.max(np.abs(lam))
    return (V[:, keep] / lam[keep]) @ V[:, keep].T


def sqrt_sym(M: np.ndarray) -> np.ndarray:
    """Principal square root of a symmetric matrix, negative eigenvalues clipped to 0."""
    lam, V = np.linalg.eigh(M)
    return (V * np.sqrt(np.clip(lam, 0.0, None))) @ V.T


def n_half(M: np.ndarray, K: np.ndarray, M_half: np.ndarray | None = None) -> np.ndarray:
    """N^1/2 = N K^T M^+ M^1/2 (Sec. 3.1)."""
    N = mobility(M, K)
    Mp = pinv_sym(M)
    Mh = sqrt_sym(M) if M_half is None else M_half
    return N @ K.T @ Mp @ Mh


def gmres(apply_A, b: np.ndarray, tol: float = 1e-10, restart: int = 200, max_iter: int = 2000,
          apply_P=None):
    """Restarted GMRES; right preconditioner apply_P optional.  Returns (x, iters, rel_res)."""
    n = b.shape[0]
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    P = apply_P if apply_P is not None else (lambda v: v)
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or it >= max_iter:
            return x, it, beta / bnorm
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(restart):
            Z[k] = P(V[k])
            w = apply_A(Z[k])
            for i in range(k + 1):
                H[i, k] = w @ V[i]
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            d = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / d, H[k + 1, k] / d
            H[k, k] = d
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_used = k + 1
            if abs(g[k + 1]) / bnorm <= tol or it >= max_iter:
                break
        y = sla.solve_triangular(H[:k_used, :k_used], g[:k_used])
        x = x + y @ Z[:k_used]


def block_preconditioner(r_mu: np.ndarray, r_U: np.ndarray, Q: np.ndarray, ref_nodes: np.ndarray, L: float,
                         xi: float, eta: float = 1.0, order: int = 4):
    """P^-1 [r_mu; r_U] for bodies Q [N_b, 3]: returns (mu [N, 2], U [N_b, 3]).

    M_ref is the single-layer matrix of the reference body alone in the box (theta = 0),
    M_ref^+ its pseudo-inverse (|lambda| <= 1e-12 max |lambda| dropped), rotated to each
    body as R_b M_ref^+ R_b^T (Eq. M-block-inverse).  Per body b the 2 x 2 block system
    gives U_b = -N~_b (r_U,b + K_b^T M~_b^+ r_mu,b) and mu_b = M~_b^+ (r_mu,b + K_b U_b).
    """
    from . import singlelayer
    n_b, n_p = Q.shape[0], ref_nodes.shape[0]
    Xr = singlelayer.node_positions(np.array([[0.5 * L, 0.5 * L, 0.0]]), ref_nodes)
    Mp_ref = pinv_sym(singlelayer.single_layer(Xr, L, xi, eta, order))
    X = singlelayer.node_positions(Q, ref_nodes)
    r_mu = np.asarray(r_mu, dtype=np.float64).reshape(n_b, 2 * n_p)
    r_U = np.asarray(r_U, dtype=np.float64).reshape(n_b, 3)
    mu = np.zeros((n_b, 2 * n_p))
    U = np.zeros((n_b, 3))
    for b in range(n_b):
        c, s = np.cos(Q[b, 2]), np.sin(Q[b, 2])
        R = np.kron(np.eye(n_p), np.array([[c, -s], [s, c]]))
        Mp = R @ Mp_ref @ R.T
        Kb = k_matrix(X[b:b + 1], Q[b:b + 1])
        Nt = np.linalg.inv(Kb.T @ Mp @ Kb)
        U[b] = -Nt @ (r_U[b] + Kb.T @ Mp @ r_mu[b])
        mu[b] = Mp @ (r_mu[b] + Kb @ U[b])
    return mu.reshape(-1, 2), U
