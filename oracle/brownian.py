"""Random slip M^1/2 W by the positively split Ewald sum -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The slip is split into independent near- and far-field parts (Sec. 3.3,
Eq. sqrtM-split):

    slip = sqrt(2 kT / dt) [ (M^(r))^1/2 W^(r) + (M^(w))^1/2 W^(w) ].

* ``near_field``  y = G^+ (G M^(r) G^T)^1/2 W^(r) with the block-diagonal G built
                  from the reference body's real-space block (Sec. 3.4,
                  Eqs. preconditioned-real-part, Gprecond-decomp, Gprecond-precompute),
                  here by dense eigendecomposition (principal square root).
* ``far_field``   (eta V)^-1/2 sum_kappa e^{i k.x} B^1/2(k) W(kappa) with
                  B^1/2 = H^^1/2 / k (I - k^ k^^T)          (Sec. 3.3, Eq. sqrtMwave),
                  as a direct sum over the same lattice of modes as an M x M grid,
                  without the Nyquist lines (see the reading below).
* ``hermitian_noise`` builds W(kappa) on that lattice from standard normals
                  Z [M, M, 2, 2] (Sec. 3.3: zero mode 0; the three Nyquist modes
                  real N(0, I); other modes a + i b with a, b ~ N(0, I/2) and
                  W(kappa) = conj W(-kappa mod M)).

Readings: the paper sets G_ref = (Sigma^+)^1/2 V^*, which depends on the
eigenvector basis.  Here G_ref = V (Sigma^+)^1/2 V^T and G_ref^+ = V Sigma^1/2 V^T
(the principal inverse square root and square root of M^(r)_ref): basis-free,
same covariance.  Eigenvalues below 1e-12 of the largest are treated as
spurious and zeroed.  Of each conjugate pair of modes, the member with the
smaller linear index j_y M + j_x (j = kappa mod M) is the canonical one and
takes a = Z[..., 0]/sqrt 2, b = Z[..., 1]/sqrt 2; a self-conjugate mode takes
Z[..., 0].  The far-field sum leaves out the Nyquist lines kappa_x = -M/2 and
kappa_y = -M/2 (including the three real Nyquist modes that Sec. 3.3 draws from
N(0, I)): on an M-point grid such a mode stands for both +k_N and -k_N, so its
gridded interpolation is not the value of the single lattice mode, and the grid
is chosen so that the Hasimoto weight there is below the Ewald tolerance; the
covariance changes by less than that tolerance.

Parity: pinned by the covariance identities (the far field's covariance is
M^(w); G^+ G M^(r)_ref G^T G^+T = M^(r)_ref, Sec. 3.4) and the statistical
fluctuation-dissipation test.
"""
from __future__ import annotations

import numpy as np

from . import ewald, singlelayer

SPURIOUS_REL = 1e-12


def rotation_blocks(theta: np.ndarray, n_p: int) -> np.ndarray:
    """Block-diagonal R = diag(R(theta_beta) per node) [2N, 2N]."""
    n_b = theta.shape[0]
    R = np.zeros((2 * n_b * n_p, 2 * n_b * n_p))
    for b in range(n_b):
        c, s = np.cos(theta[b]), np.sin(theta[b])
        for j in range(n_p):
            i = 2 * (b * n_p + j)
            R[i:i + 2, i:i + 2] = [[c, -s], [s, c]]
    return R


def reference_real_block(ref_nodes: np.ndarray, L: float, xi: float, eta: float = 1.0,
                         order: int = 4) -> np.ndarray:
    """M^(r)_ref: the real-space block of the reference body alone in the box."""
    Q = np.array([[0.5 * L, 0.5 * L, 0.0]])
    X = singlelayer.node_positions(Q, ref_nodes)
    return singlelayer.real_matrix(X, L, xi, eta, order)


def g_factors(Mr_ref: np.ndarray, rel: float = SPURIOUS_REL):
    lam, V = np.linalg.eigh(Mr_ref)
    keep = lam > rel * np.max(np.abs(lam))
    G = (V[:, keep] / np.sqrt(lam[keep])) @ V[:, keep].T
    Gd = (V[:, keep] * np.sqrt(lam[keep])) @ V[:, keep].T
    return G, Gd


def near_field(X: np.ndarray, Q: np.ndarray, ref_nodes: np.ndarray, L: float, xi: float,
               W_r: np.ndarray, eta: float = 1.0, order: int = 4) -> np.ndarray:
    """G^+ (G M^(r) G^T)^1/2 W^(r); W_r [N, 2] standard normals -> [N, 2]."""
    n_b, n_p = X.shape[:2]
    Mr = singlelayer.real_matrix(X, L, xi, eta, order)
    G_ref, Gd_ref = g_factors(reference_real_block(ref_nodes, L, xi, eta, order))
    R = rotation_blocks(Q[:, 2], n_p)
    G = R @ np.kron(np.eye(n_b), G_ref) @ R.T
    Gd = R @ np.kron(np.eye(n_b), Gd_ref) @ R.T
    A = G @ Mr @ G.T
    A = 0.5 * (A + A.T)
    lam, V = np.linalg.eigh(A)
    y = (V * np.sqrt(np.clip(lam, 0.0, None))) @ (V.T @ W_r.reshape(-1))
    return (Gd @ y).reshape(-1, 2)


def mode_lattice(M: int):
    """Signed mode indices kappa for j = 0..M-1 (kappa = j, or j - M for j >= M/2)."""
    j = np.arange(M)
    return np.where(j < M // 2, j, j - M)


def hermitian_noise(Z: np.ndarray) -> np.ndarray:
    """W [M, M, 2] complex on the lattice (index [j_y, j_x, comp]) from normals Z [M, M, 2, 2]."""
    M = Z.shape[0]
    jy, jx = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    lin = jy * M + jx
    py, px = (-jy) % M, (-jx) % M
    plin = py * M + px
    W = np.zeros((M, M, 2), dtype=np.complex128)
    canon = lin < plin
    W[canon] = (Z[canon][..., 0] + 1j * Z[canon][..., 1]) / np.sqrt(2.0)
    other = lin > plin
    W[other] = np.conj(W[py[other], px[other]])
    selfc = (lin == plin) & (lin != 0)
    W[selfc] = Z[selfc][..., 0]
    return W


def far_field(Xf: np.ndarray, L: float, xi: float, Z: np.ndarray, eta: float = 1.0) -> np.ndarray:
    """(M^(w))^1/2 W^(w) at nodes Xf [N, 2] by the direct sum over the M x M lattice."""
    M = Z.shape[0]
    W = hermitian_noise(Z)
    kap = mode_lattice(M)
    ky, kx = np.meshgrid(kap, kap, indexing="ij")
    kvec = np.stack([kx.ravel(), ky.ravel()], axis=1) * (2.0 * np.pi / L)
    Wf = W.reshape(-1, 2)
    nyq = ((ky == -(M // 2)) | (kx == -(M // 2))).ravel()
    nz = np.any(kvec != 0.0, axis=1) & ~nyq
    kvec, Wf = kvec[nz], Wf[nz]
    k2 = np.sum(kvec * kvec, axis=1)
    s = np.sqrt(ewald.hasimoto(np.sqrt(k2), xi)) / np.sqrt(k2)      # H^1/2 / k
    Bh = np.empty((kvec.shape[0], 2, 2))
    Bh[:, 0, 0] = s * (1.0 - kvec[:, 0] ** 2 / k2)
    Bh[:, 1, 1] = s * (1.0 - kvec[:, 1] ** 2 / k2)
    Bh[:, 0, 1] = -s * kvec[:, 0] * kvec[:, 1] / k2
    Bh[:, 1, 0] = Bh[:, 0, 1]
    u = np.einsum("kab,kb->ka", Bh, Wf)
    out = np.zeros((Xf.shape[0], 2))
    for c0 in range(0, kvec.shape[0], 100000):
        e = np.exp(1j * (Xf @ kvec[c0:c0 + 100000].T))
        out += np.real(e @ u[c0:c0 + 100000])
    return out / np.sqrt(eta * L * L)


def slip(X, Q, ref_nodes, L, xi, kT, dt, W_r, Z, eta=1.0, order=4):
    """sqrt(2kT/dt) [near + far] at all nodes, [N, 2]."""
    near = near_field(X, Q, ref_nodes, L, xi, W_r, eta, order)
    far = far_field(X.reshape(-1, 2), L, xi, Z, eta)
    return np.sqrt(2.0 * kT / dt) * (near + far)
