"""Dense single-layer matrix M = M(t) + M(a) + M(w) -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Vector layout: nodes are body-major (body beta, node j), so a density or a
velocity is an array [N_b * N_p, 2]; matrices act on its row-major
flattening (index 2 m + c).  mu_m is the force carried by node m (Sec. 3.1:
mu = psi * Delta s, read as the node force psi |gamma'| Delta s).

* ``trapezoid_real``  M(t): G^(r)(x_m - x_n) summed over periodic images, zero
                      for m = n                          (Sec. 3.2, Eq. Mreal-decompose)
* ``wave_matrix``     M(w): G^(w)(x_m - x_n), diagonal included (Sec. 3.2, Eq. Mwave-elements)
* ``alpert_body``     M(a) for one body from its actual node coordinates: the
                      Alpert rule of ``oracle.alpert`` applied to the log-singular
                      real-space integrand, with the density carried from the
                      nodes to the auxiliary points by Lagrange interpolation,
                      minus the trapezoidal terms it replaces (Sec. 3.2)
* ``single_layer``    M = M(t) + M(w) + (M(a) + M(a)^T)/2

Reading: only the symmetric part of M(a) is used, in the solves as well as in
the square root (Sec. 3.3 uses it for the square root; using it everywhere
keeps M symmetric so that the discrete fluctuation-dissipation identity,
Eq. discreteFDB, holds exactly).

Parity: M(t) + M(w) off the diagonal is pinned by xi-independence; M(a) by the
closed-form tests of the rule and, through the whole solve, by the drag on a
square array of disks (Sec. 4.2, Eq. DiluteTheory).
"""
from __future__ import annotations

import numpy as np

from . import alpert, ewald


def trig_interp(nodes: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Trigonometric interpolant of closed-curve nodes [N_p, 2] at parameters s."""
    n = nodes.shape[0]
    c = np.fft.fft(nodes, axis=0) / n
    k = np.fft.fftfreq(n, d=1.0 / n)
    s = np.atleast_1d(s)
    if n % 2 == 0:
        h = n // 2
        kk = k.copy()
        out = np.real(np.exp(1j * np.outer(s, kk)) @ np.where(np.arange(n)[:, None] == h, 0, c))
        # split the Nyquist coefficient symmetrically: cos(h s) * Re-part
        out += np.real(np.outer(np.cos(h * s), c[h]))
        return out
    return np.real(np.exp(1j * np.outer(s, k)) @ c)


def alpert_body(X: np.ndarray, xi: float, eta: float = 1.0, order: int = 4) -> np.ndarray:
    """M(a) of one body with nodes X [N_p, 2] (not symmetrised), [2N_p, 2N_p]."""
    n_p = X.shape[0]
    v, w, a = alpert.alpert_rule(order)
    q = alpert.interp_points(order)
    h = 2.0 * np.pi / n_p
    Ma = np.zeros((n_p, 2, n_p, 2))
    for i in range(n_p):
        # drop the trapezoidal terms that the end corrections replace
        for o in range(1, a):
            for n in ((i + o) % n_p, (i - o) % n_p):
                Ma[i, :, n, :] -= ewald.g_real(X[i] - X[n], xi, eta)
        for k in range(len(v)):
            for sign in (1.0, -1.0):
                t = sign * v[k]
                y = trig_interp(X, np.array([(i + t) * h]))[0]
                Gk = ewald.g_real(X[i] - y, xi, eta)
                offs, lw = alpert.lagrange_stencil(t, q)
                for o, l in zip(offs, lw):
                    Ma[i, :, (i + o) % n_p, :] += w[k] * l * Gk
    return Ma.reshape(2 * n_p, 2 * n_p)


def node_positions(Q: np.ndarray, ref_nodes: np.ndarray) -> np.ndarray:
    """x_{beta,j} = q_beta + R(theta_beta) gamma_ref(s_j), [N_b, N_p, 2] (Sec. 3.1)."""
    c, s = np.cos(Q[:, 2]), np.sin(Q[:, 2])
    gx, gy = ref_nodes[:, 0], ref_nodes[:, 1]
    x = Q[:, None, 0] + c[:, None] * gx[None, :] - s[:, None] * gy[None, :]
    y = Q[:, None, 1] + s[:, None] * gx[None, :] + c[:, None] * gy[None, :]
    return np.stack([x, y], axis=-1)


def trapezoid_real(Xf: np.ndarray, L: float, xi: float, eta: float = 1.0) -> np.ndarray:
    """M(t) for all nodes Xf [N, 2]: dense [2N, 2N]."""
    n = Xf.shape[0]
    r = (Xf[:, None, :] - Xf[None, :, :]).reshape(-1, 2)
    G = ewald.g_real_periodic(r, L, xi, eta).reshape(n, n, 2, 2)
    G[np.arange(n), np.arange(n)] = 0.0
    return G.transpose(0, 2, 1, 3).reshape(2 * n, 2 * n)


def wave_matrix(Xf: np.ndarray, L: float, xi: float, eta: float = 1.0, modes=None) -> np.ndarray:
    """M(w) for all nodes Xf [N, 2]: dense [2N, 2N] via cos(k.(x_m - x_n)) = C C^T + S S^T."""
    kvec, B = modes if modes is not None else ewald.wave_modes(L, xi)
    ph = Xf @ kvec.T
    C, S = np.cos(ph), np.sin(ph)
    n = Xf.shape[0]
    out = np.empty((n, 2, n, 2))
    for a_ in range(2):
        for b_ in range(2):
            wgt = B[:, a_, b_]
            out[:, a_, :, b_] = (C * wgt) @ C.T + (S * wgt) @ S.T
    return out.reshape(2 * n, 2 * n) / (eta * L * L)


def alpert_all(X: np.ndarray, xi: float, eta: float = 1.0, order: int = 4, sym: bool = True) -> np.ndarray:
    """Block-diagonal M(a) for all bodies X [N_b, N_p, 2], symmetrised if asked."""
    n_b, n_p = X.shape[:2]
    out = np.zeros((2 * n_b * n_p, 2 * n_b * n_p))
    for b in range(n_b):
        Ma = alpert_body(X[b], xi, eta, order)
        if sym:
            Ma = 0.5 * (Ma + Ma.T)
        sl = slice(2 * n_p * b, 2 * n_p * (b + 1))
        out[sl, sl] = Ma
    return out


def single_layer(X: np.ndarray, L: float, xi: float, eta: float = 1.0, order: int = 4,
                 parts: bool = False):
    """Dense M for bodies X [N_b, N_p, 2]; optionally also (M(t), M(a)_sym, M(w))."""
    Xf = X.reshape(-1, 2)
    Mt = trapezoid_real(Xf, L, xi, eta)
    Mw = wave_matrix(Xf, L, xi, eta)
    Ma = alpert_all(X, xi, eta, order, sym=True)
    M = Mt + Ma + Mw
    if parts:
        return M, (Mt, Ma, Mw)
    return M


def real_matrix(X: np.ndarray, L: float, xi: float, eta: float = 1.0, order: int = 4) -> np.ndarray:
    """M(r) = M(t) + M(a)_sym (the near field used by the square root, Sec. 3.3)."""
    Xf = X.reshape(-1, 2)
    return trapezoid_real(Xf, L, xi, eta) + alpert_all(X, xi, eta, order, sym=True)


# --------------------------------------------------------------------------
# Matrix-free forms for sampled checks at sizes the dense matrix cannot reach
# --------------------------------------------------------------------------

def apply_real_rows(X: np.ndarray, mu: np.ndarray, rows, L: float, xi: float, eta: float = 1.0,
                    order: int = 4) -> np.ndarray:
    """(M(t) + M(a)_sym) mu at the listed node rows only; X [N_b, N_p, 2], mu [N, 2]."""
    n_b, n_p = X.shape[:2]
    Xf = X.reshape(-1, 2)
    out = np.zeros((len(rows), 2))
    cache = {}
    src = np.nonzero(np.any(mu != 0.0, axis=1))[0]      # zero forces contribute nothing
    for t, m in enumerate(rows):
        r = Xf[m] - Xf[src]
        G = ewald.g_real_periodic(r, L, xi, eta)
        G[src == m] = 0.0
        out[t] = np.einsum("nab,nb->a", G, mu[src])
        b = m // n_p
        if b not in cache:
            Ma = alpert_body(X[b], xi, eta, order)
            cache[b] = 0.5 * (Ma + Ma.T)
        blk = cache[b][2 * (m - b * n_p):2 * (m - b * n_p) + 2]
        out[t] += blk @ mu[b * n_p:(b + 1) * n_p].reshape(-1)
    return out


def apply_wave_rows(Xf: np.ndarray, mu: np.ndarray, rows, L: float, xi: float, eta: float = 1.0,
                    cut: float = ewald.WAVE_CUT, chunk: int = 8192) -> np.ndarray:
    """M(w) mu at listed rows by the direct non-uniform Fourier sum (sources: nonzero mu only).

    The lattice sum over kappa in [-K, K]^2 with k^2/(4 xi^2) <= cut uses the
    separability e^{-i k.x} = e^{-i k_x x} e^{-i k_y y}: the source transform
    S(kappa) = sum_n mu_n e^{-i k.x_n} is the matrix product Ex^T diag(mu) Ey,
    summed over blocks of ``chunk`` sources so that Ex and Ey stay small.
    """
    kmax = 2.0 * xi * np.sqrt(cut)
    K = int(np.ceil(kmax * L / (2.0 * np.pi)))
    kap = np.arange(-K, K + 1) * (2.0 * np.pi / L)
    src = np.nonzero(np.any(mu != 0.0, axis=1))[0]
    Sx = np.zeros((kap.size, kap.size), dtype=np.complex128)   # [kx, ky]
    Sy = np.zeros_like(Sx)
    for c0 in range(0, src.size, chunk):
        s = src[c0:c0 + chunk]
        Ex = np.exp(-1j * np.outer(Xf[s, 0], kap))            # [S, 2K+1]
        Ey = np.exp(-1j * np.outer(Xf[s, 1], kap))
        Sx += Ex.T @ (mu[s, 0:1] * Ey)
        Sy += Ex.T @ (mu[s, 1:2] * Ey)
    kx, ky = np.meshgrid(kap, kap, indexing="ij")
    k2 = kx * kx + ky * ky
    keep = (k2 > 0) & (k2 / (4.0 * xi * xi) <= cut)
    k2s = np.where(keep, k2, 1.0)
    sc = np.where(keep, ewald.hasimoto(np.sqrt(k2s), xi) / k2s, 0.0)
    Ux = sc * ((1.0 - kx * kx / k2s) * Sx - kx * ky / k2s * Sy)
    Uy = sc * (-kx * ky / k2s * Sx + (1.0 - ky * ky / k2s) * Sy)
    Fx = np.exp(1j * np.outer(Xf[rows, 0], kap))             # [R, 2K+1]
    Fy = np.exp(1j * np.outer(Xf[rows, 1], kap))
    out = np.stack([np.real(np.sum((Fx @ Ux) * Fy, axis=1)),
                    np.real(np.sum((Fx @ Uy) * Fy, axis=1))], axis=1)
    return out / (eta * L * L)
