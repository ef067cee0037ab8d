"""Hasimoto split of the 2D periodic Stokeslet -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``hasimoto``    H^(k; xi) = (1 + k^2/4xi^2) exp(-k^2/4xi^2)         (Sec. 3.2, Eq. HasimotoFunction)
* ``g_real``      G^(r)(r) = 1/(4 pi eta) [E1(xi^2 r^2)/2 I + (r r^T/r^2 - I) exp(-xi^2 r^2)]
                                                                       (Sec. 3.2, Eqs. real-space-kernel, expint)
* ``wave_modes``  the lattice k = 2 pi kappa / L, kappa != 0, with the tensor
                  B(k) = H^(k)/k^2 (I - k^ k^^T)                       (Sec. 3.2, Eq. wave-space-kernel)
* ``g_wave``      G^(w)(r) = 1/(eta V) sum_{k != 0} B(k) cos(k . r)   (Sec. 3.2, Eq. wave-space-kernel)
* ``g_real_periodic`` the real-space part summed over periodic images.

The exponential integral comes from ``scipy.special.exp1`` (a library
primitive).  The wave-space sum is a direct lattice sum truncated where
k^2/(4 xi^2) > 50, i.e. terms below e^-50 of the leading ones.

Parity: pinned by the xi-independence of G^(r) + G^(w) (Sec. 3.2: the split
does not change the periodic Stokeslet), by 0 <= H^ <= 1 and the positive
semi-definiteness of the wave-space matrix (Sec. 3.2 and 3.3), and by the
small-r limit of G^(r) against the free-space 2D Stokeslet
(-log r I + r r^T / r^2)/(4 pi eta).
"""
from __future__ import annotations

import numpy as np
from scipy.special import exp1

WAVE_CUT = 50.0  # keep modes with k^2 / (4 xi^2) <= WAVE_CUT


def hasimoto(k, xi):
    z = np.asarray(k, dtype=np.float64) ** 2 / (4.0 * xi * xi)
    return (1.0 + z) * np.exp(-z)


def g_real(r, xi, eta=1.0):
    """Real-space kernel at separation vectors r [..., 2] -> [..., 2, 2]; r != 0."""
    r = np.asarray(r, dtype=np.float64)
    r2 = np.sum(r * r, axis=-1)
    z = xi * xi * r2
    e = np.exp(-z)
    a = 0.5 * exp1(z) - e                                   # coefficient of I
    b = e / r2                                              # coefficient of r r^T
    out = np.empty(r.shape[:-1] + (2, 2))
    out[..., 0, 0] = a + b * r[..., 0] * r[..., 0]
    out[..., 1, 1] = a + b * r[..., 1] * r[..., 1]
    out[..., 0, 1] = b * r[..., 0] * r[..., 1]
    out[..., 1, 0] = out[..., 0, 1]
    return out / (4.0 * np.pi * eta)


def wave_modes(L, xi, cut=WAVE_CUT):
    """All lattice wavevectors k != 0 with k^2/(4 xi^2) <= cut, and B(k) [K, 2, 2]."""
    kmax = 2.0 * xi * np.sqrt(cut)
    nmax = int(np.ceil(kmax * L / (2.0 * np.pi)))
    ks = np.arange(-nmax, nmax + 1)
    kx, ky = np.meshgrid(ks, ks, indexing="ij")
    kx = kx.ravel() * (2.0 * np.pi / L)
    ky = ky.ravel() * (2.0 * np.pi / L)
    k2 = kx * kx + ky * ky
    keep = (k2 > 0) & (k2 / (4.0 * xi * xi) <= cut)
    kx, ky, k2 = kx[keep], ky[keep], k2[keep]
    kvec = np.stack([kx, ky], axis=1)
    return kvec, wave_tensor(kvec, xi)


def wave_tensor(kvec, xi):
    """B(k) = H^(k)/k^2 (I - k^ k^^T) for each row of kvec."""
    kx, ky = kvec[:, 0], kvec[:, 1]
    k2 = kx * kx + ky * ky
    s = hasimoto(np.sqrt(k2), xi) / k2
    B = np.empty((kvec.shape[0], 2, 2))
    B[:, 0, 0] = s * (1.0 - kx * kx / k2)
    B[:, 1, 1] = s * (1.0 - ky * ky / k2)
    B[:, 0, 1] = -s * kx * ky / k2
    B[:, 1, 0] = B[:, 0, 1]
    return B


def g_wave(r, L, xi, eta=1.0, modes=None):
    """Wave-space kernel at separations r [P, 2] -> [P, 2, 2] (r = 0 allowed)."""
    kvec, B = modes if modes is not None else wave_modes(L, xi)
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    c = np.cos(r @ kvec.T)                                   # [P, K]
    return np.einsum("pk,kab->pab", c, B) / (eta * L * L)


def image_shifts(L, cutoff):
    n = int(np.ceil(cutoff / L)) + 1
    s = np.arange(-n, n + 1)
    px, py = np.meshgrid(s, s, indexing="ij")
    return np.stack([px.ravel(), py.ravel()], axis=1) * L


def real_cutoff(xi):
    """exp(-xi^2 r^2) < e^-64 beyond this radius."""
    return 8.0 / xi


def g_real_periodic(r, L, xi, eta=1.0, exclude_origin=False):
    """sum_p G^(r)(r + pL) over images within the real-space cutoff; r [P, 2]."""
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    cut = real_cutoff(xi)
    out = np.zeros(r.shape[:1] + (2, 2))
    for s in image_shifts(L, cut):
        rr = r + s
        d2 = np.sum(rr * rr, axis=1)
        m = (d2 < cut * cut) & (d2 > 0.0)
        if exclude_origin:
            m &= d2 > 0.0
        if np.any(m):
            out[m] += g_real(rr[m], xi, eta)
    return out


def g_periodic(r, L, xi, eta=1.0, modes=None):
    """The full periodic Stokeslet G = G^(r) + G^(w) at r != 0 (mod L)."""
    return g_real_periodic(r, L, xi, eta) + g_wave(r, L, xi, eta, modes)
