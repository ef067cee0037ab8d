"""Completed second-kind (double-layer) mobility solver -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

App. B's formulation (Eqs. DLrepresentation, second-kind-formulation, q2torque): the
exterior flow is a double layer of density phi on every body plus a Stokeslet (force f)
and a rotlet (torque tau) at each tracking point q, and on each body

    u + omega (x - q)^perp = 1/2 phi(x) + (D phi)(x) + sum_b [G(x - q_b) f_b + R(x - q_b) tau_b]
    u = (1/|Gamma|) int phi dS,        omega = (1/W) int phi . (x - q)^perp dS,
    W = int |x - q|^2 dS,

with the free-space kernels (unit viscosity, prefactor 1/(4 pi))
G_jl = -delta_jl log r + x_j x_l / r^2,  T_jlm = -4 x_j x_l x_m / r^4,  R_j = x^perp_j / r^2,
all periodised with the Hasimoto split of App. B:

* Stokeslet: the first-kind oracle's G^(r) + G^(w) (``oracle.ewald``).
* Rotlet:    R^(r)(x) = x^perp/r^2 (1 - xi^2 r^2) e^{-xi^2 r^2} over the images, plus
             (1/V) sum_{k != 0} 2 pi k^perp H^(k)/k^2 sin(k . x), all times 1/(4 pi).
* Stresslet: T^(r)_jlm = [-4 x_j x_l x_m / r^4 (1 + xi^2 r^2) + 2 xi^2 (delta_lm x_j +
             delta_mj x_l)] e^{-xi^2 r^2} over the images, plus the wave part
             (1/V) sum_k T^(w)_jlm(k) S_lm sin(k . (x_t - x_s)) with
             T^(w)_jlm = -(4 pi / k^4) [(1 + k^2/4xi^2)(k^2 (k_j delta_lm + k_l delta_mj)
             - 2 k_j k_l k_m) + k^2 k_m delta_jl] e^{-k^2/4xi^2}, the mean-flow term
             T^(0)_jlm(x_s) = (4 pi / V) delta_lm (x_s)_j, and the self term of the
             trapezoidal rule, all times 1/(4 pi); S_lm = phi_l n_m Delta s.

Discretisation: the trapezoidal rule at the first-kind nodes (the stresslet is smooth
on a smooth curve, so the rule is spectrally accurate, App. B); tangent, outward normal,
arc-length weight |gamma'| 2 pi / N_p and curvature from the trigonometric
interpolant of the reference nodes (spectral differentiation, rotated per body).  The
dense system [phi; U] is solved by LU for unit forces and torques, giving N.

Readings (where App. B is garbled or silent):
* n in S_lm is the normal pointing into the body (out of the fluid domain): with
  r = x_t - x_s and this normal the double layer's limit from the fluid is
  1/2 phi + (D phi)^PV, as the formulation is written (for the outward normal it would
  be -1/2 phi + (D phi)^PV);
* the rotlet's wave sum carries 1/(4 pi eta V): its printed 1/(eta V) omits the 1/(4 pi)
  that its real part and the rotlet itself carry (xi-independence of the sum fixes it);
* T^(0) is evaluated at the source position, as printed: the term
  (1/V) sum_s x_s (phi_s . n_s) Delta s is the constant that makes the second-kind
  velocities follow the first-kind convention (zero mean velocity over the cell, body
  interiors moving rigidly).  It is origin-independent at the solution, where each
  body's flux sum phi . n Delta s vanishes;
* the self term is the limit of the real-space stresslet along the curve, -2 kappa
  t_j t_l for this normal (kappa > 0 on convex arcs), weighted by the node's Delta s:
  -(1/(4 pi)) 2 kappa (t t^T) phi Delta s (the printed 2 pi kappa (t t^T) phi lacks the
  weight);
* x^perp = (-x_2, x_1) and k^perp = (-k_2, k_1), the convention of the first-kind K
  (omega (x - q)^perp is a counter-clockwise rotation for omega > 0); App. B writes
  x^perp = (x_2, -x_1), which flips the sign of both omega and tau together;
* the completion Stokeslets and rotlets of all bodies act on every body, and the
  double layer of every body enters each body's equation (App. B writes one body).

Parity: pinned by the xi-independence of the periodic rotlet and stresslet sums, the
constant-density identity of the double layer (D 1 = -1/2 on a closed curve, free
space), spectral convergence in N_p, agreement with the first-kind oracle's N at high
resolution (an independent formulation), and the Sangani-Acrivos expansion for a dilute
square array of disks (Sec. 4.1, Eq. DiluteTheory).
"""
from __future__ import annotations

import numpy as np

from . import ewald, singlelayer


def perp(v):
    """v^perp = (-v_2, v_1) along the last axis."""
    v = np.asarray(v, dtype=np.float64)
    return np.stack([-v[..., 1], v[..., 0]], axis=-1)


# ---------------------------------------------------------------------------
# curve geometry
# ---------------------------------------------------------------------------
def curve_geometry(ref_nodes: np.ndarray):
    """Unit tangent, outward unit normal, |gamma'| and curvature at the reference nodes
    (counter-clockwise curve sampled at s_j = 2 pi j / N_p), by spectral differentiation
    of the trigonometric interpolant."""
    n_p = ref_nodes.shape[0]
    c = np.fft.fft(ref_nodes, axis=0)
    k = np.fft.fftfreq(n_p, d=1.0 / n_p)
    if n_p % 2 == 0:
        k[n_p // 2] = 0.0          # the Nyquist term of a real interpolant has zero derivative
    d1 = np.real(np.fft.ifft(1j * k[:, None] * c, axis=0))
    d2 = np.real(np.fft.ifft(-(k[:, None] ** 2) * c, axis=0))
    speed = np.linalg.norm(d1, axis=1)
    tang = d1 / speed[:, None]
    normal = np.stack([tang[:, 1], -tang[:, 0]], axis=1)      # tangent turned clockwise: outward
    kappa = (d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]) / speed ** 3
    return tang, normal, speed, kappa


def body_geometry(Q: np.ndarray, ref_nodes: np.ndarray):
    """Per node of every body: position, unit tangent, outward normal, weight Delta s,
    curvature.  Shapes [N_b, N_p, 2] (or [N_b, N_p])."""
    X = singlelayer.node_positions(Q, ref_nodes)
    t0, n0, speed, kappa = curve_geometry(ref_nodes)
    n_b, n_p = X.shape[:2]
    T = np.empty_like(X)
    Nrm = np.empty_like(X)
    for b in range(n_b):
        c, s = np.cos(Q[b, 2]), np.sin(Q[b, 2])
        R = np.array([[c, -s], [s, c]])
        T[b] = t0 @ R.T
        Nrm[b] = n0 @ R.T
    ds = np.broadcast_to(speed * (2.0 * np.pi / n_p), (n_b, n_p)).copy()
    kap = np.broadcast_to(kappa, (n_b, n_p)).copy()
    return X, T, Nrm, ds, kap


# ---------------------------------------------------------------------------
# periodic rotlet
# ---------------------------------------------------------------------------
def rotlet_real(r, xi):
    """R^(r)(r) / (4 pi) at separations r [..., 2] (r != 0) -> [..., 2]."""
    r = np.asarray(r, dtype=np.float64)
    r2 = np.sum(r * r, axis=-1)
    z = xi * xi * r2
    return perp(r) * ((1.0 - z) * np.exp(-z) / r2)[..., None] / (4.0 * np.pi)


def rotlet_wave_vectors(kvec, xi):
    """2 pi k^perp H^(k) / k^2 for each row of kvec -> [K, 2]."""
    k2 = np.sum(kvec * kvec, axis=1)
    return 2.0 * np.pi * perp(kvec) * (ewald.hasimoto(np.sqrt(k2), xi) / k2)[:, None]


def rotlet_periodic(r, L, xi, modes=None):
    """The periodic rotlet sum_p R(r + pL) / (4 pi) at r [P, 2] (r != 0 mod L) -> [P, 2]."""
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    cut = ewald.real_cutoff(xi)
    out = np.zeros_like(r)
    for s in ewald.image_shifts(L, cut):
        rr = r + s
        d2 = np.sum(rr * rr, axis=1)
        m = (d2 < cut * cut) & (d2 > 0.0)
        if np.any(m):
            out[m] += rotlet_real(rr[m], xi)
    kvec = modes[0] if modes is not None else ewald.wave_modes(L, xi)[0]
    Rw = rotlet_wave_vectors(kvec, xi)
    out += np.sin(r @ kvec.T) @ Rw / (4.0 * np.pi * L * L)
    return out


# ---------------------------------------------------------------------------
# periodic stresslet
# ---------------------------------------------------------------------------
def stresslet_real(r, xi):
    """T^(r)_jlm(r) / (4 pi) at separations r [..., 2] (r != 0) -> [..., 2, 2, 2] (j, l, m)."""
    r = np.asarray(r, dtype=np.float64)
    r2 = np.sum(r * r, axis=-1)
    z = xi * xi * r2
    e = np.exp(-z)
    I = np.eye(2)
    xxx = np.einsum("...j,...l,...m->...jlm", r, r, r)
    out = -4.0 * xxx * ((1.0 + z) * e / (r2 * r2))[..., None, None, None]
    a = 2.0 * xi * xi * e
    out += a[..., None, None, None] * (np.einsum("lm,...j->...jlm", I, r) + np.einsum("mj,...l->...jlm", I, r))
    return out / (4.0 * np.pi)


def stresslet_wave_tensor(kvec, xi):
    """T^(w)_jlm(k) for each row of kvec -> [K, 2, 2, 2]."""
    k2 = np.sum(kvec * kvec, axis=1)
    I = np.eye(2)
    h = 1.0 + k2 / (4.0 * xi * xi)
    e = np.exp(-k2 / (4.0 * xi * xi))
    kkk = np.einsum("kj,kl,km->kjlm", kvec, kvec, kvec)
    a = (k2[:, None, None, None] * (np.einsum("kj,lm->kjlm", kvec, I) + np.einsum("kl,mj->kjlm", kvec, I))
         - 2.0 * kkk)
    b = k2[:, None, None, None] * np.einsum("km,jl->kjlm", kvec, I)
    return -(4.0 * np.pi / (k2 * k2))[:, None, None, None] * (h[:, None, None, None] * a + b) * e[:, None, None, None]


def stresslet_periodic(r, L, xi, modes=None):
    """sum_p T^(r)(r + pL) + (1/V) sum_k T^(w)(k) sin(k . r), over 4 pi, at r [P, 2]
    (r != 0 mod L) -> [P, 2, 2, 2]: the periodic stresslet without its mean-flow term."""
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    cut = ewald.real_cutoff(xi)
    out = np.zeros(r.shape[:1] + (2, 2, 2))
    for s in ewald.image_shifts(L, cut):
        rr = r + s
        d2 = np.sum(rr * rr, axis=1)
        m = (d2 < cut * cut) & (d2 > 0.0)
        if np.any(m):
            out[m] += stresslet_real(rr[m], xi)
    kvec = modes[0] if modes is not None else ewald.wave_modes(L, xi)[0]
    Tw = stresslet_wave_tensor(kvec, xi)
    out += np.einsum("pk,kjlm->pjlm", np.sin(r @ kvec.T), Tw) / (4.0 * np.pi * L * L)
    return out


# ---------------------------------------------------------------------------
# dense operators
# ---------------------------------------------------------------------------
def double_layer_matrix(Xf, Nf, dsf, kapf, Tf, L, xi, modes=None):
    """D [2N, 2N]: (D phi) at the nodes (principal value) for nodes Xf [N, 2] with normals
    Nf pointing into the bodies, weights dsf, curvatures kapf (> 0 on convex arcs) and
    tangents Tf."""
    N = Xf.shape[0]
    V = L * L
    kvec = modes[0] if modes is not None else ewald.wave_modes(L, xi)[0]
    # real space over images, s != t at the zero image
    cut = ewald.real_cutoff(xi)
    Kr = np.zeros((N, N, 2, 2))                     # [t, s, j, l]: sum_m T_jlm n_m(s) ds(s)
    Rts = Xf[:, None, :] - Xf[None, :, :]
    for sh in ewald.image_shifts(L, cut):
        rr = Rts + sh
        d2 = np.sum(rr * rr, axis=-1)
        m = (d2 < cut * cut) & (d2 > 0.0)
        if np.any(m):
            T = stresslet_real(rr[m], xi)           # [P, j, l, m]
            t_idx, s_idx = np.nonzero(m)
            Kr[t_idx, s_idx] += np.einsum("pjlm,pm->pjl", T, Nf[s_idx]) * dsf[s_idx][:, None, None]
    # wave space: sin(k.(x_t - x_s)) = sin(k x_t) cos(k x_s) - cos(k x_t) sin(k x_s)
    Tw = stresslet_wave_tensor(kvec, xi)            # [K, j, l, m]
    ph = Xf @ kvec.T
    Sx, Cx = np.sin(ph), np.cos(ph)
    for j in range(2):
        for l in range(2):
            for mm in range(2):
                w = Tw[:, j, l, mm] / (4.0 * np.pi * V)
                blk = (Sx * w) @ Cx.T - (Cx * w) @ Sx.T            # [t, s]
                Kr[:, :, j, l] += blk * (Nf[:, mm] * dsf)[None, :]
    # mean-flow term (1/V) (x_s)_j (phi_s . n_s) ds_s, the same at every target
    Kr += (Xf[None, :, :, None] * (Nf * dsf[:, None])[None, :, None, :]) / V
    # self term -(1/(4 pi)) 2 kappa t t^T ds
    for t in range(N):
        Kr[t, t] -= (2.0 * kapf[t] * np.outer(Tf[t], Tf[t]) * dsf[t]) / (4.0 * np.pi)
    return Kr.transpose(0, 2, 1, 3).reshape(2 * N, 2 * N)


def completion_matrix(Xf, Q, L, xi, modes=None):
    """C [2N, 3 N_b]: the periodic Stokeslet (f) and rotlet (tau) of every tracking point at
    every node."""
    N = Xf.shape[0]
    n_b = Q.shape[0]
    C = np.zeros((2 * N, 3 * n_b))
    for b in range(n_b):
        r = Xf - Q[b, :2]
        C[:, 3 * b:3 * b + 2] = ewald.g_periodic(r, L, xi, modes=modes).reshape(2 * N, 2)
        C[:, 3 * b + 2] = rotlet_periodic(r, L, xi, modes=modes).reshape(-1)
    return C


def second_kind_matrix(Q, ref_nodes, L, xi, modes=None):
    """The dense system A [phi; U] = B F of the completed second-kind formulation, returned
    as (A, B) with A [(2N + 3N_b) x (2N + 3N_b)], B [(2N + 3N_b) x 3N_b]."""
    X, T, Nrm, ds, kap = body_geometry(Q, ref_nodes)
    n_b, n_p = X.shape[:2]
    N = n_b * n_p
    Xf, Tf, Nf, dsf, kapf = X.reshape(-1, 2), T.reshape(-1, 2), Nrm.reshape(-1, 2), ds.reshape(-1), kap.reshape(-1)
    if modes is None:
        modes = ewald.wave_modes(L, xi)
    D = double_layer_matrix(Xf, -Nf, dsf, kapf, Tf, L, xi, modes)     # normals into the bodies
    C = completion_matrix(Xf, Q, L, xi, modes)
    n = 2 * N + 3 * n_b
    A = np.zeros((n, n))
    B = np.zeros((n, 3 * n_b))
    # node rows: K U - 1/2 phi - D phi = C F
    A[:2 * N, :2 * N] = -0.5 * np.eye(2 * N) - D
    from .saddle import k_matrix
    A[:2 * N, 2 * N:] = k_matrix(X, Q)
    B[:2 * N] = C
    # closure rows: |Gamma| u - sum phi ds = 0, W omega - sum phi . (x - q)^perp ds = 0
    for b in range(n_b):
        sl = slice(b * n_p, (b + 1) * n_p)
        rel = X[b] - Q[b, :2]
        row = 2 * N + 3 * b
        A[row, 2 * N + 3 * b] = np.sum(ds[b])
        A[row + 1, 2 * N + 3 * b + 1] = np.sum(ds[b])
        A[row + 2, 2 * N + 3 * b + 2] = np.sum(np.sum(rel * rel, axis=1) * ds[b])
        for j, i in enumerate(range(sl.start, sl.stop)):
            A[row, 2 * i] = -ds[b, j]
            A[row + 1, 2 * i + 1] = -ds[b, j]
            pv = perp(rel[j])
            A[row + 2, 2 * i] = -pv[0] * ds[b, j]
            A[row + 2, 2 * i + 1] = -pv[1] * ds[b, j]
    return A, B


def mobility(Q, ref_nodes, L, xi, modes=None, want_phi=False):
    """N [3N_b, 3N_b] from the completed second-kind formulation (U = N F); optionally
    also the densities phi [2N, 3N_b] of the unit forces and torques."""
    A, B = second_kind_matrix(Q, ref_nodes, L, xi, modes)
    n3 = 3 * Q.shape[0]
    sol = np.linalg.solve(A, B)
    Nmat = sol[-n3:]
    return (Nmat, sol[:-n3]) if want_phi else Nmat
