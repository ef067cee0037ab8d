"""Free diffusion of one four-fold starfish in the periodic unit cell -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 4.4.1: in a square periodic lattice the body mobility of a four-fold starfish is
diagonal, N = diag(N_xx, N_yy, N_thth) with N_xx = N_yy, and depends on the orientation
theta alone, with period pi/2.  Under free diffusion (no force or torque):

* the Euler-Maruyama step with the random finite difference (Eq. EM-RFD) samples the
  Gibbs-Boltzmann distribution, uniform in theta;
* the step without it (Eq. EM-noRFD) is consistent with an Ito equation that misses
  the stochastic drift kT dN_thth/dtheta, and samples the biased distribution
  P~(theta) proportional to 1 / N_thth(theta) (Eq. biased-dist);
* the translational mean square displacement grows as 4 kT <N_xx> t, the average
  taken over the scheme's own equilibrium distribution.

``mobility_table`` evaluates N(theta) with the dense first-kind oracle at equispaced
orientations over one period; ``equilibrium_averages`` averages the statistics over
either distribution by the trapezoidal rule on those periodic samples (spectrally
accurate for the smooth periodic N).  ``theta_walk`` is a plain Monte Carlo of the
orientation alone, with or without the drift term, that pins the two stationary
distributions independently of their derivation.
"""
from __future__ import annotations

import math

import numpy as np

from . import saddle, singlelayer


def mobility_table(ref_nodes, L, n_theta, xi, order=4, eta=1.0, centre=(0.5, 0.5)):
    """theta_j = j (pi/2) / n_theta, j < n_theta, and N(theta_j) [n_theta, 3, 3] of one body
    with reference nodes ref_nodes at centre (in units of L) in the periodic cell of side L."""
    th = np.arange(n_theta) * (0.5 * math.pi / n_theta)
    out = np.zeros((n_theta, 3, 3))
    for j, t in enumerate(th):
        Q = np.array([[centre[0] * L, centre[1] * L, t]])
        X = singlelayer.node_positions(Q, ref_nodes)
        M = singlelayer.single_layer(X, L, xi, eta, order)
        K = saddle.k_matrix(X, Q)
        out[j] = saddle.mobility(M, K)
    return th, out


def equilibrium_averages(N_table):
    """Averages of cos 4 theta, N_xx (the mean of N_xx and N_yy) and N_thth over the uniform
    and the biased (proportional to 1 / N_thth) distribution, from the periodic table."""
    n = N_table.shape[0]
    th = np.arange(n) * (0.5 * math.pi / n)
    nxx = 0.5 * (N_table[:, 0, 0] + N_table[:, 1, 1])
    nthth = N_table[:, 2, 2]
    stats = {"cos4": np.cos(4.0 * th), "nxx": nxx, "nthth": nthth}
    w_u = np.full(n, 1.0 / n)
    w_b = (1.0 / nthth) / np.sum(1.0 / nthth)
    return {name: {k: float(w @ v) for k, v in stats.items()} for name, w in (("uniform", w_u), ("biased", w_b))}


def periodic_interpolant(values):
    """The trigonometric interpolant of samples at theta_j = j (pi/2)/n over the period pi/2,
    returned as f(theta) and its derivative f'(theta)."""
    v = np.asarray(values, dtype=float)
    n = v.size
    c = np.fft.rfft(v) / n
    k = np.arange(c.size)
    if n % 2 == 0:
        c[-1] *= 0.5          # the Nyquist term split between +k and -k
    w = 4.0 * k               # angular frequency in theta (period pi/2)

    def f(theta):
        t = np.asarray(theta, dtype=float)[..., None]
        return np.real(c[0]) + 2.0 * np.sum(np.real(c[1:] * np.exp(1j * w[1:] * t)), axis=-1)

    def fp(theta):
        t = np.asarray(theta, dtype=float)[..., None]
        return 2.0 * np.sum(np.real(1j * w[1:] * c[1:] * np.exp(1j * w[1:] * t)), axis=-1)

    return f, fp


def theta_walk(nthth_values, kT, dt, n_steps, n_walkers, seed, drift=True, burn=0):
    """Euler-Maruyama walk of the orientation alone:
        theta += [kT N_thth'(theta) dt if drift] + sqrt(2 kT N_thth(theta) dt) w,
    the rotational part of Eqs. EM-RFD (drift = the expectation of its random finite
    difference) and EM-noRFD (drift = False).  Walkers start uniform on [0, pi/2); returns
    the mean of cos 4 theta over the steps after ``burn`` and over the walkers, and the
    standard error of that mean from the walkers' own means."""
    f, fp = periodic_interpolant(nthth_values)
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 0.5 * math.pi, n_walkers)
    acc = np.zeros(n_walkers)
    cnt = 0
    for s in range(n_steps):
        n_th = f(th)
        step = math.sqrt(2.0 * kT * dt) * np.sqrt(n_th) * rng.standard_normal(n_walkers)
        if drift:
            step += kT * fp(th) * dt
        th = th + step
        if s >= burn:
            acc += np.cos(4.0 * th)
            cnt += 1
    m = acc / cnt
    return float(m.mean()), float(m.std(ddof=1) / math.sqrt(n_walkers))
