"""Euler-Maruyama and Adams-Bashforth steps with a random finite difference -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

    Q^{n+1} = Q^n + dt N F + sqrt(2 kT dt) N^1/2 W
              + dt kT/delta [ N(Q + delta/2 W~) W~ - N(Q - delta/2 W~) W~ ]   (Sec. 4.4, Eq. EM-RFD)

The first two terms come from one saddle solve with right-hand side
[slip; F] where slip = sqrt(2kT/dt) M^1/2 W; the drift from two solves with
force W~ and no slip at the displaced configurations.

    Q^{n+1} = Q^n + dt (3/2 N^n F^n - 1/2 N^{n-1} F^{n-1}) + sqrt(2 kT dt) N^1/2 W
              + dt kT/delta [ N(Q + delta/2 W~) W~ - N(Q - delta/2 W~) W~ ]   (Sec. 4.4, Eq. AB2-RFD)

takes four solves: N^n F^n alone, the slip alone (force zero), and the pair; the
previous step's N F is carried over, and the first step uses N^n F^n for both
(the Euler step).  The RFD pair may be solved at a looser tolerance than the rest
(Sec. 4.4.2); the oracle's dense solves are exact either way.

Parity: pinned by what Sec. 4.4 fixes about the step: the RFD term's expectation
over W~ equals dt kT (d/dQ . N) (checked against central differences of this
package's N), at fixed W~ it tends to dt kT (D_W~ N) W~ as delta -> 0 at second
order, and the deterministic part is dt N F.  ``em_no_rfd_step`` (Eq. EM-noRFD) is
pinned by reducing to dt N F without noise and to ``em_rfd_step`` at W~ = 0 with it.
``ab2_rfd_step`` is pinned by the
order of its deterministic part: on a two-body spring problem at kT = 0 its
trajectory converges at second order in dt where the Euler step converges at first.
"""
from __future__ import annotations

import numpy as np

from . import brownian, saddle, singlelayer


def mobility_velocity(Q, ref_nodes, L, xi, F, slip_vec=None, eta=1.0, order=4):
    X = singlelayer.node_positions(Q, ref_nodes)
    M = singlelayer.single_layer(X, L, xi, eta, order)
    K = saddle.k_matrix(X, Q)
    _, U = saddle.solve_saddle(M, K, F.reshape(-1), None if slip_vec is None else slip_vec.reshape(-1))
    return U.reshape(-1, 3)


def em_rfd_step(Q, ref_nodes, L, xi, F, dt, kT, delta, W_r, Z, W_tilde, eta=1.0, order=4):
    X = singlelayer.node_positions(Q, ref_nodes)
    sl = brownian.slip(X, Q, ref_nodes, L, xi, kT, dt, W_r, Z, eta, order)
    U = mobility_velocity(Q, ref_nodes, L, xi, F, sl, eta, order)
    Wt = W_tilde.reshape(-1, 3)
    Up = mobility_velocity(Q + 0.5 * delta * Wt, ref_nodes, L, xi, Wt, None, eta, order)
    Um = mobility_velocity(Q - 0.5 * delta * Wt, ref_nodes, L, xi, Wt, None, eta, order)
    return Q + dt * U + dt * kT / delta * (Up - Um)


def em_no_rfd_step(Q, ref_nodes, L, xi, F, dt, kT, W_r, Z, eta=1.0, order=4):
    """The biased step of Sec. 4.4.1 (Eq. EM-noRFD, with the force term kept): Eq. EM-RFD
    without its random finite difference, Q + dt N F + sqrt(2 kT dt) N^1/2 W from one
    saddle solve with right-hand side [slip; F]."""
    X = singlelayer.node_positions(Q, ref_nodes)
    sl = brownian.slip(X, Q, ref_nodes, L, xi, kT, dt, W_r, Z, eta, order)
    return Q + dt * mobility_velocity(Q, ref_nodes, L, xi, F, sl, eta, order)


def ab2_rfd_step(Q, ref_nodes, L, xi, F, NF_prev, dt, kT, delta, W_r, Z, W_tilde, eta=1.0, order=4):
    """One step of Eq. AB2-RFD; returns (Q^{n+1}, N^n F^n).  NF_prev = None: first step."""
    X = singlelayer.node_positions(Q, ref_nodes)
    sl = brownian.slip(X, Q, ref_nodes, L, xi, kT, dt, W_r, Z, eta, order)
    U_noise = mobility_velocity(Q, ref_nodes, L, xi, np.zeros_like(F), sl, eta, order)
    NF = mobility_velocity(Q, ref_nodes, L, xi, F, None, eta, order)
    det = NF if NF_prev is None else 1.5 * NF - 0.5 * NF_prev
    Wt = W_tilde.reshape(-1, 3)
    Up = mobility_velocity(Q + 0.5 * delta * Wt, ref_nodes, L, xi, Wt, None, eta, order)
    Um = mobility_velocity(Q - 0.5 * delta * Wt, ref_nodes, L, xi, Wt, None, eta, order)
    return Q + dt * det + dt * U_noise + dt * kT / delta * (Up - Um), NF
