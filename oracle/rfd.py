"""Euler-Maruyama step with a random finite difference -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

    Q^{n+1} = Q^n + dt N F + sqrt(2 kT dt) N^1/2 W
              + dt kT/delta [ N(Q + delta/2 W~) W~ - N(Q - delta/2 W~) W~ ]   (Sec. 4.4, Eq. EM-RFD)

The first two terms come from one saddle solve with right-hand side
[slip; F] where slip = sqrt(2kT/dt) M^1/2 W; the drift from two solves with
force W~ and no slip at the displaced configurations.

Parity: pinned by what Sec. 4.4 fixes about the step: the RFD term's expectation
over W~ equals dt kT (d/dQ . N) (checked against central differences of this
package's N), at fixed W~ it tends to dt kT (D_W~ N) W~ as delta -> 0 at second
order, and the deterministic part is dt N F.
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
