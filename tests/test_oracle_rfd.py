"""Pins for the oracle's random-finite-difference steps (Sec. 4.4, Eqs. EM-RFD, AB2-RFD).

What the paper fixes about the step:

* Its deterministic part is dt N F, and its noise part sqrt(2 kT dt) N^1/2 W enters
  through the slip of the same saddle solve (Sec. 3.1, Eq. discreteParticleVelocity).
* Its last term, (dt kT / delta) [N(Q + delta/2 W~) - N(Q - delta/2 W~)] W~, has the
  expectation dt kT (d/dQ . N)(Q) + O(delta^2) over W~ ~ N(0, I) (Sec. 4.4: the
  RFD approximates the stochastic drift; Sec. 2, Eq. BDeqns).  Because the term is,
  to O(delta^2), the quadratic form W~ -> (D_W~ N) W~, its expectation is the sum of
  that form over the unit vectors e_j: sum_j (d_j N)[:, j], the divergence.
* At fixed W~, the term tends to dt kT (D_W~ N) W~ as delta -> 0.
* The Adams-Bashforth step's deterministic part, dt (3/2 N^n F^n - 1/2 N^{n-1} F^{n-1}),
  is second-order accurate where the Euler step's dt N F is first-order.

The expected values come from central differences (with Richardson extrapolation)
of the oracle's mobility N, computed column by column from dense saddle solves at
displaced configurations with steps unrelated to delta.  A dropped factor 1/2 in
the displacement, a swapped sign of the difference, a missing kT or dt, or a force
applied on one side only each fail these tests.
"""
import math

import numpy as np
import pytest

import fbim_synth
from oracle import rfd, saddle, singlelayer

L = 3.0
N_P = 32
XI = math.sqrt(math.log(100.0 / 1e-12)) / (L / 4)


def _case():
    ref = fbim_synth.starfish_ref_nodes(N_P)
    # two starfish close enough that N depends strongly on their relative position
    Q = np.array([[1.0, 1.2, 0.3], [2.25, 1.55, 1.7]])
    return ref, Q


def _mobility(Q, ref):
    X = singlelayer.node_positions(Q, ref)
    M = singlelayer.single_layer(X, L, XI)
    return saddle.mobility(M, saddle.k_matrix(X, Q))


def _directional_derivative(Q, ref, w, h):
    """(D_w N)(Q) by a Richardson-extrapolated central difference with step h."""
    def cd(s):
        Qp = Q + s * w.reshape(-1, 3)
        Qm = Q - s * w.reshape(-1, 3)
        return (_mobility(Qp, ref) - _mobility(Qm, ref)) / (2.0 * s)
    return (4.0 * cd(0.5 * h) - cd(h)) / 3.0


def _zero_noise(n, M=16):
    return np.zeros((n, 2)), np.zeros((M, M, 2, 2))


def _step(Q, ref, F, dt, kT, delta, Wt):
    W_r, Z = _zero_noise(Q.shape[0] * N_P)
    return rfd.em_rfd_step(Q, ref, L, XI, F, dt, kT, delta, W_r, Z, Wt)


def test_rfd_drift_mean_is_kT_times_divergence_of_N():
    ref, Q = _case()
    n = Q.size
    dt, kT, delta = 0.37, 1.9, 2e-4
    F = np.zeros_like(Q)
    # expectation over W~ of the drift = sum over unit vectors e_j of the drift at W~ = e_j
    drift = np.zeros(n)
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        drift += (_step(Q, ref, F, dt, kT, delta, e) - Q).reshape(-1)
    div = np.zeros(n)
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        div += _directional_derivative(Q, ref, e, 2e-3)[:, j]
    expect = dt * kT * div
    # the divergence is not negligible here: the test is not vacuous
    assert np.max(np.abs(expect)) > 1e-3 * dt * kT * np.max(np.abs(_mobility(Q, ref))) / L
    err = np.max(np.abs(drift - expect)) / np.max(np.abs(expect))
    print(f"RFD mean drift vs kT div N: rel err {err:.2e}")
    assert err < 1e-5


def test_rfd_term_tends_to_directional_derivative_at_fixed_wtilde():
    ref, Q = _case()
    Wt = np.random.default_rng(8).standard_normal(Q.size)
    dt, kT = 0.5, 1.0
    F = np.zeros_like(Q)
    dN = _directional_derivative(Q, ref, Wt, 2e-3)
    expect = dt * kT * dN @ Wt
    errs = []
    for delta in (4e-2, 2e-2):
        got = (_step(Q, ref, F, dt, kT, delta, Wt) - Q).reshape(-1)
        errs.append(np.max(np.abs(got - expect)) / np.max(np.abs(expect)))
    print(f"RFD term vs (D_W~ N) W~: rel err {errs}")
    # second-order convergence of the centred difference in delta
    assert errs[1] < 1e-3
    assert errs[0] / errs[1] > 3.0


def test_deterministic_part_is_dt_N_F():
    ref, Q = _case()
    F = fbim_synth.random_forces(2, seed=4, net_zero=False)
    dt = 0.01
    got = _step(Q, ref, F, dt, 1.0, 1e-3, np.zeros(Q.size))
    expect = Q + dt * (_mobility(Q, ref) @ F.reshape(-1)).reshape(-1, 3)
    assert np.max(np.abs(got - expect)) < 1e-12 * np.max(np.abs(Q))


def test_biased_step_is_the_rfd_step_without_its_drift():
    """Eq. EM-noRFD: the Euler-Maruyama step without the random finite difference.  With
    zero noise it is Q + dt N F; with noise it equals the EM-RFD step at W~ = 0 (whose
    difference term then vanishes), the slip entering the same saddle solve."""
    ref, Q = _case()
    F = fbim_synth.random_forces(2, seed=5, net_zero=False)
    dt, kT = 0.01, 1.3
    W_r, Z = _zero_noise(Q.shape[0] * N_P)
    got = rfd.em_no_rfd_step(Q, ref, L, XI, F, dt, kT, W_r, Z)
    expect = Q + dt * (_mobility(Q, ref) @ F.reshape(-1)).reshape(-1, 3)
    assert np.max(np.abs(got - expect)) < 1e-12 * np.max(np.abs(Q))
    rng = np.random.default_rng(6)
    W_r = rng.standard_normal((Q.shape[0] * N_P, 2))
    Z = rng.standard_normal((16, 16, 2, 2))
    got = rfd.em_no_rfd_step(Q, ref, L, XI, F, dt, kT, W_r, Z)
    ref_step = rfd.em_rfd_step(Q, ref, L, XI, F, dt, kT, 1e-3, W_r, Z, np.zeros(Q.size))
    assert np.max(np.abs(got - ref_step)) < 1e-13 * np.max(np.abs(Q))
    assert np.max(np.abs(got - expect)) > 1e-6     # the noise moved the bodies


def _spring_force(Q):
    """Forces and torques of a spring between the two tracking points (rest length 1.5,
    stiffness 40) and angular springs to pi/4 and pi/2 (stiffness 2): F = -dU/dQ."""
    d = Q[1, :2] - Q[0, :2]
    r = np.linalg.norm(d)
    f = 40.0 * (r - 1.5) * d / r
    F = np.zeros_like(Q)
    F[0, :2] = f
    F[1, :2] = -f
    F[0, 2] = -2.0 * (Q[0, 2] - 0.25 * math.pi)
    F[1, 2] = -2.0 * (Q[1, 2] - 0.5 * math.pi)
    return F


def _trajectory(scheme, dt, T, ref):
    Q = np.array([[1.0, 1.2, 0.3], [2.25, 1.55, 1.7]])
    W_r, Z = _zero_noise(Q.shape[0] * ref.shape[0], M=8)
    zero = np.zeros(Q.size)
    NF = None
    for _ in range(int(round(T / dt))):
        F = _spring_force(Q)
        if scheme == "ab2":
            Q, NF = rfd.ab2_rfd_step(Q, ref, L, XI, F, NF, dt, 0.0, 1e-3, W_r, Z, zero)
        else:
            Q = rfd.em_rfd_step(Q, ref, L, XI, F, dt, 0.0, 1e-3, W_r, Z, zero)
    return Q


def test_ab2_deterministic_part_converges_at_second_order():
    # Sec. 4.4, Eq. AB2-RFD: 3/2 N^n F^n - 1/2 N^{n-1} F^{n-1} is the second-order
    # Adams-Bashforth step; at kT = 0 (no noise, no drift) the trajectory's successive
    # differences under halving dt shrink by ~4 (second order) against ~2 for Euler
    ref = fbim_synth.starfish_ref_nodes(12)
    T = 0.4
    ratios = {}
    for scheme in ("ab2", "em"):
        q = [_trajectory(scheme, dt, T, ref) for dt in (0.1, 0.05, 0.025)]
        ratios[scheme] = np.linalg.norm(q[0] - q[1]) / np.linalg.norm(q[1] - q[2])
    print(f"successive-difference ratios: AB2 {ratios['ab2']:.2f}, EM {ratios['em']:.2f}")
    assert 3.0 < ratios["ab2"] < 5.5
    assert 1.5 < ratios["em"] < 2.6
