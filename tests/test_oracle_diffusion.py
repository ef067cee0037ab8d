"""Pins for the free-diffusion expectations of the oracle (Sec. 4.4.1, oracle/diffusion.py).

* The orientation-averaged self-mobilities of the four-fold starfish reproduce the
  diffusion coefficients the paper prints, chi_trans = kT <N_xx> ~ 2.47e-3 and
  chi_rot = kT <N_thth> ~ 2.081e-1 (kT = 1, eta = 1).
* N(theta) has the symmetries of the body and the lattice: diagonal, N_xx = N_yy,
  and N(-theta) = N(theta).
* The stationary distributions that the averages assume (uniform with the drift term,
  proportional to 1/N_thth without it, Eq. biased-dist) are those a plain Monte Carlo
  walk of the orientation reaches, with and without the drift kT dN_thth/dtheta.
"""
import math

import numpy as np
import pytest

import fbim_synth
from oracle import diffusion, saddle, singlelayer

N_THETA = 16


@pytest.fixture(scope="module")
def table():
    ref = fbim_synth.starfish_ref_nodes(64, r_s=0.45 / 1.3, b=0.3, arms=4)
    return diffusion.mobility_table(ref, 1.0, N_THETA, 12.0, order=4)


def test_averages_reproduce_printed_diffusion_coefficients(table):
    _, N = table
    a = diffusion.equilibrium_averages(N)
    assert abs(a["uniform"]["nxx"] / 2.47e-3 - 1.0) < 5e-3
    assert abs(a["uniform"]["nthth"] / 0.2081 - 1.0) < 1e-3
    assert abs(a["uniform"]["cos4"]) < 1e-14
    # the biased distribution favours the orientations of small N_thth
    assert a["biased"]["nthth"] < a["uniform"]["nthth"]
    assert a["biased"]["cos4"] > 0.1


def test_table_has_the_symmetries_of_body_and_lattice(table):
    th, N = table
    scale = N[:, 2, 2].max()
    assert np.max(np.abs(N[:, 0, 0] - N[:, 1, 1])) < 1e-9 * scale
    off = N.copy()
    for i in range(3):
        off[:, i, i] = 0.0
    assert np.max(np.abs(off)) < 1e-9 * scale
    # N(-theta) = N(theta): theta_j and theta_{n-j} = pi/2 - theta_j = -theta_j (mod pi/2)
    assert np.max(np.abs(N[1:, 2, 2] - N[:0:-1, 2, 2])) < 1e-9 * scale
    # the interpolant reproduces its samples, and between them it is close enough for the
    # orientation walk (the averages themselves converge much faster: 16 vs 32 samples
    # agree to 1e-6)
    f, _ = diffusion.periodic_interpolant(N[:, 2, 2])
    assert np.max(np.abs(f(th) - N[:, 2, 2])) < 1e-14
    ref = fbim_synth.starfish_ref_nodes(64, r_s=0.45 / 1.3, b=0.3, arms=4)
    t_mid = (N_THETA // 4 + 0.5) * (0.5 * math.pi / N_THETA)
    Q = np.array([[0.5, 0.5, t_mid]])
    X = singlelayer.node_positions(Q, ref)
    Nd = saddle.mobility(singlelayer.single_layer(X, 1.0, 12.0, 1.0, 4), saddle.k_matrix(X, Q))
    assert abs(f(t_mid) - Nd[2, 2]) < 1e-3 * Nd[2, 2]


def test_orientation_walk_reaches_the_predicted_distributions(table):
    _, N = table
    a = diffusion.equilibrium_averages(N)
    m_d, se_d = diffusion.theta_walk(N[:, 2, 2], 1.0, 0.02, 1200, 2000, 3, drift=True, burn=100)
    m_n, se_n = diffusion.theta_walk(N[:, 2, 2], 1.0, 0.02, 1200, 2000, 4, drift=False, burn=100)
    print(f"<cos 4 theta>: with drift {m_d:.4f} +- {se_d:.4f} (uniform 0); without {m_n:.4f} +- {se_n:.4f} "
          f"(biased {a['biased']['cos4']:.4f})")
    # 4 standard errors plus the walk's own O(dt) bias (about 0.002 at dt = 0.02)
    assert abs(m_d - a["uniform"]["cos4"]) < 4 * se_d + 0.003
    assert abs(m_n - a["biased"]["cos4"]) < 4 * se_n + 0.003
