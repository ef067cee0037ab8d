"""Pin for the oracle's coarse-level body velocities (learned coarse level on Sec. 3.4).

For two bodies alone in the box, the exact pair correction C = N_pair -
blockdiag(N~_a, N~_b) turns the coarse-level velocities into the pair's true
mobility: N~ a + C a = N_pair a (Sec. 3.1, Eq. discreteParticleVelocity, for the
pair).  N_pair is assembled here independently of ``oracle.coarse``: one dense
saddle solve of the two bodies at their lab-frame coordinates.  The per-body
mobilities N~_b follow the library's block preconditioner: the reference body's
mobility rotated by theta_b.  With body a at theta = 0 the frame of
``two_body`` is the lab frame, so the identity is exact; a wrong sign, a
correction added to the wrong body, the rotated block subtracted from the wrong
body or the halves of a_pair swapped each break it.
"""
import math

import numpy as np

import fbim_synth
from oracle import coarse, saddle, singlelayer

L = 8.0
XI = math.sqrt(math.log(100.0 / 1e-12)) / (L / 8)


def _mob(Q, ref):
    X = singlelayer.node_positions(Q, ref)
    M = singlelayer.single_layer(X, L, XI)
    return saddle.mobility(M, saddle.k_matrix(X, Q))


def _T3(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def test_exact_pair_correction_reproduces_the_pair_mobility():
    ref = fbim_synth.starfish_ref_nodes(32)
    dx, dy, phi = 1.05, 0.62, 2.1
    c = L / 2
    Q = np.array([[c, c, 0.0], [c + dx, c + dy, phi]])
    N_pair = _mob(Q, ref)                                     # independent two-body solve
    N_ref = _mob(np.array([[c, c, 0.0]]), ref)                # reference body alone
    Np, Ns = coarse.two_body(ref, L, XI, dx, dy, phi)
    C = coarse.to_lab(coarse.pair_target(Np, Ns, phi), 0.0)
    N_tilde = np.stack([N_ref, _T3(phi) @ N_ref @ _T3(phi).T])
    a = np.random.default_rng(2).standard_normal((2, 3))
    U = coarse.coarse_velocity(N_tilde, np.array([[0, 1]]), C[None], a)
    expect = (N_pair @ a.reshape(-1)).reshape(2, 3)
    err = np.max(np.abs(U - expect)) / np.max(np.abs(expect))
    print(f"coarse velocity vs pair mobility: rel err {err:.2e}")
    assert err < 1e-10
    # the correction is not negligible: without it the velocities differ visibly
    U0 = np.einsum("bij,bj->bi", N_tilde, a)
    assert np.max(np.abs(U0 - expect)) > 1e-3 * np.max(np.abs(expect))


def test_pair_listed_in_reverse_order_gives_the_same_velocities():
    # the pair (1, 0) with the correction expressed for body 1 first
    ref = fbim_synth.starfish_ref_nodes(32)
    dx, dy, phi = -0.9, 0.8, 0.7
    c = L / 2
    Q = np.array([[c + dx, c + dy, phi], [c, c, 0.0]])        # body 1 is at the centre, theta = 0
    N_pair = _mob(Q, ref)
    N_ref = _mob(np.array([[c, c, 0.0]]), ref)
    Np, Ns = coarse.two_body(ref, L, XI, dx, dy, phi)
    C = coarse.to_lab(coarse.pair_target(Np, Ns, phi), 0.0)   # ordered (centre body, other)
    N_tilde = np.stack([_T3(phi) @ N_ref @ _T3(phi).T, N_ref])
    a = np.random.default_rng(3).standard_normal((2, 3))
    U = coarse.coarse_velocity(N_tilde, np.array([[1, 0]]), C[None], a)
    expect = (N_pair @ a.reshape(-1)).reshape(2, 3)
    assert np.max(np.abs(U - expect)) < 1e-10 * np.max(np.abs(expect))
