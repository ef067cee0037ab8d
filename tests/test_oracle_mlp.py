"""CPU pins of the learned coarse level's oracle: the network, Adam, bf16 rounding, pair features.

The network's back-propagation is pinned by central finite differences of its
loss; the forward pass by a network reduced to one path through tanh units;
Adam by its closed-form first step and its constant-gradient sequence
(Kingma & Ba, Algorithm 1); bf16 rounding by exactly representable ties; the
pair features by brute force and invariance under a rigid motion of the whole
configuration; the two-body correction by the symmetry of the pair mobility
and the decay of the coupling with separation.
"""
import math

import numpy as np
import pytest

import fbim_synth
from oracle import coarse, mlp


def _theta(seed, scale=0.3):
    return np.random.default_rng(seed).standard_normal(mlp.n_params()) * scale


def test_param_count():
    assert mlp.n_params() == 6 * 128 + 128 + 2 * (128 * 128 + 128) + 36 * 128 + 36 == 38564


def test_bf16_rounding_ties_to_even():
    one = 1.0
    u = 2.0 ** -7  # bf16 spacing at 1
    vals = np.array([one, one + u / 2, one + 3 * u / 2, one + u / 2 + 2.0 ** -20, -(one + u / 2), 3.0e-3])
    r = mlp.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                 # halfway, mantissa 0 is even
    assert r[2] == one + 2 * u         # halfway between odd 1+u and even 1+2u
    assert r[3] == one + u             # just above halfway
    assert r[4] == -1.0
    assert abs(r[5] - 3.0e-3) <= 3.0e-3 * 2.0 ** -8


def test_forward_single_path_closed_form():
    theta = np.zeros(mlp.n_params())
    layers = mlp.unpack(theta)  # views into theta
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = layers
    W1[0, 2] = 0.75
    b1[0] = 0.1
    W2[3, 0] = 1.5
    W3[5, 3] = -2.0
    W4[7, 5] = 0.5
    b4[7] = 0.25
    b4[11] = -1.0
    X = np.array([[0.0, 0.0, 0.4, 0.0, 0.0, 0.0], [0.0, 0.0, -1.3, 0.0, 0.0, 0.0]])
    Y, _ = mlp.forward(theta, X, rounding=False)
    for i in range(2):
        h1 = math.tanh(0.75 * X[i, 2] + 0.1)
        h2 = math.tanh(1.5 * h1)
        h3 = math.tanh(-2.0 * h2)
        expect = np.zeros(36)
        expect[7] = 0.5 * h3 + 0.25
        expect[11] = -1.0
        assert np.allclose(Y[i], expect, atol=1e-15)
    # and the transposed use of any weight matrix would move the output elsewhere
    assert np.count_nonzero(Y[0]) == 2


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(4)
    theta = _theta(5)
    X = rng.standard_normal((5, 6))
    T = rng.standard_normal((5, 36))
    _, g = mlp.loss_grad(theta, X, T, rounding=False)
    h = 1e-6
    idx = np.concatenate([rng.integers(0, mlp.n_params(), 40), [0, 767, 768, 38563, 38527]])
    for i in idx:
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_grad(tp, X, T, rounding=False)[0] - mlp.loss_grad(tm, X, T, rounding=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_rounded_gradient_close_to_exact():
    rng = np.random.default_rng(6)
    theta = _theta(7)
    X = rng.standard_normal((64, 6))
    T = rng.standard_normal((64, 36))
    _, g0 = mlp.loss_grad(theta, X, T, rounding=False)
    _, g1 = mlp.loss_grad(theta, X, T, rounding=True)
    rel = np.linalg.norm(g1 - g0) / np.linalg.norm(g0)
    assert 1e-4 < rel < 3e-2  # bf16 operands: relative error of order 2^-8, not zero


def test_adam_first_step_and_constant_gradient():
    rng = np.random.default_rng(8)
    theta = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, eps = 1e-3, 1e-8
    m = np.zeros(50)
    v = np.zeros(50)
    t1, m, v = mlp.adam(theta, m, v, g, 1, lr, eps=eps)
    assert np.allclose(t1 - theta, -lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    t2, m, v = mlp.adam(t1, m, v, g, 2, lr, eps=eps)
    assert np.allclose(t2 - t1, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)


def _config():
    ref = fbim_synth.starfish_ref_nodes(32)
    Q = np.array([[2.0, 2.0, 0.3], [3.25, 2.2, 1.9], [2.2, 3.3, -0.7], [5.0, 5.5, 2.5]])
    return ref, Q


def test_pair_features_brute_force_and_rigid_motion():
    ref, Q = _config()
    L = 8.0
    pairs, F = coarse.pair_features(Q, ref, L, g_c=0.6)
    assert pairs.tolist() == sorted(pairs.tolist()) and len(pairs) >= 2
    # brute force on one pair
    X = ref
    a, b = pairs[0]
    Ra = np.array([[math.cos(Q[a, 2]), -math.sin(Q[a, 2])], [math.sin(Q[a, 2]), math.cos(Q[a, 2])]])
    Rb = np.array([[math.cos(Q[b, 2]), -math.sin(Q[b, 2])], [math.sin(Q[b, 2]), math.cos(Q[b, 2])]])
    xa = Q[a, :2] + X @ Ra.T
    xb = Q[b, :2] + X @ Rb.T
    gap = min(np.hypot(*(p - q)) for p in xa for q in xb)
    d = Q[b, :2] - Q[a, :2]
    assert np.allclose(F[0], [*(Ra.T @ d), np.hypot(*d), math.cos(Q[b, 2] - Q[a, 2]),
                              math.sin(Q[b, 2] - Q[a, 2]), gap], atol=1e-13)
    # a common rotation about the box centre plus a translation across the periodic
    # boundary leaves every feature unchanged
    t = 0.83
    R = np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
    Q2 = Q.copy()
    Q2[:, :2] = (Q[:, :2] - L / 2) @ R.T + L / 2 + np.array([3.1, -2.4])
    Q2[:, :2] %= L
    Q2[:, 2] += t
    # rotation is exact only away from periodic images: use a box large enough
    pairs2, F2 = coarse.pair_features(Q2, ref, 40.0, g_c=0.6)
    pairs1, F1 = coarse.pair_features(Q, ref, 40.0, g_c=0.6)
    assert pairs1.tolist() == pairs2.tolist()
    assert np.allclose(F1, F2, atol=1e-12)


def test_two_body_target_symmetric_and_decaying():
    ref = fbim_synth.starfish_ref_nodes(32)
    L = 6.0
    xi = math.sqrt(math.log(1e12)) / (L / 8)
    norms = []
    for dist in (1.45, 2.0, 2.8):
        Np, Ns = coarse.two_body(ref, L, xi, dist * math.cos(0.4), dist * math.sin(0.4), 1.1)
        assert np.linalg.norm(Np - Np.T) <= 1e-10 * np.linalg.norm(Np)
        assert np.min(np.linalg.eigvalsh(Np)) > 0
        C = coarse.pair_target(Np, Ns, 1.1)
        norms.append(np.linalg.norm(C))
    assert norms[0] > norms[1] > norms[2] > 0


def test_coarse_velocity_adds_pair_terms():
    rng = np.random.default_rng(9)
    Nt = rng.standard_normal((3, 3, 3))
    C = rng.standard_normal((1, 6, 6))
    a = rng.standard_normal((3, 3))
    U = coarse.coarse_velocity(Nt, np.array([[0, 2]]), C, a)
    assert np.allclose(U[1], Nt[1] @ a[1])
    assert np.allclose(U[0], Nt[0] @ a[0] + C[0][:3, :3] @ a[0] + C[0][:3, 3:] @ a[2])
    assert np.allclose(U[2], Nt[2] @ a[2] + C[0][3:, :3] @ a[0] + C[0][3:, 3:] @ a[2])
