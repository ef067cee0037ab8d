"""Pins for the oracle's Hasimoto split (Sec. 3.2)."""
import math

import numpy as np

from oracle import ewald, singlelayer

EULER_GAMMA = 0.57721566490153286061


def test_hasimoto_between_zero_and_one():
    k = np.linspace(0.0, 500.0, 20001)
    for xi in (0.5, 3.0, 20.0, 70.0):
        H = ewald.hasimoto(k, xi)
        assert np.all(H >= 0.0) and np.all(H <= 1.0 + 1e-15)
        assert abs(H[0] - 1.0) < 1e-15


def test_split_is_independent_of_xi():
    # G^(r)_xi + G^(w)_xi is the periodic Stokeslet for every xi
    L = 1.5
    rng = np.random.default_rng(3)
    r = rng.uniform(-0.7, 0.7, size=(12, 2))
    G1 = ewald.g_periodic(r, L, 4.0)
    G2 = ewald.g_periodic(r, L, 7.5)
    assert np.max(np.abs(G1 - G2)) < 1e-12 * np.max(np.abs(G1))


def test_real_kernel_small_r_matches_free_space_stokeslet():
    xi = 5.0
    for ang in (0.0, 0.7, 2.0):
        rv = 1e-6 * np.array([math.cos(ang), math.sin(ang)])
        G = ewald.g_real(rv[None, :], xi)[0] * 4 * math.pi
        rh = rv / np.linalg.norm(rv)
        expect = (-math.log(1e-6) - math.log(xi) - 0.5 * EULER_GAMMA - 1.0) * np.eye(2) + np.outer(rh, rh)
        assert np.max(np.abs(G - expect)) < 1e-9


def test_real_kernel_decays_like_gaussian():
    xi = 4.0
    r = np.array([[3.0 / xi, 0.0]])
    G = ewald.g_real(r, xi)[0]
    assert np.max(np.abs(G)) < math.exp(-9.0)


def test_wave_matrix_is_positive_semidefinite():
    L = 1.0
    rng = np.random.default_rng(5)
    X = rng.uniform(0, L, size=(40, 2))
    Mw = singlelayer.wave_matrix(X, L, 6.0)
    lam = np.linalg.eigvalsh(0.5 * (Mw + Mw.T))
    assert np.max(np.abs(Mw - Mw.T)) < 1e-13 * np.max(np.abs(Mw))
    assert lam.min() > -1e-13 * lam.max()


def test_wave_kernel_has_zero_mean_over_the_cell():
    # the k = 0 mode is excluded: the cell average of G^(w) vanishes
    L = 1.0
    n = 64
    g = (np.arange(n) + 0.5) / n * L
    X, Y = np.meshgrid(g, g, indexing="ij")
    r = np.stack([X.ravel(), Y.ravel()], axis=1)
    G = ewald.g_wave(r, L, 3.0)
    assert np.max(np.abs(G.mean(axis=0))) < 1e-12
