"""Pins for the oracle's random slip (Secs. 3.3-3.4) and generator."""
import numpy as np

import fbim_synth
from oracle import brownian, ewald, philox, singlelayer


def test_philox_normals_have_unit_moments():
    z = philox.normals(400000, seed=12345, stream=0)
    n = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 0.05
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 5.0 / np.sqrt(n)


def test_philox_streams_and_counters_differ_and_prefix_is_stable():
    a = philox.normals(1000, 7, 0, 0)
    b = philox.normals(1000, 7, 1, 0)
    c = philox.normals(1000, 7, 0, 1)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.15 and abs(np.corrcoef(a, c)[0, 1]) < 0.15
    assert np.array_equal(philox.normals(333, 7, 0, 0), a[:333])


def test_philox_round_function_is_a_bijection_on_a_sample():
    ctr = np.arange(4096 * 4, dtype=np.uint32).reshape(-1, 4)
    out = philox.philox4x32_10(ctr, np.array([1, 2], dtype=np.uint32))
    assert len({tuple(r) for r in out}) == out.shape[0]


def test_hermitian_noise_layout():
    M = 8
    Z = np.random.default_rng(0).standard_normal((M, M, 2, 2))
    W = brownian.hermitian_noise(Z)
    # W(kappa) = conj W(-kappa mod M); zero mode 0; Nyquist modes real
    for jy in range(M):
        for jx in range(M):
            assert np.allclose(W[jy, jx], np.conj(W[(-jy) % M, (-jx) % M]))
    assert np.all(W[0, 0] == 0)
    for jy, jx in ((0, M // 2), (M // 2, 0), (M // 2, M // 2)):
        assert np.all(W[jy, jx].imag == 0) and np.all(W[jy, jx].real == Z[jy, jx, :, 0])


def test_far_field_covariance_is_wave_matrix():
    L, xi, M = 1.0, 6.0, 32
    rng = np.random.default_rng(1)
    X = rng.uniform(0, L, size=(6, 2))
    # linear map Z -> far field, column by column
    cols = []
    for i in range(M * M * 4):
        Z = np.zeros(M * M * 4)
        Z[i] = 1.0
        cols.append(brownian.far_field(X, L, xi, Z.reshape(M, M, 2, 2)).reshape(-1))
    A = np.array(cols).T
    C = A @ A.T
    kap = brownian.mode_lattice(M)
    ky, kx = np.meshgrid(kap, kap, indexing="ij")
    kv = np.stack([kx.ravel(), ky.ravel()], 1) * 2 * np.pi / L
    kv = kv[np.any(kv != 0, axis=1)]
    Mw = singlelayer.wave_matrix(X, L, xi, modes=(kv, ewald.wave_tensor(kv, xi)))
    assert np.max(np.abs(C - Mw)) < 1e-12 * np.max(np.abs(Mw))


def test_near_field_reproduces_real_space_covariance():
    # two well-separated, resolved bodies: M^(r) is positive definite and the
    # preconditioned square root must reproduce it exactly (Sec. 3.4)
    ref = fbim_synth.starfish_ref_nodes(48)
    L, xi = 3.0, 4.0
    Q = np.array([[0.8, 0.9, 0.4], [2.2, 1.6, 2.0]])
    X = singlelayer.node_positions(Q, ref)
    n = X.shape[0] * X.shape[1] * 2
    A = np.array([brownian.near_field(X, Q, ref, L, xi, e.reshape(-1, 2)).reshape(-1)
                  for e in np.eye(n)]).T
    Mr = singlelayer.real_matrix(X, L, xi)
    assert np.linalg.eigvalsh(Mr).min() > 0.0
    err = np.linalg.norm(A @ A.T - Mr) / np.linalg.norm(Mr)
    assert err < 1e-9
