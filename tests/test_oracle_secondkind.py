"""Pins for the oracle's completed second-kind solver (App. B).

What fixes the formulation independently of the code under test:

* Each periodic sum is independent of the splitting parameter xi (the Hasimoto split
  changes only how the sum is computed, App. B): a wrong prefactor or sign in a real or
  a wave part, or a real part that is not the wave part's complement, fails.
* The double layer of a constant density on a closed curve is -1/2 of it at the curve
  (principal value, normal into the body: the classical identity of the stresslet,
  whose divergence is a point force), and the trapezoidal rule reaches it spectrally
  once the self term is the kernel's limit along the curve weighted by Delta s.
* N is spectrally convergent in N_p and symmetric (Lorentz reciprocity, App. A).
* N equals the first-kind oracle's N (Sec. 3.1, an independent formulation and
  quadrature) to the first kind's own accuracy: dropping the mean-flow term T^(0)
  shifts N by ~7%, a flipped closure or completion sign breaks symmetry or agreement.
* A dilute square array of disks follows Sangani and Acrivos's expansion
  F/(eta U) = 4 pi / (-ln sqrt(phi) - 0.738 + phi - 0.887 phi^2 + 2.039 phi^3) (Sec. 4.1,
  Eq. DiluteTheory): its constant is printed to three digits, so the level of 4 pi U / F
  is checked to half a unit of that digit, and its phi-dependence (the expansion's
  phi, phi^2, phi^3 terms) to 3e-5 over phi = 0.002 ... 0.03.
"""
import math

import numpy as np

import fbim_synth
from oracle import saddle, secondkind, singlelayer


def test_periodic_rotlet_and_stresslet_do_not_depend_on_xi():
    rng = np.random.default_rng(0)
    L = 3.0
    r = rng.uniform(-1.5, 1.5, (25, 2))
    for f in (secondkind.rotlet_periodic, secondkind.stresslet_periodic):
        a, b = f(r, L, 2.0), f(r, L, 3.5)
        assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))


def test_rotlet_real_part_is_the_free_rotlet_near_the_origin():
    # R^(r) -> x^perp / r^2 / (4 pi) as xi r -> 0
    r = np.array([[1e-4, 3e-5], [-2e-5, 7e-5]])
    free = secondkind.perp(r) / np.sum(r * r, axis=1)[:, None] / (4.0 * np.pi)
    got = secondkind.rotlet_real(r, 2.0)
    assert np.max(np.abs(got - free) / np.abs(free).max()) < 1e-7


def _constant_density_defect(n_p):
    ref = fbim_synth.starfish_ref_nodes(n_p)
    t, n, speed, kappa = secondkind.curve_geometry(ref)
    ds = speed * 2.0 * np.pi / n_p
    rr = ref[:, None, :] - ref[None, :, :]
    r2 = np.sum(rr * rr, axis=-1)
    np.fill_diagonal(r2, 1.0)
    T = -4.0 * np.einsum("tsj,tsl,tsm->tsjlm", rr, rr, rr) / (r2 ** 2)[..., None, None, None]
    K = np.einsum("tsjlm,sm->tsjl", T, -n) * ds[None, :, None, None]
    for i in range(n_p):
        K[i, i] = -2.0 * kappa[i] * np.outer(t[i], t[i]) * ds[i]
    D = K.sum(axis=1) / (4.0 * np.pi)
    return float(np.max(np.abs(D + 0.5 * np.eye(2))))


def test_constant_density_double_layer_is_minus_one_half():
    errs = [_constant_density_defect(n_p) for n_p in (64, 128, 256)]
    assert errs[2] < 1e-12
    assert errs[0] > 1e3 * errs[1] > 1e3 * errs[2]     # spectral, not algebraic


def test_curve_geometry_of_a_circle():
    t, n, speed, kappa = secondkind.curve_geometry(fbim_synth.disk_ref_nodes(32, 2.0))
    s = 2.0 * np.pi * np.arange(32) / 32
    assert np.allclose(speed, 2.0, atol=1e-13) and np.allclose(kappa, 0.5, atol=1e-13)
    assert np.allclose(n, np.stack([np.cos(s), np.sin(s)], axis=1), atol=1e-13)   # outward
    assert np.allclose(t, np.stack([-np.sin(s), np.cos(s)], axis=1), atol=1e-13)


Q2 = np.array([[0.8, 0.9, 0.4], [2.2, 1.6, 2.0]])
L2, XI2 = 3.0, 3.0


def test_second_kind_mobility_converges_spectrally_and_is_symmetric():
    N = {n_p: secondkind.mobility(Q2, fbim_synth.starfish_ref_nodes(n_p), L2, XI2) for n_p in (64, 128, 256)}
    scale = np.max(np.abs(N[256]))
    assert np.max(np.abs(N[128] - N[256])) < 1e-9 * scale
    assert np.max(np.abs(N[64] - N[256])) > 1e2 * np.max(np.abs(N[128] - N[256]))
    assert np.max(np.abs(N[256] - N[256].T)) < 1e-13 * scale
    assert np.all(np.linalg.eigvalsh(0.5 * (N[256] + N[256].T)) > 0)


def test_second_kind_matches_the_first_kind_oracle():
    N2 = secondkind.mobility(Q2, fbim_synth.starfish_ref_nodes(256), L2, XI2)
    ref = fbim_synth.starfish_ref_nodes(192)
    X = singlelayer.node_positions(Q2, ref)
    N1 = saddle.mobility(singlelayer.single_layer(X, L2, 6.0, order=8), saddle.k_matrix(X, Q2))
    err = np.max(np.abs(N1 - N2)) / np.max(np.abs(N2))
    print(f"first kind (192 nodes, order 8) vs second kind (256 nodes): {err:.2e}")
    assert err < 1e-9


def test_dilute_square_array_of_disks_follows_sangani_acrivos():
    ref = fbim_synth.disk_ref_nodes(64, 1.0)
    gaps = []
    for phi in (0.002, 0.01, 0.03):
        l = math.sqrt(math.pi / phi)
        N = secondkind.mobility(np.array([[0.5 * l, 0.5 * l, 0.0]]), ref, l, max(24.0 / l, 1.2))
        assert abs(N[0, 1]) < 1e-12 * N[0, 0] and abs(N[0, 2]) < 1e-12 * N[0, 0]
        denom = -math.log(math.sqrt(phi)) - 0.738 + phi - 0.887 * phi ** 2 + 2.039 * phi ** 3
        gaps.append(4.0 * math.pi * N[0, 0] - denom)
    print("4 pi U/F minus the expansion:", gaps)
    assert max(abs(g) for g in gaps) < 5e-4          # the printed constant's last digit
    assert max(gaps) - min(gaps) < 3e-5              # the phi-dependence
