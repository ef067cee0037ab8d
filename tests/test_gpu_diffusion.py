"""Free diffusion of a four-fold starfish in the periodic unit cell on the GPU (Sec. 4.4.1).

The body (b = 0.3, a = 1.3 r_s = 0.45, 64 nodes, 4th-order Alpert) diffuses freely in a
unit cell, Ewald and solver tolerance 1e-7, dt = 0.02, kT = 1, delta / a = eps^(1/3).

* The GPU's N(theta) equals the oracle's dense mobility (first kind, same xi).
* The biased step (Eq. EM-noRFD) equals the oracle's on the same noise.
* A step of the batched trajectories (``freediffusion``) equals ``fbim_bd_step`` on a
  single handle with the same seed and step, for both schemes.
* Statistics of 64 trajectories: with the random finite difference (Eq. EM-RFD) the
  orientation samples the uniform Gibbs-Boltzmann distribution (<cos 4 theta> = 0);
  without it the biased distribution proportional to 1 / N_thth (Eq. biased-dist),
  <cos 4 theta> = 0.123 from the oracle's N(theta).  The one-step translational mean
  square displacement is 4 kT <N_xx> dt with the average over each scheme's own
  distribution (2.46e-3 uniform, 2.26e-3 biased).  Bars: 4 standard errors of the
  trajectory means plus the Euler-Maruyama step's O(dt) bias (0.01 in <cos 4 theta>,
  1% in the displacement).
"""
import math

import numpy as np
import pytest

import fbim_synth
from oracle import brownian, diffusion, rfd, saddle, singlelayer

pytestmark = pytest.mark.gpu

L = 1.0
TOL = 1e-7
DT, KT = 0.02, 1.0
DELTA = 0.45 * TOL ** (1.0 / 3.0)
R, STEPS, BURN = 64, 400, 50


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def fb():
    import paper_1709_01480_gb300 as fb
    return fb


@pytest.fixture(scope="module")
def ref():
    return fbim_synth.starfish_ref_nodes(64, r_s=0.45 / 1.3, b=0.3, arms=4)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_gpu_mobility_of_the_starfish_matches_oracle(torch, fb, ref):
    for th in (0.0, 0.3, math.pi / 4):
        Q = np.array([[0.5, 0.5, th]])
        op = fb.FBIM(ref, Q, L, tol=1e-11, grid_tune=False)
        xi = op.info["xi"]
        N = np.zeros((3, 3))
        for c in range(3):
            F = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
            F[0, c] = 1.0
            U, _, it, res = op.mobility_solve(F, None, tol=1e-12, max_iter=400)
            N[:, c] = U.cpu().numpy()[0]
        op.close()
        X = singlelayer.node_positions(Q, ref)
        N_or = saddle.mobility(singlelayer.single_layer(X, L, xi, 1.0, 4), saddle.k_matrix(X, Q))
        err = np.abs(N - N_or) / np.sqrt(np.outer(np.diag(N_or), np.diag(N_or)))
        print(f"theta {th:.3f}: N_xx {N[0, 0]:.6e} N_thth {N[2, 2]:.6e}, max rel err {err.max():.2e}")
        assert err.max() < 1e-7


def test_biased_step_matches_oracle(torch, fb, ref):
    """One step of Eq. EM-noRFD (force kept) with given noise against the oracle's."""
    Q0 = np.array([[0.5, 0.5, 0.4]])
    op = fb.FBIM(ref, Q0, L, tol=1e-12, grid_tune=False)
    # a grid about 1.2 times the rule's smallest side: at the smallest one the gridded
    # far-field noise (which carries H^1/2 where the operator carries H) meets the
    # oracle's mode sum only to ~1e-8
    grid = 16 * math.ceil(1.2 * op.info["grid_min"] / 16)
    op.close()
    op = fb.FBIM(ref, Q0, L, tol=1e-12, grid=grid)
    xi = op.info["xi"]
    assert op.info["grid"] == grid
    rng = np.random.default_rng(8)
    W_r = rng.standard_normal((64, 2))
    Z = rng.standard_normal((grid, grid, 2, 2))
    F = rng.standard_normal((1, 3))
    Q = torch.tensor(Q0, device="cuda")
    it = op.bd_step(torch.tensor(F, device="cuda"), Q, DT, KT, DELTA, scheme="em_no_rfd",
                    W_r=torch.tensor(W_r, device="cuda"), Z_w=torch.tensor(Z, device="cuda"), tol=1e-12)
    dQ = Q.cpu().numpy() - Q0
    dQ_or = rfd.em_no_rfd_step(Q0, ref, L, xi, F, DT, KT, W_r, Z) - Q0
    err = _rel(dQ, dQ_or)
    print(f"biased step: GMRES iterations {it}, rel err of the displacement {err:.2e}")
    assert err < 1e-8
    op.close()


@pytest.mark.parametrize("scheme", ["em", "em_no_rfd"])
def test_batched_step_equals_single_handle_steps(torch, fb, ref, scheme):
    from paper_1709_01480_gb300.freediffusion import FreeDiffusion
    Q0 = np.array([[0.5, 0.5, 0.1], [0.3, 0.6, 1.0], [0.7, 0.2, 2.5]])
    seeds, step = [11, 12, 13], 5
    fd = FreeDiffusion(ref, L, Q0, scheme=scheme, dt=DT, kT=KT, delta=DELTA, tol=1e-11, ewald_tol=1e-10,
                       seeds=seeds)
    fd.step(step)
    got = fd.Q.cpu().numpy() - Q0
    fd.close()
    for j in range(3):
        op = fb.FBIM(ref, Q0[j:j + 1], L, tol=1e-10, grid_tune=False, wave="warp")
        Q = torch.tensor(Q0[j:j + 1], device="cuda")
        op.bd_step(torch.zeros((1, 3), dtype=torch.float64, device="cuda"), Q, DT, KT, DELTA, scheme=scheme,
                   seed=seeds[j], step=step, tol=1e-11)
        want = Q.cpu().numpy() - Q0[j:j + 1]
        op.close()
        err = _rel(got[j:j + 1], want)
        print(f"{scheme} trajectory {j}: batched vs single-handle step rel err {err:.2e}")
        assert err < 1e-8


@pytest.fixture(scope="module")
def expected(ref):
    _, N = diffusion.mobility_table(ref, L, 16, 12.0, order=4)
    return diffusion.equilibrium_averages(N)


@pytest.mark.parametrize("scheme,dist", [("em", "uniform"), ("em_no_rfd", "biased")])
def test_free_diffusion_statistics(torch, fb, ref, expected, scheme, dist):
    from paper_1709_01480_gb300.freediffusion import FreeDiffusion
    rng = np.random.default_rng(2024)
    Q0 = np.column_stack([np.full(R, 0.5), np.full(R, 0.5), rng.uniform(0.0, 0.5 * math.pi, R)])
    fd = FreeDiffusion(ref, L, Q0, scheme=scheme, dt=DT, kT=KT, delta=DELTA, tol=TOL, ewald_tol=TOL,
                       seeds=[5000 + 97 * (scheme == "em") + j for j in range(R)])
    traj = fd.run(STEPS)
    iters = np.array(fd.iters)
    fd.close()
    th = traj[BURN:, :, 2]
    c4 = np.cos(4.0 * th).mean(axis=0)                      # per trajectory
    m, se = c4.mean(), c4.std(ddof=1) / math.sqrt(R)
    d2 = np.sum(np.diff(traj[:, :, :2], axis=0) ** 2, axis=2)[BURN:] / (4.0 * KT * DT)
    per = d2.mean(axis=0)
    nxx, se_x = per.mean(), per.std(ddof=1) / math.sqrt(R)
    e = expected[dist]
    print(f"{scheme}: <cos 4 theta> {m:.4f} +- {se:.4f} (expected {e['cos4']:.4f}); MSD / 4 kT dt "
          f"{nxx:.4e} +- {se_x:.1e} (expected <N_xx> {e['nxx']:.4e}); GMRES iterations per solve "
          f"{iters.mean():.1f}")
    assert abs(m - e["cos4"]) < 4 * se + 0.01
    assert abs(nxx - e["nxx"]) < 4 * se_x + 0.01 * e["nxx"]
