"""The 8th-order Alpert rule on the GPU and the splitting-parameter sweep of Sec. 4.1.

Sec. 4.1 fixes the packing fraction at pi/16 (one disk of radius 1 in a box of side 4),
N_p = 64, and measures the error of the body mobility N (matrix 2-norm, relative to an
accurate N) as the cutoff shrinks, i.e. as r_Alpert / r_c grows (r_Alpert: distance from a
node to the farthest node the end correction touches): the error grows by at least two
orders of magnitude over the range, and r_Alpert / r_c <~ 0.6 keeps the rule accurate.

Here the library computes N from three unit solves (FP64 handles, Ewald tolerance 1e-12,
GMRES to 1e-12) for Alpert orders 4 and 8 over cutoffs L/3 ... L/12.  Each point is
checked against the oracle's N at the same parameters (parity of the order-8 and order-4
rules on the GPU at six splits), and the sweep against the oracle's N at N_p = 256 with
the order-8 rule and r_c = L/4 (r_Alpert / r_c = 0.2) as the accurate reference.
"""
import math

import numpy as np
import pytest

import fbim_synth
from oracle import saddle, singlelayer

pytestmark = pytest.mark.gpu

L = 4.0
Q = np.array([[2.0, 2.0, 0.0]])
N_BOXES = (3, 4, 5, 6, 8, 10, 12)


def _xi(n_box):
    return math.sqrt(math.log(100.0 / 1e-12)) / (L / n_box)


def _oracle_N(n_p, order, n_box):
    ref = fbim_synth.disk_ref_nodes(n_p, 1.0)
    X = singlelayer.node_positions(Q, ref)
    M = singlelayer.single_layer(X, L, _xi(n_box), order=order)
    return saddle.mobility(M, saddle.k_matrix(X, Q))


def _gpu_N(torch, fb, order, n_box):
    ref = fbim_synth.disk_ref_nodes(64, 1.0)
    op = fb.FBIM(ref, Q, L, tol=1e-12, r_c=L / n_box, xi=_xi(n_box), order=order, precision="fp64")
    info = op.info
    N = np.zeros((3, 3))
    for j in range(3):
        F = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
        F[0, j] = 1.0
        U, _, _, _ = op.mobility_solve(F, tol=1e-12, max_iter=300)
        N[:, j] = U.cpu().numpy().reshape(-1)
    # r_Alpert: the chord to the farthest node of the correction band
    r_alpert = 2.0 * math.sin(math.pi * info["alpert_band"] / 64)
    op.close()
    return N, r_alpert / info["r_c"]


def test_alpert_orders_on_the_gpu_and_the_splitting_sweep():
    import torch
    import paper_1709_01480_gb300 as fb
    assert torch.cuda.is_available()
    N_ref = _oracle_N(256, 8, 4)
    nref = np.linalg.norm(N_ref, 2)
    curves = {}
    for order in (4, 8):
        pts = []
        for n_box in N_BOXES:
            N, ratio = _gpu_N(torch, fb, order, n_box)
            N_or = _oracle_N(64, order, n_box)
            parity = np.linalg.norm(N - N_or, 2) / np.linalg.norm(N_or, 2)
            err = np.linalg.norm(N - N_ref, 2) / nref
            print(f"order {order} r_c = L/{n_box}: r_Alpert/r_c {ratio:.2f}, error vs reference {err:.2e}, "
                  f"vs oracle at the same split {parity:.1e}")
            assert parity < 1e-9
            pts.append((ratio, err))
        curves[order] = pts
    for order, pts in curves.items():
        errs = [e for _, e in pts]
        # the error grows steeply with r_Alpert / r_c: measured 63x for order 4 (ratios
        # 0.29 ... 1.17, where the N_p = 64 rule's own error floors it near 2e-5) and 8e4x
        # for order 8 (0.57 ... 2.30); the paper reports at least two orders of magnitude
        # over its range
        assert max(errs[-2:]) > (50.0 if order == 4 else 1000.0) * min(errs[:2])
        # within r_Alpert / r_c <= 0.6 the rule keeps its accuracy
        good = [e for r, e in pts if r <= 0.6]
        assert good and max(good) < (1e-3 if order == 4 else 1e-5)
    # at the same cutoff the 8th-order rule is the more accurate (where both resolve it)
    assert curves[8][0][1] < curves[4][0][1]


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 2e-6)])
def test_order8_matvec_matches_oracle(precision, bar):
    import torch
    import paper_1709_01480_gb300 as fb
    ref = fbim_synth.starfish_ref_nodes(64)
    Qs = fbim_synth.place_bodies(3, 4.0, ref, 0.2, 7)
    xi = math.sqrt(math.log(100.0 / 1e-13)) / (4.0 / 4)
    op = fb.FBIM(ref, Qs, 4.0, tol=1e-13, r_c=1.0, xi=xi, order=8, precision=precision)
    assert op.info["alpert_order"] == 8
    X = singlelayer.node_positions(Qs, ref)
    M = singlelayer.single_layer(X, 4.0, xi, order=8)
    mu = np.random.default_rng(3).standard_normal((3 * 64, 2))
    v = op.apply_stokeslet(torch.tensor(mu, device="cuda")).cpu().numpy()
    expect = (M @ mu.reshape(-1)).reshape(-1, 2)
    err = float(np.max(np.abs(v - expect)) / np.max(np.abs(expect)))
    print(f"order-8 matvec {precision}: rel err {err:.2e}")
    assert err < bar
    op.close()
