"""GPU parity of the block-diagonal body operators (Sec. 3.4) with the oracle.

fbim_precondition applies the preconditioner once; the oracle restates Sec. 3.4
body by body (``oracle.saddle.block_preconditioner``: dense pseudo-inverse of the
reference block, rotated, Schur complement from each body's actual nodes).  Three
library forms are checked: the FP64 handle (library FP64 GEMM), the FP32 handle on
the tensor cores (tcgen05, three-term TF32) and the FP32 handle on the library's
FP32 GEMM.  Cases span one and two 128-row tiles of the reference block (2 n_p =
64 ... 256), K padding (2 n_p = 96, 192), and more bodies than one CTA holds (16)
with a ragged last CTA.

Bars (max-norm relative to the oracle's output): U 1e-9 for FP64 and 5e-7 for FP32
(measured 3e-8 to 9e-8); mu 1e-7 for FP64 and 1e-5 for FP32 (measured 2e-7 to 2e-6:
mu is weighted by M_ref^+, whose smallest kept eigenvalues, the near-null normal
modes, amplify the rounding of the contraction).
"""
import math

import numpy as np
import pytest

import fbim_synth
from oracle import saddle

pytestmark = pytest.mark.gpu

CASES = [
    # (n_b, n_p, L, seed, n_box): 2 n_p = 128, 96, 64 (one tile), 192, 256 (two tiles)
    (4, 64, 4.0, 0, 6),
    (3, 48, 3.2, 5, 4),
    (21, 32, 8.0, 9, 10),
    (5, 96, 6.0, 3, 6),
    (3, 128, 5.0, 4, 5),
]
FORMS = [("fp64", True), ("fp32", True), ("fp32", False)]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def fb():
    import paper_1709_01480_gb300 as fb
    return fb


def _xi(L, n_box, tol):
    return math.sqrt(math.log(100.0 / tol)) / (L / n_box)


_oracle = {}


def _case(n_b, n_p, L, seed, n_box):
    key = (n_b, n_p, L, seed, n_box)
    if key not in _oracle:
        ref = fbim_synth.starfish_ref_nodes(n_p)
        Q = fbim_synth.place_bodies(n_b, L, ref, 0.15, seed)
        xi = _xi(L, n_box, 1e-12)
        rng = np.random.default_rng(seed + 40)
        r_mu = rng.standard_normal((n_b * n_p, 2))
        r_U = rng.standard_normal((n_b, 3))
        mu, U = saddle.block_preconditioner(r_mu, r_U, Q, ref, L, xi)
        _oracle[key] = (ref, Q, xi, r_mu, r_U, mu, U)
    return _oracle[key]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision,tc", FORMS)
@pytest.mark.parametrize("case", CASES)
def test_preconditioner_matches_oracle(torch, fb, case, precision, tc):
    n_b, n_p, L, seed, n_box = case
    ref, Q, xi, r_mu, r_U, mu_or, U_or = _case(*case)
    op = fb.FBIM(ref, Q, L, tol=1e-12, r_c=L / n_box, xi=xi, precision=precision, tensor_cores=tc)
    r = torch.tensor(np.concatenate([r_mu.reshape(-1), r_U.reshape(-1)]), device="cuda")
    out = op.precondition(r).cpu().numpy()
    mu = out[:2 * n_b * n_p].reshape(-1, 2)
    U = out[2 * n_b * n_p:].reshape(-1, 3)
    eU, emu = _rel(U, U_or), _rel(mu, mu_or)
    print(f"{precision} tc={tc} {n_b}x{n_p}: U rel err {eU:.2e}, mu rel err {emu:.2e}")
    fp64 = precision == "fp64"
    assert eU < (1e-9 if fp64 else 5e-7)
    assert emu < (1e-7 if fp64 else 1e-5)
    op.close()


def test_tensor_core_slip_and_solve_match_the_library_gemm(torch, fb):
    w = fbim_synth.workload("starfish4_np64_L4")
    # the grid rule's side for both (a timed grid choice could differ between the handles,
    # and the far-field draws follow the grid)
    ops = {tc: fb.FBIM(w.ref_nodes, w.Q, w.L, tol=1e-10, r_c=w.L / 6, precision="fp32", tensor_cores=tc,
                       grid_tune=False)
           for tc in (True, False)}
    assert ops[True].info["grid"] == ops[False].info["grid"]
    slips = {tc: op.brownian_slip(kT=1.0, dt=1e-3, seed=5, counter=2, tol=1e-8)[0] for tc, op in ops.items()}
    es = float((slips[True] - slips[False]).abs().max() / slips[False].abs().max())
    F = torch.tensor(w.F, device="cuda")
    sol = {tc: op.mobility_solve(F, slips[False], tol=1e-8, max_iter=300) for tc, op in ops.items()}
    eU = float((sol[True][0] - sol[False][0]).abs().max() / sol[False][0].abs().max())
    print(f"tensor cores vs library GEMM: slip {es:.2e}, U {eU:.2e}, iterations {sol[True][2]} vs {sol[False][2]}")
    assert es < 1e-5
    assert eU < 1e-6
    assert abs(sol[True][2] - sol[False][2]) <= 2
    for op in ops.values():
        op.close()
