"""GPU parity of the batched mobility solve (graph-captured batch of independent suspensions).

Three suspensions of different size, shape sampling and box, with 3, 1 and 2
right-hand sides (forces, forces plus slip, slip only).  Bars: the FP64 batch
reaches relative residual 1e-12 on every system and each U matches the oracle's
dense LU solution to 1e-9 (the bar of the single-system solve).  The
mixed-precision batch reaches FP64 residual 1e-6 on every system and each U
matches the oracle to 2e-5 (the 1e-6 residual times the saddle system's
amplification, which is below 20 on these suspensions).
"""
import math

import numpy as np
import pytest

import fbim_synth
from oracle import saddle, singlelayer

pytestmark = pytest.mark.gpu

EWALD_TOL = 1e-13


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


@pytest.fixture(scope="module")
def suspensions():
    """(workload, n_box, grid) of three suspensions with the oracle's dense blocks."""
    out = []
    specs = [(fbim_synth.workload("starfish4_np64_L4"), 6, 160),
             (fbim_synth.make_workload("b6", 6, 48, L=5.0, tol=EWALD_TOL, min_gap=0.2, seed=3), 8, 0),
             (fbim_synth.make_workload("b9", 9, 32, L=6.0, tol=EWALD_TOL, min_gap=0.2, seed=4), 8, 0)]
    for w, n_box, grid in specs:
        xi = _xi(w.L, n_box, EWALD_TOL)
        X = singlelayer.node_positions(w.Q, w.ref_nodes)
        M = singlelayer.single_layer(X, w.L, xi)
        K = saddle.k_matrix(X, w.Q)
        out.append(dict(w=w, n_box=n_box, grid=grid, xi=xi, M=M, K=K))
    return out


def _ops(fb, sus, precision):
    return [fb.FBIM(s["w"].ref_nodes, s["w"].Q, s["w"].L, tol=EWALD_TOL, r_c=s["w"].L / s["n_box"], xi=s["xi"],
                    grid=s["grid"], precision=precision) for s in sus]


N_RHS = [3, 1, 2]


def _rhs(sus):
    """Per system: (F [n_b, 3], slip [N, 2] or zeros)."""
    F, S = [], []
    for k, s in enumerate(sus):
        w = s["w"]
        rng = np.random.default_rng(100 + k)
        for r in range(N_RHS[k]):
            f = rng.standard_normal((w.n_b, 3)) if (k, r) != (2, 1) else np.zeros((w.n_b, 3))
            sl = rng.standard_normal((w.n, 2)) if (k, r) in ((0, 2), (2, 1), (1, 0)) else np.zeros((w.n, 2))
            F.append(f)
            S.append(sl)
    return F, S


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _oracle_U(s, f, sl):
    _, U = saddle.solve_saddle(s["M"], s["K"], f.reshape(-1), sl.reshape(-1))
    return U


def test_fp64_batch_matches_dense_oracle(torch, fb, suspensions):
    ops = _ops(fb, suspensions, "fp64")
    batch = fb.Batch(ops, N_RHS)
    F, S = _rhs(suspensions)
    tF = [torch.tensor(f, device="cuda") for f in F]
    tS = [torch.tensor(s, device="cuda") for s in S]
    U, it, res = batch.solve(tF, tS, tol=1e-12, max_iter=400)
    info = batch.info()
    print(f"fp64 batch: iterations {it}, residuals {['%.1e' % r for r in res]}, info {info}")
    assert info["n_systems"] == sum(N_RHS) and info["branches"] == 3
    assert info["graph_kernels"][1] > 0 and info["graph_kernels"][3] > 0
    i = 0
    for k, s in enumerate(suspensions):
        for r in range(N_RHS[k]):
            assert res[i] <= 1e-12
            err = _rel(U[i].cpu().numpy().reshape(-1), _oracle_U(s, F[i], S[i]))
            print(f"  system ({k},{r}): U rel err vs oracle {err:.2e}")
            assert err < 1e-9
            i += 1
    batch.close()
    for o in ops:
        o.close()


def test_batch_equals_single_solves_after_a_move(torch, fb, suspensions):
    """Move every body of one suspension, solve again: each system equals its single solve."""
    ops = _ops(fb, suspensions, "fp64")
    batch = fb.Batch(ops, N_RHS)
    F, S = _rhs(suspensions)
    tF = [torch.tensor(f, device="cuda") for f in F]
    tS = [torch.tensor(s, device="cuda") for s in S]
    batch.solve(tF, tS, tol=1e-12, max_iter=400)
    w = suspensions[2]["w"]
    Q2 = w.Q.copy()
    Q2[:, 2] += 0.05  # rotate every body a little (stays non-overlapping at gap 0.2)
    ops[2].update_config(torch.tensor(Q2, device="cuda"))
    U, it, res = batch.solve(tF, tS, tol=1e-12, max_iter=400)
    i = 0
    for k, op in enumerate(ops):
        for r in range(N_RHS[k]):
            Us, _, its, ress = op.mobility_solve(tF[i], tS[i], tol=1e-12, max_iter=400)
            err = _rel(U[i].cpu().numpy(), Us.cpu().numpy())
            print(f"system ({k},{r}): batch {it[i]} it / single {its} it, U rel diff {err:.2e}")
            assert err < 1e-9
            i += 1
    # the moved suspension against the oracle at its new configuration
    X2 = singlelayer.node_positions(Q2, w.ref_nodes)
    M2 = singlelayer.single_layer(X2, w.L, suspensions[2]["xi"])
    K2 = saddle.k_matrix(X2, Q2)
    _, U_or = saddle.solve_saddle(M2, K2, F[4].reshape(-1), S[4].reshape(-1))
    assert _rel(U[4].cpu().numpy().reshape(-1), U_or) < 1e-9
    batch.close()
    for o in ops:
        o.close()


def test_mixed_precision_batch(torch, fb, suspensions):
    ops = _ops(fb, suspensions, "fp32")
    batch = fb.Batch(ops, N_RHS)
    F, S = _rhs(suspensions)
    tF = [torch.tensor(f, device="cuda") for f in F]
    tS = [torch.tensor(s, device="cuda") for s in S]
    U, it, res = batch.solve(tF, tS, tol=1e-6, max_iter=400)
    print(f"mixed batch: iterations {it}, residuals {['%.1e' % r for r in res]}")
    i = 0
    for k, s in enumerate(suspensions):
        for r in range(N_RHS[k]):
            assert res[i] <= 1e-6
            U_or = _oracle_U(s, F[i], S[i])
            err = _rel(U[i].cpu().numpy().reshape(-1), U_or)
            print(f"  system ({k},{r}): U rel err vs oracle {err:.2e}")
            assert err < 2e-5
            i += 1
    batch.close()
    for o in ops:
        o.close()


def test_zero_rhs_system_returns_zero(torch, fb, suspensions):
    ops = _ops(fb, suspensions[:2], "fp64")
    batch = fb.Batch(ops, [1, 1])
    w0, w1 = suspensions[0]["w"], suspensions[1]["w"]
    F = [torch.zeros((w0.n_b, 3), dtype=torch.float64, device="cuda"), torch.tensor(w1.F, device="cuda")]
    U, it, res = batch.solve(F, None, tol=1e-10, max_iter=300)
    assert it[0] == 0 and res[0] == 0.0
    assert float(U[0].abs().max()) == 0.0
    assert res[1] <= 1e-10
    batch.close()
    for o in ops:
        o.close()


def test_batch_rejects_mismatched_handles(torch, fb, suspensions):
    a = _ops(fb, suspensions[:1], "fp64")[0]
    b = _ops(fb, suspensions[1:2], "fp32")[0]
    with pytest.raises(fb.FbimError):
        fb.Batch([a, b])
    with pytest.raises(fb.FbimError):
        fb.Batch([a, a])
    a.close()
    b.close()
