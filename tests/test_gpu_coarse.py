"""GPU parity of the learned coarse level: the pair network's kernels, the pair list, the coarse solve.

Bars.  Network forward and gradient against the oracle, which rounds the same
operands to bfloat16 and sums in float64: relative (max-norm) error <= 5e-3 for
the outputs and (2-norm) <= 5e-3 for the gradient; an activation whose FP32 and
FP64 values round to neighbouring bfloat16 numbers (2^-8 apart) is what the
margin covers.  Adam: the first step moves each parameter by -lr g / (|g| + eps)
on both sides; compared where |g| > 1e-3 max |g| to 1e-2 lr.  Pair list: the
same pairs (exact) and features to 1e-12.  Coarse-level solve: the same
solution as the block-diagonal solve to 1e-8 (both FP64 to residual 1e-11),
with both iteration counts reported.
"""
import math

import numpy as np
import pytest

import fbim_synth
from oracle import coarse as ocoarse
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def fb():
    import paper_1709_01480_gb300 as fb
    return fb


def _theta(seed):
    return (np.random.default_rng(seed).standard_normal(omlp.n_params()) * 0.25).astype(np.float32)


def test_mlp_forward_matches_oracle(torch, fb):
    theta = _theta(1)
    X = np.random.default_rng(2).standard_normal((300, 6)).astype(np.float32)
    m = fb.MLP(max_batch=512)
    m.set_params(theta)
    Y = m.forward(torch.tensor(X, device="cuda")).cpu().numpy()
    Yo, _ = omlp.forward(theta.astype(np.float64), X.astype(np.float64), rounding=True)
    err = np.max(np.abs(Y - Yo)) / np.max(np.abs(Yo))
    print(f"mlp forward: max rel err {err:.2e}, launches {m.launches}")
    assert err < 5e-3
    assert m.launches == 4
    m.close()


def test_mlp_gradient_matches_oracle(torch, fb):
    theta = _theta(3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((200, 6)).astype(np.float32)
    T = rng.standard_normal((200, 36)).astype(np.float32)
    m = fb.MLP(max_batch=256)
    m.set_params(theta)
    loss, g = m.gradient(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"))
    lo, go = omlp.loss_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64), rounding=True)
    g = g.cpu().numpy().astype(np.float64)
    gerr = np.linalg.norm(g - go) / np.linalg.norm(go)
    print(f"mlp gradient: loss {loss:.6f} vs oracle {lo:.6f}, gradient rel err {gerr:.2e}")
    assert abs(loss - lo) <= 1e-4 * lo
    assert gerr < 5e-3
    m.close()


def test_adam_step_matches_oracle(torch, fb):
    theta = _theta(5)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((128, 6)).astype(np.float32)
    T = rng.standard_normal((128, 36)).astype(np.float32)
    m = fb.MLP(max_batch=128)
    m.set_params(theta)
    lr = 1e-3
    m.adam_step(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), lr=lr)
    t1 = m.get_params().astype(np.float64)
    _, go = omlp.loss_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64), rounding=True)
    t1o, _, _ = omlp.adam(theta.astype(np.float64), np.zeros_like(go), np.zeros_like(go), go, 1, lr)
    sel = np.abs(go) > 1e-3 * np.max(np.abs(go))
    dev = np.max(np.abs((t1 - theta) - (t1o - theta))[sel])
    print(f"adam: {sel.sum()} compared, max deviation {dev:.2e} (lr {lr})")
    assert dev < 1e-2 * lr
    m.close()


def test_training_fits_a_smooth_map(torch, fb):
    """The library's own training loop reduces the loss on a smooth 6 -> 36 map by 10x."""
    from paper_1709_01480_gb300 import coarse_train
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, (4096, 6))
    A = rng.standard_normal((6, 36))
    T = np.tanh(X @ A) + 0.1 * (X[:, :1] ** 2)
    model, hist = coarse_train.train(X, T, epochs=60, batch=512, lr=3e-3, log=None)
    print(f"training: first epoch {hist['train'][0]:.3e}, last {hist['train'][-1]:.3e}, val {hist['val'][-1]:.3e}")
    assert hist["val"][-1] < 0.1 * hist["train"][0]
    model.close()


def _suspension():
    w = fbim_synth.make_workload("c8", 8, 64, phi=0.35, tol=1e-10, min_gap=0.05, seed=7)
    return w


def test_coarse_pairs_match_oracle(torch, fb):
    w = _suspension()
    op = fb.FBIM(w.ref_nodes, w.Q, w.L, tol=1e-10, r_c=0.5)
    for g_c in (0.3, 1.0):
        pairs, feats = op.coarse_pairs(g_c)
        po, fo = ocoarse.pair_features(w.Q, w.ref_nodes, w.L, g_c)
        print(f"g_c {g_c}: {len(po)} pairs")
        assert pairs.cpu().numpy().tolist() == po.tolist()
        assert np.allclose(feats.cpu().numpy(), fo, atol=1e-12, rtol=0)
    op.close()


def test_coarse_level_solve(torch, fb):
    """A network trained on FBIM two-body solves, used as the coarse level: same solution, iterations reported."""
    from paper_1709_01480_gb300 import coarse_train
    X, T, st = coarse_train.two_body_dataset(192, n_p=64, n_handles=64, seed=3, log=None)
    assert np.all(np.isfinite(T)) and X[:, 5].min() < 0.05 and X[:, 5].max() > 0.5
    model, hist = coarse_train.train(X, T, epochs=80, batch=128, lr=3e-3, log=None)
    print(f"two-body data: {len(X)} pairs, mean iterations {st['mean_iters']:.1f}; "
          f"validation loss {hist['val'][-1]:.3e} (standardised)")
    w = _suspension()
    op = fb.FBIM(w.ref_nodes, w.Q, w.L, tol=1e-10, r_c=0.5)
    F = torch.tensor(w.F, device="cuda")
    U0, _, it0, r0 = op.mobility_solve(F, tol=1e-11, max_iter=500)
    op.coarse_enable(model, 1.3)
    n_pairs, n_rej = op.coarse_stats()
    U1, _, it1, r1 = op.mobility_solve(F, tol=1e-11, max_iter=500)
    err = float((U1 - U0).abs().max() / U0.abs().max())
    print(f"coarse level: {n_pairs} pairs ({n_rej} dropped); GMRES iterations block-diagonal {it0}, "
          f"with the learned coarse level {it1}; residuals {r0:.1e} / {r1:.1e}; U rel diff {err:.1e}")
    assert n_pairs > 0
    assert r1 <= 1e-11 and err < 1e-8
    # fallback: a network with non-finite outputs has every pair dropped -> the block solve
    bad = fb.MLP(max_batch=64)
    bad.set_params(np.full(omlp.n_params(), np.nan, dtype=np.float32))
    bad.set_normalization(*model.normalization)
    op.coarse_enable(bad, 1.3)
    n_pairs2, n_rej2 = op.coarse_stats()
    U2, _, it2, r2 = op.mobility_solve(F, tol=1e-11, max_iter=500)
    assert n_rej2 == n_pairs2 > 0 and abs(it2 - it0) <= 1
    assert float((U2 - U0).abs().max() / U0.abs().max()) < 1e-8
    op.coarse_enable(None, 1.0)
    op.close()
    model.close()
    bad.close()


def test_coarse_stagnation_guard_falls_back_to_the_block_preconditioner(torch, fb):
    """A coarse level that passes the positive-definiteness check but misleads GMRES (every
    close pair corrected by C = c I): the stagnation guard ends the cycle after 20 steps
    without a tenfold residual drop, and the solve reaches its tolerance on the
    block-diagonal preconditioner with the block solve's solution."""
    w = _suspension()
    op = fb.FBIM(w.ref_nodes, w.Q, w.L, tol=1e-10, r_c=0.5)
    F = torch.tensor(w.F, device="cuda")
    U0, _, it0, _ = op.mobility_solve(F, tol=1e-10, max_iter=500)
    bad = fb.MLP(max_batch=64)
    theta = np.zeros(fb.mlp_param_count(), dtype=np.float32)
    theta[-36:][[0, 7, 14, 21, 28, 35]] = 1.0e4   # output bias: C = 1e4 I, weights zero
    bad.set_params(theta)
    bad.set_normalization(np.zeros(6), np.ones(6), np.ones(36))
    op.coarse_enable(bad, 1.3)
    n_pairs, n_rej = op.coarse_stats()
    U1, _, it1, r1 = op.mobility_solve(F, tol=1e-10, max_iter=500, check=False)
    fallbacks = op.info["coarse_fallbacks"]
    err = float((U1 - U0).abs().max() / U0.abs().max())
    print(f"misleading coarse level on {n_pairs} pairs ({n_rej} dropped): {it1} iterations "
          f"(block-diagonal {it0}), residual {r1:.1e}, fallbacks {fallbacks}, U rel diff {err:.1e}")
    assert n_pairs > 0 and n_rej < n_pairs
    assert fallbacks >= 1
    assert r1 <= 1e-10 and err < 1e-8
    assert it1 <= it0 + 25
    op.coarse_enable(None, 1.0)
    op.close()
    bad.close()


def test_coarse_preconditioner_matches_oracle(torch, fb):
    """fbim_precondition with the coarse level on (FP64 handle) against the oracle's
    composition: pair features, the bf16-faithful network, C = T sym(y s) T^T, the coarse
    velocities U = -(N~ a + sum C a_pair) and the tractions from that U."""
    w = _suspension()
    g_c = 1.3
    xi = math.sqrt(math.log(100.0 / 1e-10)) / 0.5
    op = fb.FBIM(w.ref_nodes, w.Q, w.L, tol=1e-10, r_c=0.5, precision="fp64")
    xi = op.info["xi"]
    theta = _theta(9)
    shift = np.array([0.0, 0.0, 1.2, 0.0, 0.0, 0.3], dtype=np.float32)
    scale = np.array([1.0, 1.0, 0.5, 1.0, 1.0, 0.3], dtype=np.float32)
    out = np.full(36, 2e-3, dtype=np.float32)   # corrections small enough to keep every pair
    m = fb.MLP(max_batch=64)
    m.set_params(theta)
    m.set_normalization(shift, scale, out)
    op.coarse_enable(m, g_c)
    n_pairs, n_rej = op.coarse_stats()
    rng = np.random.default_rng(21)
    r_mu = rng.standard_normal((w.n, 2))
    r_U = rng.standard_normal((w.n_b, 3))
    r = torch.tensor(np.concatenate([r_mu.reshape(-1), r_U.reshape(-1)]), device="cuda")
    got = op.precondition(r).cpu().numpy()
    pairs, feats = ocoarse.pair_features(w.Q, w.ref_nodes, w.L, g_c)
    xn = ((feats - shift.astype(np.float64)) / scale.astype(np.float64)).astype(np.float32).astype(np.float64)
    y, _ = omlp.forward(theta.astype(np.float64), xn, rounding=True)
    C_lab = []
    for p, (a, _) in enumerate(pairs):
        Cf = (y[p] * out.astype(np.float64)).reshape(6, 6)
        C_lab.append(ocoarse.to_lab(0.5 * (Cf + Cf.T), w.Q[a, 2]))
    mu_or, U_or = ocoarse.coarse_preconditioner(r_mu, r_U, w.Q, w.ref_nodes, w.L, xi, pairs, np.array(C_lab))
    mu = got[:2 * w.n].reshape(-1, 2)
    U = got[2 * w.n:].reshape(-1, 3)
    eU = float(np.max(np.abs(U - U_or)) / np.max(np.abs(U_or)))
    emu = float(np.max(np.abs(mu - mu_or)) / np.max(np.abs(mu_or)))
    # the pairs' share of U, so that the comparison is not the block solve's alone
    _, U_bd = ocoarse.coarse_preconditioner(r_mu, r_U, w.Q, w.ref_nodes, w.L, xi, pairs[:0], np.zeros((0, 6, 6)))
    share = float(np.max(np.abs(U_or - U_bd)) / np.max(np.abs(U_or)))
    print(f"coarse preconditioner: {n_pairs} pairs ({n_rej} dropped), pair share of U {share:.1e}; "
          f"U rel err {eU:.2e}, mu rel err {emu:.2e}")
    assert n_pairs == len(pairs) and n_rej == 0
    assert share > 1e-3
    assert eU < 1e-6 and emu < 1e-6
    op.coarse_enable(None, 1.0)
    op.close()
    m.close()
