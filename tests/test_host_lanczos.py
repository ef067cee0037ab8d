"""The host routine of the Lanczos square root (Sec. 3.3): c = |w| sqrt(T) e_1 from the
tridiagonal T the iteration builds, checked without a GPU against numpy's dense
eigen-decomposition (the definition: S sqrt(max(Lambda, 0)) S^T e_1).

Cases: random tridiagonals of sizes 1 ... 60, with zero off-diagonals (deflation), a
near-identity T, negative Ritz values (clipped) and clustered spectra; and the T of
plain Lanczos runs (full reorthogonalisation, numpy) on the near-field operator
G M(r) G^T of a suspension whose reference block has dropped modes (the oracle's
matrices), continued far past convergence, where T carries a cluster of zero Ritz
values and off-diagonals down to 1e-13: from the projected start the library uses,
c against the dense definition; from W itself, the slip's G^+ V c against the exact
G^+ (G M(r) G^T)^1/2 W.  Bar: 1e-12 relative.  (A deflation test relative only to the
neighbouring diagonal entries never deflates a cluster of zero eigenvalues: such a
routine is off by up to 1e-1 on these matrices.)
"""
import math

import numpy as np

import fbim_synth
import paper_1709_01480_gb300 as fb
from oracle import brownian, philox, singlelayer


def _reference(a, b, wn):
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    lam, S = np.linalg.eigh(T)
    return wn * S @ (np.sqrt(np.clip(lam, 0.0, None)) * S[0])


def _check(a, b, wn=1.7):
    got = fb.host_lanczos_sqrt(a, b, wn)
    ref = _reference(a, b, wn)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def test_random_tridiagonals():
    rng = np.random.default_rng(0)
    worst = 0.0
    for k in (1, 2, 3, 5, 8, 13, 21, 34, 60):
        for t in range(5):
            a = rng.uniform(0.5, 2.0, k)
            b = rng.uniform(0.0, 0.6, k - 1)
            if t == 1:
                b[::3] = 0.0
            elif t == 2:
                a[:] = 1.0
                b[:] = 1e-9
            elif t == 3:
                a = rng.uniform(-0.01, 2.0, k)
            elif t == 4:
                a[:] = 1.0
                b = rng.uniform(0.3, 0.5, k - 1)
            worst = max(worst, _check(a, b))
    assert worst < 1e-12


def _lanczos(A, w0, steps):
    """Plain Lanczos with full reorthogonalisation (two classical Gram-Schmidt passes)."""
    V = [w0 / np.linalg.norm(w0)]
    al, be = [], []
    for _ in range(steps):
        x = A @ V[-1]
        Vm = np.array(V)
        for _ in range(2):
            x = x - Vm.T @ (Vm @ x)
        al.append(float(V[-1] @ (A @ V[-1])))
        be.append(float(np.linalg.norm(x)))
        V.append(x / be[-1])
    return np.array(V), np.array(al), np.array(be)


def test_lanczos_runs_past_convergence_with_zero_ritz_values():
    w = fbim_synth.make_workload("b6", 6, 48, L=5.0, tol=1e-13, min_gap=0.2, seed=3)
    xi = math.sqrt(math.log(100.0 / 1e-13)) / (w.L / 8)
    X = singlelayer.node_positions(w.Q, w.ref_nodes)
    n_b, n_p = X.shape[:2]
    Mref = brownian.reference_real_block(w.ref_nodes, w.L, xi)
    G_ref, Gd_ref = brownian.g_factors(Mref)
    assert np.sum(np.linalg.eigvalsh(Mref) <= 0) >= 1          # modes are dropped: G is singular
    R = brownian.rotation_blocks(w.Q[:, 2], n_p)
    G = R @ np.kron(np.eye(n_b), G_ref) @ R.T
    Gd = R @ np.kron(np.eye(n_b), Gd_ref) @ R.T
    A = G @ singlelayer.real_matrix(X, w.L, xi) @ G.T
    lam, U = np.linalg.eigh(0.5 * (A + A.T))
    f = np.where(lam > 1e-12 * lam.max(), np.sqrt(np.clip(lam, 0.0, None)), 0.0)
    W = philox.normals(2 * w.n, 72, 0, 9)
    # (a) the library's start, W projected onto the range of G: T's near-zero Ritz values
    # (from rounding) carry no weight, and c must match the dense definition
    Wp = Gd @ (G @ W)
    V, al, be = _lanczos(A, Wp, 100)
    assert min(be) < 1e-11                                     # the run reaches near-breakdown
    worst = max(_check(al[:K], be[:K - 1], np.linalg.norm(Wp)) for K in range(2, 101, 7))
    assert worst < 1e-12
    # (b) W itself: T then holds Ritz values at +-1e-17 with weight, where sqrt(max(., 0))
    # amplifies rounding to ~1e-9 for any eigensolver; what the slip uses, G^+ V c, must
    # still be G^+ A^1/2 W (the null space of G carries f(0) = 0 and G^+ removes it)
    V, al, be = _lanczos(A, W, 100)
    exact = Gd @ (U @ (f * (U.T @ W)))
    worst = 0.0
    for K in range(9, 101, 7):           # converged from about 9 steps on
        c = fb.host_lanczos_sqrt(al[:K], be[:K - 1], np.linalg.norm(W))
        worst = max(worst, float(np.max(np.abs(Gd @ (V[:K].T @ c) - exact)) / np.max(np.abs(exact))))
    assert worst < 1e-12


def test_invalid_arguments():
    import ctypes
    out = np.zeros(3)
    lib = fb.lib()
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.fbim_host_lanczos_sqrt(p, p, 0, 1.0, p) != 0
    assert lib.fbim_host_lanczos_sqrt(None, p, 3, 1.0, p) != 0
