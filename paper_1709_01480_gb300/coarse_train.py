"""Training data and training of the learned coarse level's pair network.

The targets come from FBIM itself: for each sampled pair geometry, the 6x6
two-body mobility N_pair is solved on the GPU (six saddle solves with unit
forces and torques, Sec. 3.1, batched over many pair configurations through
``Batch``), and the correction is C = N_pair - blockdiag(N_1, N_1(phi)) with
N_1 the single-body mobility in the same periodic box.  Pairs are sampled with
the gap log-uniform in [0.05 R, 2 R] (R = the body's largest radius), the
direction of the second body and its relative orientation uniform on [0, 2 pi),
in a box of side 16, body a at the centre with theta = 0 (so the lab frame is
a's frame).  The network is trained by ``MLP.adam_step`` (the library's own
tensor-core forward and backward kernels) on standardised inputs and outputs.

Usage as a script (on a machine with the GPU)::

    python -m paper_1709_01480_gb300.coarse_train --pairs 20000 --out model.npz
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import FBIM, MLP, Batch

BOX = 16.0


def _rot(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s], [s, c]])


def node_gap(ref: np.ndarray, d: np.ndarray, psi: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Smallest node-to-node distance of body a (origin, theta 0) and body b at distance d."""
    c, s = np.cos(phi), np.sin(phi)
    R = np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)  # [P, 2, 2]
    xb = np.einsum("pij,nj->pni", R, ref) + (d[:, None] * np.stack([np.cos(psi), np.sin(psi)], -1))[:, None, :]
    diff = xb[:, None, :, :] - ref[None, :, None, :]
    return np.sqrt(np.min(np.sum(diff * diff, axis=-1), axis=(1, 2)))


def sample_geometries(n: int, ref: np.ndarray, seed: int):
    """(d, psi, phi, gap) of n pairs: gap log-uniform in [0.05 R, 2 R], centre distance by bisection."""
    rng = np.random.default_rng(seed)
    R = float(np.max(np.linalg.norm(ref, axis=1)))
    target = np.exp(rng.uniform(math.log(0.05 * R), math.log(2.0 * R), n))
    psi = rng.uniform(0.0, 2.0 * math.pi, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    d = np.empty(n)
    gap = np.empty(n)
    for o in range(0, n, 64):
        sl = slice(o, min(n, o + 64))
        lo = np.full(sl.stop - sl.start, 0.5 * R)
        hi = 2.0 * R + target[sl] + 0.05
        for _ in range(14):  # the realised gap is measured below; the target only shapes the mix
            mid = 0.5 * (lo + hi)
            below = node_gap(ref, mid, psi[sl], phi[sl]) < target[sl]
            lo = np.where(below, mid, lo)
            hi = np.where(below, hi, mid)
        d[sl] = hi
        gap[sl] = node_gap(ref, hi, psi[sl], phi[sl])
    return d, psi, phi, gap


def features(d, psi, phi, gap) -> np.ndarray:
    return np.stack([d * np.cos(psi), d * np.sin(psi), d, np.cos(phi), np.sin(phi), gap], -1)


def pair_targets(N_pair: np.ndarray, N_1: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """C [P, 36] = sym(N_pair - blockdiag(N_1, T(phi) N_1 T(phi)^T)), row-major 6 x 6."""
    P = N_pair.shape[0]
    C = N_pair.copy()
    C[:, :3, :3] -= N_1
    T = np.zeros((P, 3, 3))
    T[:, 0, 0] = np.cos(phi)
    T[:, 0, 1] = -np.sin(phi)
    T[:, 1, 0] = np.sin(phi)
    T[:, 1, 1] = np.cos(phi)
    T[:, 2, 2] = 1.0
    C[:, 3:, 3:] -= np.einsum("pij,jk,plk->pil", T, N_1, T)
    C = 0.5 * (C + np.transpose(C, (0, 2, 1)))
    return C.reshape(P, 36)


def two_body_dataset(n_pairs: int, n_p: int = 128, tol: float = 1e-8, solve_tol: float = 1e-7, seed: int = 0,
                     n_handles: int = 128, r_c: float = 0.5, log=print):
    """(features [n, 6], targets [n, 36], stats) from two-body FBIM solves on the GPU."""
    import torch
    import fbim_synth

    ref = fbim_synth.starfish_ref_nodes(n_p)
    c = BOX / 2.0
    t0 = time.time()
    one = FBIM(ref, np.array([[c, c, 0.0]]), BOX, tol=tol, r_c=r_c, precision="fp32")
    cols = []
    for k in range(3):
        F = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
        F[0, k] = 1.0
        U, _, _, _ = one.mobility_solve(F, tol=solve_tol, max_iter=300)
        cols.append(U.cpu().numpy().reshape(3))
    N_1 = np.stack(cols, axis=1)
    N_1 = 0.5 * (N_1 + N_1.T)
    one.close()
    d, psi, phi, gap = sample_geometries(n_pairs, ref, seed)
    H = min(n_handles, n_pairs)
    ops = [FBIM(ref, np.array([[c, c, 0.0], [c + 3.0, c, 0.0]]), BOX, tol=tol, r_c=r_c, precision="fp32")
           for _ in range(H)]
    batch = Batch(ops, [6] * H)
    eye = torch.eye(6, dtype=torch.float64, device="cuda")
    N_pair = np.empty((n_pairs, 6, 6))
    iters = []
    for o in range(0, n_pairs, H):
        n = min(H, n_pairs - o)
        for k in range(H):
            i = o + min(k, n - 1)  # spare handles repeat the last pair of a short chunk
            Q = torch.tensor([[c, c, 0.0], [c + d[i] * math.cos(psi[i]), c + d[i] * math.sin(psi[i]), phi[i]]],
                             dtype=torch.float64, device="cuda")
            ops[k].update_config(Q)
        F = [eye[r].reshape(2, 3) for k in range(H) for r in range(6)]
        U, it, res = batch.solve(F, None, tol=solve_tol, max_iter=400)
        iters.extend(it)
        for k in range(n):
            N_pair[o + k] = np.stack([U[6 * k + r].cpu().numpy().reshape(6) for r in range(6)], axis=1)
        if log and (o // H) % 20 == 0:
            log(f"  two-body solves: {o + n}/{n_pairs} pairs, {time.time() - t0:.1f} s")
    batch.close()
    for op in ops:
        op.close()
    N_pair = 0.5 * (N_pair + np.transpose(N_pair, (0, 2, 1)))
    X = features(d, psi, phi, gap)
    T = pair_targets(N_pair, N_1, phi)
    stats = dict(seconds=time.time() - t0, mean_iters=float(np.mean(iters)), N_1=N_1.tolist())
    return X, T, stats


def normalization(X: np.ndarray, T: np.ndarray):
    in_shift = X.mean(axis=0)
    in_scale = np.maximum(X.std(axis=0), 1e-6)
    out_scale = np.maximum(T.std(axis=0), 1e-8)
    return in_shift.astype(np.float32), in_scale.astype(np.float32), out_scale.astype(np.float32)


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases, in the library's parameter layout."""
    rng = np.random.default_rng(seed)
    widths = (6, 128, 128, 128, 36)
    parts = []
    for i in range(4):
        a = math.sqrt(6.0 / (widths[i] + widths[i + 1]))
        parts.append(rng.uniform(-a, a, widths[i + 1] * widths[i]))
        parts.append(np.zeros(widths[i + 1]))
    return np.concatenate(parts).astype(np.float32)


def train(X: np.ndarray, T: np.ndarray, epochs: int = 200, batch: int = 1024, lr: float = 2e-3, seed: int = 0,
          val_frac: float = 0.1, log=print):
    """Train a fresh network; returns (MLP, history dict)."""
    import torch

    in_shift, in_scale, out_scale = normalization(X, T)
    Xn = ((X - in_shift) / in_scale).astype(np.float32)
    Tn = (T / out_scale).astype(np.float32)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(X))
    n_val = max(1, int(val_frac * len(X)))
    val, tr = perm[:n_val], perm[n_val:]
    dev = torch.device("cuda")
    Xt = torch.tensor(Xn[tr], device=dev)
    Tt = torch.tensor(Tn[tr], device=dev)
    Xv = torch.tensor(Xn[val], device=dev)
    Tv = torch.tensor(Tn[val], device=dev)
    model = MLP(max_batch=max(batch, n_val), device=0)
    model.set_params(init_params(seed))
    model.set_normalization(in_shift, in_scale, out_scale)
    hist = dict(train=[], val=[])
    n = len(tr)
    steps = 0
    for ep in range(epochs):
        lr_ep = lr * (0.5 * (1 + math.cos(math.pi * ep / epochs)))  # cosine decay
        order = torch.randperm(n, generator=torch.Generator().manual_seed(seed * 100003 + ep)).to(dev)
        tot = 0.0
        for o in range(0, n - batch + 1, batch):
            idx = order[o:o + batch]
            tot += model.adam_step(Xt[idx].contiguous(), Tt[idx].contiguous(), lr=lr_ep)
            steps += 1
        nb = max(1, n // batch)
        vloss, _ = model.gradient(Xv, Tv)
        hist["train"].append(tot / nb)
        hist["val"].append(vloss)
        if log and (ep % max(1, epochs // 10) == 0 or ep == epochs - 1):
            log(f"  epoch {ep}: train {tot / nb:.4e}, validation {vloss:.4e}")
    hist["steps"] = steps
    return model, hist


def save(path: str, model: MLP, meta: dict):
    in_shift, in_scale, out_scale = model.normalization
    np.savez(path, theta=model.get_params(), in_shift=in_shift, in_scale=in_scale, out_scale=out_scale,
             **{k: np.asarray(v) for k, v in meta.items()})


def load(path: str, max_batch: int = 4096, device: int = 0) -> tuple:
    z = np.load(path)
    model = MLP(max_batch=max_batch, device=device)
    model.set_params(z["theta"])
    model.set_normalization(z["in_shift"], z["in_scale"], z["out_scale"])
    meta = {k: z[k] for k in z.files if k not in ("theta", "in_shift", "in_scale", "out_scale")}
    return model, meta


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--n-p", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    X, T, st = two_body_dataset(a.pairs, n_p=a.n_p, seed=a.seed)
    print(f"dataset: {len(X)} pairs in {st['seconds']:.1f} s, mean GMRES iterations {st['mean_iters']:.1f}")
    model, hist = train(X, T, epochs=a.epochs, seed=a.seed)
    R = float(np.max(X[:, 5])) / 2.0
    save(a.out, model, dict(g_c=float(np.max(X[:, 5])), pairs=a.pairs, n_p=a.n_p, box=BOX,
                            final_train=hist["train"][-1], final_val=hist["val"][-1], R=R))
    print(f"saved {a.out}: validation loss {hist['val'][-1]:.4e} (standardised targets)")


if __name__ == "__main__":
    main()
