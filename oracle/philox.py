"""Philox4x32-10 counter-based generator and Box-Muller normals -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The method needs Gaussian vectors (Sec. 3.1: W with covariance (2kT/dt) I;
Sec. 3.3: W^(r) and the complex wave-space W^(w); Sec. 4.4: W~ of the random
finite difference) but fixes no generator.  Reading: both this oracle and the
CUDA library draw them from Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), each side implementing
it from that published definition:

    round:  (hi0, lo0) = mulhilo(0xD2511F53, x0); (hi1, lo1) = mulhilo(0xCD9E8D57, x2)
            x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0)
    key schedule between rounds: k0 += 0x9E3779B9, k1 += 0xBB67AE85 (mod 2^32)

Counter layout used by this project: key = (seed mod 2^32, seed >> 32),
counter = (pair index mod 2^32, pair index >> 32, stream, call counter).  One
block of four words yields two 53-bit uniforms u1 = (x0, x1), u2 = (x2, x3) in
(0, 1) and two normals sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2); normal i of a
vector is element i mod 2 of block i // 2.

Streams: 0 = near-field W^(r) [node, comp]; 1 = wave-space Z [ky, kx, comp, re/im];
2 = W~ [body, dof] of the random finite difference.

Parity: the exact bits are a convention of this project, not of the paper;
pinned statistically (moments and independence of the normals).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

STREAM_NEAR = 0
STREAM_WAVE = 1
STREAM_RFD = 2


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """ctr [n, 4] uint32, key [2] uint32 -> [n, 4] uint32."""
    x = ctr.astype(np.uint64)
    k0 = np.uint64(key[0])
    k1 = np.uint64(key[1])
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(W0)) & MASK
            k1 = (k1 + np.uint64(W1)) & MASK
        p0 = M0 * x[:, 0]
        p1 = M1 * x[:, 2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        x = np.stack([hi1 ^ x[:, 1] ^ k0, lo1, hi0 ^ x[:, 3] ^ k1, lo0], axis=1)
    return x.astype(np.uint32)


def _u53(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return ((a >> np.uint32(5)).astype(np.float64) * 67108864.0
            + (b >> np.uint32(6)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normals(n: int, seed: int, stream: int, counter: int = 0) -> np.ndarray:
    """The first n standard normals of (seed, stream, counter)."""
    n_blk = (n + 1) // 2
    idx = np.arange(n_blk, dtype=np.uint64)
    ctr = np.zeros((n_blk, 4), dtype=np.uint32)
    ctr[:, 0] = (idx & MASK).astype(np.uint32)
    ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(stream)
    ctr[:, 3] = np.uint32(counter & 0xFFFFFFFF)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    x = philox4x32_10(ctr, key)
    u1 = _u53(x[:, 0], x[:, 1])
    u2 = _u53(x[:, 2], x[:, 3])
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * n_blk)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:n]
