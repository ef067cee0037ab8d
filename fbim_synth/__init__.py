"""Seeded synthetic inputs for the FBIM hot path.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle.  It holds none of the method's arithmetic: it only draws body shapes,
positions, orientations, forces and Gaussian vectors from fixed seeds, with the
sizes and structure of the paper's suspensions (starfish-shaped rigid bodies
in a periodic square box, Sec. 4.4; random suspensions of Sec. 4.3).

Everything is float64 numpy.  Layouts:

* ``ref_nodes``  [N_p, 2]  reference-shape nodes gamma_ref(s_j), s_j = 2 pi j / N_p,
  measured from the body's tracking point.
* ``Q``          [N_b, 3]  (q_x, q_y, theta) per body.
* ``F``          [N_b, 3]  (f_x, f_y, torque) per body.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "starfish_ref_nodes", "starfish_area", "disk_ref_nodes", "place_bodies",
    "random_forces", "Workload", "WORKLOADS", "make_workload", "box_for_fraction",
    "BATCHES", "suspension_batch", "batch", "place_lattice", "dense_workload",
]


def starfish_ref_nodes(n_p: int, r_s: float = 0.5, b: float = 0.3, arms: int = 5) -> np.ndarray:
    """Nodes of the starfish r(s) = r_s (1 + b cos(arms s)), s_j = 2 pi j / n_p."""
    s = 2.0 * np.pi * np.arange(n_p) / n_p
    r = r_s * (1.0 + b * np.cos(arms * s))
    return np.stack([r * np.cos(s), r * np.sin(s)], axis=1)


def starfish_area(r_s: float = 0.5, b: float = 0.3) -> float:
    """Area of the starfish r(s) = r_s (1 + b cos(k s)) for any k >= 1."""
    return math.pi * r_s * r_s * (1.0 + 0.5 * b * b)


def disk_ref_nodes(n_p: int, a: float = 1.0) -> np.ndarray:
    s = 2.0 * np.pi * np.arange(n_p) / n_p
    return np.stack([a * np.cos(s), a * np.sin(s)], axis=1)


def box_for_fraction(n_b: int, area: float, phi: float) -> float:
    return math.sqrt(n_b * area / phi)


def _dense_outline(ref_nodes: np.ndarray, n_fine: int = 256) -> np.ndarray:
    """Outline resampled by trigonometric interpolation, for overlap tests only."""
    n_p = ref_nodes.shape[0]
    c = np.fft.fft(ref_nodes, axis=0) / n_p
    k = np.fft.fftfreq(n_p, d=1.0 / n_p)
    if n_p % 2 == 0:
        c[n_p // 2] *= 0.5
        c = np.concatenate([c, c[n_p // 2:n_p // 2 + 1]], axis=0)
        k = np.concatenate([k, [n_p // 2]])
        k[n_p // 2] = -n_p // 2
    s = 2.0 * np.pi * np.arange(n_fine) / n_fine
    return np.real(np.exp(1j * np.outer(s, k)) @ c)


def _rot(theta):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, -s], [s, c]])


def place_bodies(n_b: int, L: float, ref_nodes: np.ndarray, min_gap: float, seed: int,
                 max_tries: int = 200000) -> np.ndarray:
    """Random non-overlapping placement in the periodic box [0, L)^2.

    Centres are uniform, orientations uniform on [0, 2 pi); a candidate is kept
    when its outline stays at least ``min_gap`` from every placed outline
    (periodic minimum image).  Returns Q [n_b, 3].
    """
    rng = np.random.default_rng(seed)
    outline = _dense_outline(ref_nodes)
    r_env = float(np.max(np.linalg.norm(outline, axis=1)))
    # Outline subsets (every 8th, 4th, 2nd point) decide most pairs exactly before
    # the full test.  With delta_s the largest distance from an outline point to the
    # nearest point of subset s, the full minimum distance D and the subset one D_s
    # obey D <= D_s <= D + 2 delta_s: D_s < gap rejects, D_s >= gap + 2 delta_s accepts.
    gap2 = min_gap * min_gap
    levels = []
    for stride in (8, 4, 2):
        sub = outline[::stride]
        delta = float(np.max(np.min(np.linalg.norm(outline[:, None, :] - sub[None, :, :], axis=2), axis=1)))
        levels.append((stride, (min_gap + 2.0 * delta) ** 2))
    reach = 2.0 * r_env + min_gap
    n_cell = max(1, int(L // reach))
    cell = L / n_cell
    grid: dict[tuple[int, int], list[int]] = {}
    Q = np.zeros((n_b, 3))
    placed_outlines = []
    n = 0
    tries = 0
    while n < n_b:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"placement failed after {max_tries} tries ({n}/{n_b} placed)")
        q = rng.uniform(0.0, L, size=2)
        th = rng.uniform(0.0, 2.0 * np.pi)
        cand = outline @ _rot(th).T
        cx, cy = int(q[0] // cell) % n_cell, int(q[1] // cell) % n_cell
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for other in grid.get(((cx + dx) % n_cell, (cy + dy) % n_cell), []):
                    d = Q[other, :2] - q
                    d -= L * np.round(d / L)
                    if np.hypot(*d) >= reach:
                        continue
                    other_outline = placed_outlines[other] + d
                    decided = False
                    for stride, sure2 in levels:
                        dc = other_outline[::stride, None, :] - cand[None, ::stride, :]
                        dc2 = np.min(np.einsum("ijk,ijk->ij", dc, dc))
                        if dc2 < gap2:
                            ok = False
                            decided = True
                            break
                        if dc2 >= sure2:
                            decided = True
                            break
                    if not ok:
                        break
                    if decided:
                        continue
                    diff = other_outline[:, None, :] - cand[None, :, :]
                    if np.min(np.einsum("ijk,ijk->ij", diff, diff)) < gap2:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        Q[n] = (q[0], q[1], th)
        placed_outlines.append(cand)
        grid.setdefault((cx, cy), []).append(n)
        n += 1
    return Q


def random_forces(n_b: int, seed: int, net_zero: bool = True) -> np.ndarray:
    """Per-body (f_x, f_y, torque) i.i.d. N(0,1); net force removed if asked."""
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((n_b, 3))
    if net_zero:
        F[:, :2] -= F[:, :2].mean(axis=0, keepdims=True)
    return F


def standard_normals(shape, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)


@dataclass
class Workload:
    """One synthetic suspension: geometry, Ewald tolerance and seeds."""
    name: str
    n_b: int
    n_p: int
    L: float
    tol: float
    Q: np.ndarray
    ref_nodes: np.ndarray
    F: np.ndarray
    seed: int
    min_gap: float
    phi: float
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.n_b * self.n_p


def make_workload(name: str, n_b: int, n_p: int, *, L: float | None = None, phi: float | None = None,
                  tol: float = 1e-8, min_gap: float = 0.1, seed: int = 0) -> Workload:
    ref = starfish_ref_nodes(n_p)
    area = starfish_area()
    if L is None:
        L = box_for_fraction(n_b, area, phi)
    phi_eff = n_b * area / (L * L)
    Q = place_bodies(n_b, L, ref, min_gap, seed)
    F = random_forces(n_b, seed + 1000)
    return Workload(name, n_b, n_p, float(L), tol, Q, ref, F, seed, min_gap, phi_eff)


# Named suspensions.  Sizes follow the starfish suspensions used for the
# method's accuracy and scaling studies: a tiny 4-body case that the dense
# oracle solves in seconds, and a 1024-body, 131072-node case for throughput.
WORKLOADS = {
    "starfish4_np64_L4": dict(n_b=4, n_p=64, L=4.0, tol=1e-10, min_gap=0.2, seed=0),
    "starfish1024_np128_phi0.25": dict(n_b=1024, n_p=128, phi=0.25, tol=1e-8, min_gap=0.1, seed=0),
}


def workload(name: str) -> Workload:
    kw = dict(WORKLOADS[name])
    return make_workload(name, **kw)


def suspension_batch(name: str, n_sys: int, n_min: int, n_max: int, n_p: int, phi_lo: float, phi_hi: float,
                     tol: float = 1e-8, min_gap: float = 0.1, seed: int = 0) -> list:
    """Independent starfish suspensions of uneven size.

    Body counts are log-uniform on [n_min, n_max] (rounded down), area
    fractions uniform on [phi_lo, phi_hi]; suspension i is placed with seed
    1000 seed + i + 1.  Returns a list of Workload.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_sys):
        n_b = int(np.floor(np.exp(rng.uniform(np.log(n_min), np.log(n_max + 1)))))
        n_b = min(max(n_b, n_min), n_max)
        phi = float(rng.uniform(phi_lo, phi_hi))
        out.append(make_workload(f"{name}[{i}]", n_b, n_p, phi=phi, tol=tol, min_gap=min_gap,
                                 seed=1000 * seed + i + 1))
    return out


# Named batches of independent suspensions: 64 starfish suspensions with
# 16..512 bodies (log-uniform), 96 nodes per body and area fractions 0.1..0.35.
BATCHES = {
    "batch64_starfish_np96": dict(n_sys=64, n_min=16, n_max=512, n_p=96, phi_lo=0.1, phi_hi=0.35, tol=1e-8,
                                  min_gap=0.1, seed=2),
}


def batch(name: str) -> list:
    return suspension_batch(name, **BATCHES[name])


def place_lattice(n_b: int, L: float, ref_nodes: np.ndarray, min_gap: float, seed: int) -> np.ndarray:
    """Jittered square lattice for dense suspensions (random sequential placement jams there).

    Sites of a k x k lattice (k = ceil(sqrt(n_b)), spacing a = L / k; n_b of them
    drawn at random when n_b < k^2), each centre moved uniformly by at most
    j = (a - 2 r_env - min_gap) / 2 per axis, orientations uniform on [0, 2 pi).
    Any two bodies then stay at least min_gap apart whatever their orientation
    (r_env = the outline's largest radius).  Returns Q [n_b, 3].
    """
    rng = np.random.default_rng(seed)
    k = int(math.ceil(math.sqrt(n_b)))
    a = L / k
    r_env = float(np.max(np.linalg.norm(_dense_outline(ref_nodes), axis=1)))
    j = 0.5 * (a - 2.0 * r_env - min_gap)
    if j < 0:
        raise ValueError(f"lattice spacing {a:.4f} too small for envelope {2 * r_env:.4f} + gap {min_gap}")
    sites = rng.permutation(k * k)[:n_b] if n_b < k * k else np.arange(k * k)
    ix, iy = sites % k, sites // k
    Q = np.zeros((n_b, 3))
    Q[:, 0] = ((ix + 0.5) * a + rng.uniform(-j, j, n_b)) % L
    Q[:, 1] = ((iy + 0.5) * a + rng.uniform(-j, j, n_b)) % L
    Q[:, 2] = rng.uniform(0.0, 2.0 * np.pi, n_b)
    return Q


def dense_workload(name: str, n_b: int, n_p: int, phi: float, min_gap: float, tol: float = 1e-8,
                   seed: int = 0) -> Workload:
    """Workload placed on a jittered lattice (``place_lattice``), forces as ``make_workload``."""
    ref = starfish_ref_nodes(n_p)
    L = box_for_fraction(n_b, starfish_area(), phi)
    Q = place_lattice(n_b, L, ref, min_gap, seed)
    F = random_forces(n_b, seed + 1000)
    return Workload(name, n_b, n_p, float(L), tol, Q, ref, F, seed, min_gap, n_b * starfish_area() / (L * L))


# The dense suspension of the learned coarse level: 4096 starfish, 128 nodes each, area
# fraction 0.40, gaps down to 0.05 R (R = 0.65, the largest radius).
DENSE = dict(n_b=4096, n_p=128, phi=0.40, min_gap=0.05 * 0.65, tol=1e-8, seed=0)
