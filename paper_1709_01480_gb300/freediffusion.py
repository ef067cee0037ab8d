"""Free diffusion of many independent single-body trajectories through the batched path.

Sec. 4.4.1 runs Brownian dynamics of one four-fold starfish in the periodic unit cell,
with and without the random finite difference, to show that the stochastic drift is
what makes the scheme sample the Gibbs-Boltzmann distribution.  Here R independent
trajectories advance together, one step being:

* every trajectory's handle moved to its configuration Q_k (``fbim_update_config``);
* EM-RFD only: W~_k from Philox (seed_k, stream 2, counter = step), the two displaced
  handles moved to Q_k +- delta/2 W~_k (``fbim_update_config_displaced``);
* the Brownian slips of all trajectories in one batched Lanczos (``fbim_batch_slip``,
  seed_k, counter 3 step -- the draws of ``fbim_bd_step``);
* all saddle solves of the step in one batched solve (``fbim_batch_solve``): the slip
  with zero force at Q_k, and for EM-RFD the force W~_k at Q_k +- delta/2 W~_k;
* Q <- Q + dt U (+ dt kT/delta (U+ - U-)) on the device (``fbim_bd_update``), Eqs.
  EM-noRFD and EM-RFD with F = 0.

Step k of trajectory j equals ``fbim_bd_step`` on a single handle with seed_j and the
same step index, up to the solve tolerance.  Every operation is a call of the C ABI;
this module only allocates the stacked buffers and orders the calls.
"""
from __future__ import annotations

import numpy as np

from . import FBIM, Batch, bd_update


class FreeDiffusion:
    """R independent trajectories of one body each (reference nodes ``ref_nodes``, periodic
    cell of side L), starting from Q0 [R, 3]; scheme "em" (Eq. EM-RFD) or "em_no_rfd"
    (Eq. EM-noRFD).  ``seeds[j]`` seeds trajectory j's Philox draws."""

    def __init__(self, ref_nodes, L, Q0, scheme="em", dt=0.02, kT=1.0, delta=1e-3, tol=1e-7, ewald_tol=1e-7,
                 seeds=None, precision="fp64", order=4, r_c=0.0, max_iter=400):
        import torch
        if scheme not in ("em", "em_no_rfd"):
            raise ValueError("scheme: 'em' or 'em_no_rfd'")
        Q0 = np.ascontiguousarray(Q0, dtype=np.float64).reshape(-1, 3)
        self.R = R = Q0.shape[0]
        self.rfd = scheme == "em"
        self.dt, self.kT, self.delta, self.tol, self.max_iter = float(dt), float(kT), float(delta), float(tol), max_iter
        self.seeds = [int(s) for s in (range(R) if seeds is None else seeds)]
        if len(self.seeds) != R:
            raise ValueError("one seed per trajectory")
        # the grid rule's side and the warp kernels, untimed: every handle of a trajectory has
        # the same grid, so its far-field draws are those of a single handle with its seed
        mk = lambda q: FBIM(ref_nodes, q, L, tol=ewald_tol, r_c=r_c, precision=precision, order=order,
                            grid_tune=False, wave="warp")
        self.q_ops = [mk(Q0[j:j + 1]) for j in range(R)]
        self.pm_ops = [mk(Q0[j:j + 1]) for _ in (0, 1) for j in range(R)] if self.rfd else []   # all +, then all -
        self.slip_batch = Batch(self.q_ops)
        self.batch = Batch(self.q_ops + self.pm_ops)
        dev = torch.device("cuda", self.q_ops[0].device)
        self.Q = torch.tensor(Q0, device=dev)
        self.Wt = torch.zeros((R, 3), dtype=torch.float64, device=dev)
        n_sys = len(self.batch.systems)
        self.F = torch.zeros(3 * n_sys, dtype=torch.float64, device=dev)
        self.n_slip = sum(2 * o.n for o in self.q_ops)
        self.S = torch.zeros(self.n_slip + sum(2 * o.n for o in self.pm_ops), dtype=torch.float64, device=dev)
        self.U = torch.zeros(3 * n_sys, dtype=torch.float64, device=dev)
        self.iters = []
        self.lanczos = []

    def step(self, i):
        """Advance every trajectory by one step with step index i."""
        R = self.R
        for j, op in enumerate(self.q_ops):
            op.update_config(self.Q[j:j + 1])
        if self.rfd:
            for j, op in enumerate(self.q_ops):
                op.philox_normals(3, seed=self.seeds[j], stream=2, counter=i, out=self.Wt[j])
            w = self.Wt.view(-1)
            self.F[3 * R:6 * R].copy_(w)
            self.F[6 * R:9 * R].copy_(w)
            for j in range(R):
                self.pm_ops[j].update_config_displaced(self.Q[j:j + 1], 0.5 * self.delta, self.Wt[j:j + 1])
                self.pm_ops[R + j].update_config_displaced(self.Q[j:j + 1], -0.5 * self.delta, self.Wt[j:j + 1])
        _, lz = self.slip_batch.slip(self.seeds, counter=3 * i, kT=self.kT, dt=self.dt, tol=max(self.tol, 1e-12),
                                     max_iter=200, out=self.S[:self.n_slip])
        _, it, _ = self.batch.solve(self.F, self.S, tol=self.tol, max_iter=self.max_iter, out=self.U)
        if self.rfd:
            bd_update(self.Q.view(-1), self.U[:3 * R], self.dt, self.dt * self.kT / self.delta,
                      Up=self.U[3 * R:6 * R], Um=self.U[6 * R:9 * R])
        else:
            bd_update(self.Q.view(-1), self.U[:3 * R], self.dt)
        self.iters.append(it)
        self.lanczos.append(lz)

    def run(self, n_steps, first_step=0):
        """n_steps steps; returns the configurations [n_steps + 1, R, 3] (host), the first row
        the configurations before the first step."""
        import torch
        out = torch.empty((n_steps + 1, self.R, 3), dtype=torch.float64, device=self.Q.device)
        out[0].copy_(self.Q)
        for s in range(n_steps):
            self.step(first_step + s)
            out[s + 1].copy_(self.Q)
        return out.cpu().numpy()

    def close(self):
        for b in (getattr(self, "slip_batch", None), getattr(self, "batch", None)):
            if b is not None:
                b.close()
        for o in getattr(self, "q_ops", []) + getattr(self, "pm_ops", []):
            o.close()
