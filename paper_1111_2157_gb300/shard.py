"""k-point sharding of the lattice sum over ranks (one process per GPU).

Once Sigma(i w_n) is fixed, every (k, i w_n) point of Eq. dmftloop1 is
independent, and G_loc, N(mu) and dN/dmu are weighted sums over k (Eq. Gloc
and the occupation of Eq. fix_mu).  So each rank evaluates a contiguous slice
of the k-points, each point keeping its weight w_k of the full set, and one sum
all-reduce per evaluation joins the partial sums: of G_loc (n_w m^2 complex
numbers per system) when it is asked for, and of (N, dN/dmu) per system.  rho_k
(Eq. rho_k) stays on the rank that owns k.  The mu search (Eq. fix_mu) runs the
same safeguarded Newton iteration on every rank from the reduced N and dN/dmu,
so all ranks take identical steps without further messages.

The evaluator is any callable ``evaluate(mu, gloc) -> (gloc or None, N, dN_dmu)``
returning the rank's partial sums; ``greens_function_evaluator`` wraps a
``GreensFunction`` built for the rank's slice.  Collectives go through
``torch.distributed`` (NCCL for CUDA tensors, gloo for host tensors).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def partition_k(nb, world_size):
    """Contiguous k-slices [(k0, k1)] per rank, balanced by the cost sum of N_b(k)^3.

    The per-point work is the N_b x N_b inversion, so a slice's cost is the sum
    of N_b^3 over its k-points.  Slice r ends at the first k where the prefix
    cost reaches (r + 1) / world_size of the total; slices may be empty when
    there are fewer k-points than ranks.
    """
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    cost = np.asarray(nb, dtype=np.float64) ** 3
    if cost.ndim != 1:
        raise ValueError("nb must be one-dimensional")
    nk = len(cost)
    prefix = np.concatenate([[0.0], np.cumsum(cost)])
    total = prefix[-1]
    bounds = [0]
    for r in range(1, world_size):
        k = int(np.searchsorted(prefix, total * r / world_size, side="left"))
        bounds.append(min(max(k, bounds[-1]), nk))
    bounds.append(nk)
    return [(bounds[r], bounds[r + 1]) for r in range(world_size)]


def greens_function_evaluator(g):
    """Evaluator over a GreensFunction that holds this rank's k-slice (full-set weights)."""

    def evaluate(mu, gloc):
        out = g.evaluate(mu, gloc=gloc, rho=False, occupation=True, n_corr=False)
        return out["gloc"], out["N"], out["dN_dmu"]

    return evaluate


class ShardedLattice:
    """Lattice sums over the k-points of all ranks of ``group``."""

    def __init__(self, evaluate, n_sys=1, group=None, device="cpu"):
        self.evaluate_local = evaluate
        self.n_sys = int(n_sys)
        self.group = group
        self.device = torch.device(device)
        self.evaluations = 0

    def _allreduce(self, t):
        if dist.is_available() and dist.is_initialized():
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t

    def evaluate(self, mu, gloc=True):
        """(G_loc summed over all ranks or None, N per system, dN/dmu per system)."""
        mu = np.broadcast_to(np.asarray(mu, np.float64), (self.n_sys,)).copy()
        g_part, n_part, d_part = self.evaluate_local(mu, gloc)
        self.evaluations += 1
        nd = torch.tensor(np.concatenate([np.atleast_1d(n_part), np.atleast_1d(d_part)]),
                          dtype=torch.float64, device=self.device)
        self._allreduce(nd)
        g = None
        if gloc:
            g = torch.as_tensor(g_part).to(device=self.device, dtype=torch.complex128).contiguous()
            self._allreduce(torch.view_as_real(g))
        nd = nd.cpu().numpy()
        return g, nd[:self.n_sys], nd[self.n_sys:]

    def find_mu(self, n_target, mu0=0.0, tol=1e-10, max_iter=60, cap=4.0):
        """mu per system with |N - n_target| <= tol; returns (mu, evaluations).

        Safeguarded Newton on the reduced N(mu) (monotone increasing, dN/dmu > 0):
        a Newton step capped at ``cap`` while the bracket is one-sided, bisection
        when the step leaves the bracket.  Raises RuntimeError without convergence.
        """
        S = self.n_sys
        tgt = np.broadcast_to(np.asarray(n_target, np.float64), (S,))
        mu = np.broadcast_to(np.asarray(mu0, np.float64), (S,)).copy()
        lo, hi = np.full(S, -np.inf), np.full(S, np.inf)
        done = np.zeros(S, bool)
        for it in range(1, max_iter + 1):
            _, n, dn = self.evaluate(mu, gloc=False)
            for s in range(S):
                if done[s]:
                    continue
                f = n[s] - tgt[s]
                if abs(f) <= tol:
                    done[s] = True
                    continue
                if f < 0:
                    lo[s] = max(lo[s], mu[s])
                else:
                    hi[s] = min(hi[s], mu[s])
                step = -f / dn[s] if dn[s] > 1e-300 else (1.0 if f < 0 else -1.0)
                bracketed = np.isfinite(lo[s]) and np.isfinite(hi[s])
                if not bracketed:
                    step = float(np.clip(step, -cap, cap))
                new = mu[s] + step
                if bracketed and not (lo[s] < new < hi[s]):
                    new = 0.5 * (lo[s] + hi[s])
                mu[s] = new
            if done.all():
                return mu, it
        raise RuntimeError("sharded mu search did not reach tol within max_iter")
