"""Rank body of the k-sharding test: each gloo rank runs the oracle on its k-slice."""
import datetime

import numpy as np
import torch.distributed as dist

import oracle
from paper_1111_2157_gb300 import shard, synth


def sharded_case():
    """Ragged one-system case: N_b(k) in [3, 9], m = 3, 24 k-points, 48 frequencies."""
    rng = synth.rng_for(20240)
    m, beta, n_iw, nk = 3, 15.0, 48, 24
    nbs = rng.integers(3, 10, size=nk)
    H = [synth.hamiltonian_dense(rng, 1, int(n), -4.0, 4.0, 0.3)[0] for n in nbs]
    P = [synth.projectors(rng, 1, int(n), m)[0] for n in nbs]
    pole = synth.sigma_two_pole(rng, m, 3.0)
    w = rng.uniform(0.5, 1.5, size=nk)
    w /= w.sum()
    return synth.System(H, P, pole, pole.sample(beta, n_iw), beta, float(np.mean(nbs)) / 2.0,
                        weights=w)


def oracle_slice_evaluator(o, s, k0, k1):
    m, n_iw = s.m, s.n_iw

    def evaluate(mu, gloc):
        if k1 == k0:
            g = np.zeros((n_iw, m, m), np.complex128) if gloc else None
            return g, [0.0], [0.0]
        H, P, w = s.H[k0:k1], s.P[k0:k1], s.weights[k0:k1]
        r = o.density(H, P, s.sigma, s.sigma_inf, s.beta, float(mu[0]), weights=w, want_rho=False)
        g = o.local(H, P, s.sigma, s.beta, float(mu[0]), weights=w) if gloc else None
        return g, [r["N"]], [r["dN_dmu"]]

    return evaluate


def run(rank, world_size, port, out_path, parts=None):
    """parts: explicit k-slices per rank (e.g. one left empty), else the cost-balanced ones."""
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world_size, timeout=datetime.timedelta(seconds=60))
    try:
        s = sharded_case()
        k0, k1 = (parts or shard.partition_k(s.nb, world_size))[rank]
        lat = shard.ShardedLattice(oracle_slice_evaluator(oracle.get(), s, k0, k1))
        mu, evals = lat.find_mu(s.n_target, mu0=0.0, tol=1e-11)
        g, n, dn = lat.evaluate(mu, gloc=True)
        if rank == 0:
            np.savez(out_path, mu=mu, evals=evals, gloc=g.numpy(), N=n, dN=dn, k0=k0, k1=k1)
    finally:
        dist.destroy_process_group()


def run_gpu(rank, world_size, port, out_path):
    """Each rank builds a GreensFunction for its k-slice (weights of the full set) on cuda:0;
    gloo all-reduces host copies of the partial sums."""
    import torch
    from paper_1111_2157_gb300 import gf as gfm
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world_size, timeout=datetime.timedelta(seconds=120))
    try:
        s = sharded_case()
        k0, k1 = shard.partition_k(s.nb, world_size)[rank]
        nb = s.nb[k0:k1]
        g = gfm.GreensFunction(nb, s.m, s.n_iw, s.beta, k_weight=s.weights[k0:k1])
        g.set_hamiltonian(np.concatenate([h.reshape(-1) for h in s.H[k0:k1]]))
        g.set_projectors(np.concatenate([p.reshape(-1) for p in s.P[k0:k1]]))
        g.set_sigma(s.sigma, s.sigma_inf)
        base = shard.greens_function_evaluator(g)
        lat = shard.ShardedLattice(lambda mu, gl: _to_host(base(mu, gl)))
        mu, evals = lat.find_mu(s.n_target, mu0=0.0, tol=1e-11)
        gloc, n, dn = lat.evaluate(mu, gloc=True)
        torch.cuda.synchronize()
        if rank == 0:
            np.savez(out_path, mu=mu, evals=evals, gloc=gloc.numpy(), N=n, dN=dn)
        g.close()
    finally:
        dist.destroy_process_group()


def _to_host(r):
    g, n, dn = r
    return (None if g is None else g.cpu()), n, dn


def run_dropout(rank, world_size, port, out_path):
    """Rank 1 fails before its first evaluation; rank 0's all-reduce must end with an error
    within the process-group timeout instead of waiting forever."""
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world_size, timeout=datetime.timedelta(seconds=5))
    s = sharded_case()
    k0, k1 = shard.partition_k(s.nb, world_size)[rank]
    if rank == 1:
        raise RuntimeError("rank 1 drops out")
    lat = shard.ShardedLattice(oracle_slice_evaluator(oracle.get(), s, k0, k1))
    try:
        lat.evaluate([0.0], gloc=False)
        outcome = "no error"
    except Exception as e:  # the collective reports the lost peer
        outcome = type(e).__name__
    with open(out_path, "w") as f:
        f.write(outcome)
