"""k-sharding over ranks: partition, all-reduced lattice sums and the mu search (gloo, CPU)."""
import socket

import numpy as np
import pytest
import torch.multiprocessing as tmp

import oracle
from tests import shard_worker
from paper_1111_2157_gb300 import shard


def test_partition_covers_every_k_once_and_balances_cost():
    rng = np.random.default_rng(5)
    nb = rng.integers(8, 130, size=1000)
    for ws in (1, 2, 3, 8):
        parts = shard.partition_k(nb, ws)
        assert parts[0][0] == 0 and parts[-1][1] == len(nb)
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        cost = np.array([np.sum(nb[a:b].astype(float) ** 3) for a, b in parts])
        assert cost.max() - cost.min() <= 2 * float(nb.max()) ** 3


def test_partition_with_fewer_k_than_ranks():
    parts = shard.partition_k([5, 7], 4)
    assert sum(b - a for a, b in parts) == 2
    assert parts[-1][1] == 2


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("world_size,parts", [(2, None), (3, None), (2, [(0, 24), (24, 24)])],
                         ids=["two_ranks", "three_ranks", "one_rank_empty"])
def test_sharded_lattice_sum_and_mu_search_match_single_process(tmp_path, world_size, parts):
    out = tmp_path / "rank0.npz"
    tmp.start_processes(shard_worker.run, args=(world_size, _free_port(), str(out), parts),
                        nprocs=world_size, join=True, start_method="spawn")
    r = np.load(out)
    if parts is None:
        assert r["k1"] > r["k0"] > -1 and r["k1"] < 24  # rank 0 holds a proper part of the k-points
    s = shard_worker.sharded_case()
    o = oracle.get()
    mu = float(r["mu"][0])
    full = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu, weights=s.weights, want_rho=False)
    assert abs(full["N"] - s.n_target) <= 2e-11
    assert abs(r["N"][0] - full["N"]) <= 1e-12
    assert abs(r["dN"][0] - full["dN_dmu"]) <= 1e-12 * abs(full["dN_dmu"])
    gl = o.local(s.H, s.P, s.sigma, s.beta, mu, weights=s.weights)
    assert np.max(np.abs(r["gloc"] - gl)) <= 1e-13 * np.max(np.abs(gl))
    mu_ref, _, _ = o.find_mu(s.H, s.P, s.sigma, s.sigma_inf, s.beta, s.n_target, -5.0, 5.0,
                             weights=s.weights, tol=1e-12)
    assert abs(mu - mu_ref) <= 1e-9


@pytest.mark.gpu
def test_two_rank_sharding_over_the_cuda_path():
    """Two ranks, each a CUDA context on its k-slice; the reduced sums match the oracle."""
    import tempfile
    from pathlib import Path
    with tempfile.TemporaryDirectory() as d:
        out = Path(d) / "rank0.npz"
        tmp.start_processes(shard_worker.run_gpu, args=(2, _free_port(), str(out)), nprocs=2,
                            join=True, start_method="spawn")
        r = np.load(out)
    s = shard_worker.sharded_case()
    o = oracle.get()
    mu = float(r["mu"][0])
    full = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu, weights=s.weights, want_rho=False)
    assert abs(full["N"] - s.n_target) <= 2e-11
    assert abs(r["N"][0] - full["N"]) <= 1e-12 * full["N"]
    gl = o.local(s.H, s.P, s.sigma, s.beta, mu, weights=s.weights)
    assert np.max(np.abs(r["gloc"].reshape(gl.shape) - gl)) <= 1e-12 * np.max(np.abs(gl))


def test_a_rank_that_drops_out_is_reported_not_waited_for(tmp_path):
    import multiprocessing as mp
    out = tmp_path / "rank0.txt"
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=shard_worker.run_dropout, args=(r, 2, port, str(out))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=60)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank was still waiting after 60 s"
    assert procs[1].exitcode != 0
    # rank 0 saw its collective fail (it neither hung nor got a result)
    assert out.exists() and out.read_text() != "no error"
