"""Low-rank (eigenbasis / Woodbury) algorithm on the GPU against the oracle's direct inverse."""
import numpy as np
import pytest

import oracle
from paper_1111_2157_gb300 import synth
from tests.parity import check_system_set, make_gf, rel

pytestmark = pytest.mark.gpu

TOL = {"G_loc": 1e-10, "N": 1e-10, "dN_dmu": 1e-10, "n_corr": 1e-10, "rho": 1e-10}


def test_ce_like_small_all_outputs():
    s = synth.ce_like(nk=7, n_iw=40).systems[0]
    check_system_set([s], [0.4], TOL, lowrank=True)


def _more_orbitals_than_bands(nk=3, nb=2, m=5, n_iw=24):
    rng = synth.rng_for(8)
    H = synth.hamiltonian_dense(rng, nk, nb, -2, 2, 0.3)
    P = (rng.standard_normal((nk, m, nb)) + 1j * rng.standard_normal((nk, m, nb))) * 0.4
    pole = synth.sigma_two_pole(rng, m, 2.0)
    return synth.System(H, P, pole, pole.sample(12.0, n_iw), 12.0, 1.0)


def test_ragged_systems_and_edge_shapes():
    systems = [synth.random_system(51, 5, 9, 3, 24, 12.0),
               synth.random_system(52, 3, 1, 1, 24, 12.0),       # N_b = m = 1
               _more_orbitals_than_bands()]                      # m > N_b
    check_system_set(systems, [0.2, -0.5, 1.0], TOL, lowrank=True)


def test_equals_direct_gpu_path_bitwise_close():
    s = synth.ce_like(nk=12, n_iw=64, nb=64, m=14).systems[0]
    gd = make_gf([s])
    gl = make_gf([s], lowrank=True)
    mu = 0.1
    a = gd.evaluate(mu)
    b = gl.evaluate(mu)
    assert rel(b["gloc"].cpu().numpy(), a["gloc"].cpu().numpy()) < 1e-11
    assert rel(b["rho"].cpu().numpy(), a["rho"].cpu().numpy()) < 1e-11
    assert abs(b["N"][0] - a["N"][0]) < 1e-11 * a["N"][0]
    assert abs(b["dN_dmu"][0] - a["dN_dmu"][0]) < 1e-11 * a["dN_dmu"][0]
    assert gl.stats()["flops"] < 0.5 * gd.stats()["flops"]


def test_find_mu_and_backward():
    s = synth.ce_like(nk=5, n_iw=32).systems[0]
    g = make_gf([s], lowrank=True)
    mu, it = g.find_mu(s.n_target, 0.0, tol=1e-10)
    r = oracle.get().density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu[0], want_rho=False)
    assert abs(r["N"] - s.n_target) < 1e-9
    rng = np.random.default_rng(3)
    gbar = rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)
    sb, mb = g.backward(mu, gloc_bar=gbar.reshape(-1), n_bar=[0.7])
    sref, mref = oracle.get().backward(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu[0],
                                       gloc_bar=gbar, n_bar=0.7)
    assert rel(sb.cpu().numpy(), sref.reshape(-1)) < 1e-10
    assert abs(mb[0] - mref) < 1e-10 * abs(mref)


def test_new_hamiltonian_refreshes_the_eigenbasis():
    s1 = synth.random_system(61, 4, 10, 3, 16, 10.0)
    s2 = synth.random_system(62, 4, 10, 3, 16, 10.0)
    g = make_gf([s1], lowrank=True)
    g.occupation(0.0)
    g.set_hamiltonian(np.concatenate([h.reshape(-1) for h in s2.H]))
    g.set_projectors(np.concatenate([p.reshape(-1) for p in s2.P]))
    g.set_sigma(s2.sigma, s2.sigma_inf)
    n, _ = g.occupation(0.0)
    r = oracle.get().density(s2.H, s2.P, s2.sigma, s2.sigma_inf, s2.beta, 0.0, want_rho=False)
    assert abs(n[0] - r["N"]) < 1e-10 * r["N"]


@pytest.mark.parametrize("case", ["ce_like", "ragged"])
def test_mixed_precision_band_sums(case):
    """GF_PREC_MIXED with GF_FLAG_LOWRANK: FP32-pair band sums, FP64 m x m algebra."""
    if case == "ce_like":
        systems = [synth.ce_like(nk=6, n_iw=40).systems[0]]
        mus = [0.4]
    else:
        systems = [synth.random_system(71, 5, 9, 3, 24, 12.0), synth.random_system(72, 4, 30, 20, 24, 20.0)]
        mus = [0.2, -0.3]
    check_system_set(systems, mus, {"G_loc": 1e-9, "N": 1e-9, "dN_dmu": 1e-9, "n_corr": 1e-9, "rho": 1e-9},
                     precision="mixed", lowrank=True)


def test_graph_replay_of_the_low_rank_mu_search():
    """Graph replay gives the same bits as ordinary launches; a new H refreshes the eigenbasis."""
    systems = synth.batched(n_iw=24, nk_scale=0.002).systems[:3]
    g0 = make_gf(systems, lowrank=True)
    g1 = make_gf(systems, lowrank=True, graph=True)
    for mus in ([0.0, 0.1, 0.2], [0.3, -0.2, 0.05], [0.0, 0.1, 0.2]):
        a = g0.occupation(mus)
        b = g1.occupation(mus)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # a new Hamiltonian (same windows, shifted diagonals) must refresh the eigenbasis under replay
    flat = np.concatenate([(np.asarray(h) + 0.3 * np.eye(h.shape[0])).reshape(-1)
                           for s in systems for h in s.H])
    g0.set_hamiltonian(flat)
    g1.set_hamiltonian(flat)
    a = g0.occupation([0.0, 0.1, 0.2])
    b = g1.occupation([0.0, 0.1, 0.2])
    assert np.array_equal(a[0], b[0])
    shifted = [synth.System([np.asarray(h) + 0.3 * np.eye(h.shape[0]) for h in s.H], s.P, s.pole,
                            s.sigma, s.beta, s.n_target) for s in systems]
    r = oracle.get().density(shifted[0].H, shifted[0].P, shifted[0].sigma, shifted[0].sigma_inf,
                             shifted[0].beta, 0.0, want_rho=False)
    assert abs(b[0][0] - r["N"]) < 1e-10 * r["N"]


def test_ce_like_full_size_sampled():
    """Full Ce-like size in the low-rank mode: G_loc at four frequencies over all k and rho_k at
    two k against the oracle; N against the direct GPU path (itself checked against the oracle)."""
    s = synth.ce_like().systems[0]
    mu = 0.15
    g = make_gf([s], lowrank=True)
    out = g.evaluate([mu], gloc=True, rho=True, occupation=True, n_corr=False)
    gl = out["gloc"].cpu().numpy().reshape(s.n_iw, s.m, s.m)
    o = oracle.get()
    idx = [0, 3, 511, 1023]
    assert rel(gl[idx], o.local(s.H, s.P, s.sigma, s.beta, mu, n_idx=idx)) < 1e-10
    ks = [7, 500]
    rho = out["rho"].cpu().numpy().reshape(s.nk, 40, 40)
    r = o.density(s.H[ks], s.P[ks], s.sigma, s.sigma_inf, s.beta, mu, weights=np.full(2, 0.5))
    assert rel(rho[ks], r["rho"]) < 1e-10
    gd = make_gf([s])
    nd, _ = gd.occupation([mu])
    assert abs(out["N"][0] - nd[0]) < 1e-12 * nd[0]


def test_mixed_precision_backward_and_mu_search():
    s = synth.ce_like(nk=5, n_iw=32).systems[0]
    g = make_gf([s], precision="mixed", lowrank=True)
    mu, it = g.find_mu(s.n_target, 0.0, tol=1e-10)
    r = oracle.get().density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu[0], want_rho=False)
    assert abs(r["N"] - s.n_target) < 1e-9
    rng = np.random.default_rng(4)
    gbar = rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)
    sb, mb = g.backward(mu, gloc_bar=gbar.reshape(-1), n_bar=[0.7])
    sref, mref = oracle.get().backward(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu[0],
                                       gloc_bar=gbar, n_bar=0.7)
    assert rel(sb.cpu().numpy(), sref.reshape(-1)) < 1e-9
    assert abs(mb[0] - mref) < 1e-9 * abs(mref)
