"""Mixed path (GF_PREC_MIXED) against the FP64 oracle.

The embedding and the Gauss-Jordan inverse run in single-word FP32; the Matsubara
sums, tail and mu search in FP64; the columns G P^+ and P G that G_loc and the
adjoint consume get one refinement step with an FP32-pair residual.

Contract: N within 1e-7 and G_loc within 1e-6 of the FP64 oracle (relative).
Bounds used here:
  N        1e-7 (the contract; FP32 inverses give about 1e-9)
  G_loc    1e-8 (100x inside the contract: the refined columns carry about
           (kappa 2^-24)^2 ~ 1e-10, and an unrefined FP32 projection, about
           kappa 2^-24 ~ 1e-6, fails it, so the bound checks the refinement)
  rho_k    1e-5, n_corr 1e-6, dN/dmu 1e-5 (unrefined FP32 inverses summed in FP64;
           no contract, regression bounds)
"""
import numpy as np
import pytest

import oracle
from paper_1111_2157_gb300 import synth
from tests.parity import check_system_set, make_gf, rel

pytestmark = pytest.mark.gpu
TOL = {"G_loc": 1e-8, "N": 1e-7, "dN_dmu": 1e-5, "n_corr": 1e-6, "rho": 1e-5}


def test_d_toy_full_size():
    check_system_set([synth.d_toy().systems[0]], [0.3], TOL, precision="mixed")


def test_ce_like_small():
    check_system_set([synth.ce_like(nk=5, n_iw=48).systems[0]], [0.1], TOL, precision="mixed")


def test_nio_like_small():
    """N_b = 96, m = 20, block AFM Sigma, beta = 40."""
    check_system_set([synth.nio_like(nk=3, n_iw=40).systems[0]], [0.2], TOL, precision="mixed")


def test_window_128():
    """The largest register tiles (N_b = 128), several frequencies per item."""
    check_system_set([synth.random_system(21, 2, 128, 12, 24, 20.0)], [0.1], TOL, precision="mixed")


def test_ragged_multi_system():
    """Windows from 1 to 64 bands, three systems, m from 2 to 5."""
    rng = synth.rng_for(4242)
    systems = []
    for sidx, (m, nbs) in enumerate([(3, [1, 2, 7, 33, 5]), (5, [6, 17, 40]), (2, [64, 3])]):
        H = [synth.hamiltonian_dense(rng, 1, n, -4, 4, 0.3)[0] for n in nbs]
        P = [(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(n) for n in nbs]
        pole = synth.sigma_two_pole(rng, m, 3.0)
        systems.append(synth.System(H, P, pole, pole.sample(8.0 + 4 * sidx, 40), 8.0 + 4 * sidx, 1.0))
    check_system_set(systems, [0.2, -0.4, 1.1], TOL, precision="mixed")


def test_window_above_the_register_tiles_falls_back_to_pairs():
    """N_b = 130 exceeds the FP32 register tiles: the FP32-pair kernels take it."""
    check_system_set([synth.random_system(12, 2, 130, 4, 3, 10.0)], [0.0], TOL, precision="mixed")


def test_complex64_inputs():
    s = synth.random_system(11, 4, 12, 4, 24, 10.0)
    r = synth.System(s.H.astype(np.complex64).astype(np.complex128),
                     s.P.astype(np.complex64).astype(np.complex128),
                     synth.PoleSigma(s.pole.sigma_inf.astype(np.complex64).astype(np.complex128),
                                     s.pole.p, s.pole.V),
                     s.sigma.astype(np.complex64).astype(np.complex128), s.beta, s.n_target)
    check_system_set([r], [0.1], TOL, precision="mixed", input_dtype="c64")


def test_tail_order_one():
    check_system_set([synth.random_system(5, 4, 9, 3, 32, 10.0)], [0.05], TOL, precision="mixed",
                     tail_order=1)


def test_backward():
    """Sigma_bar from the refined A_k = P G P^+ and B_k = P G^2 P^+; mu_bar also uses dN/dmu."""
    s = synth.random_system(13, 3, 10, 4, 20, 6.0)
    rng = np.random.default_rng(1)
    gbar = rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)
    g = make_gf([s], precision="mixed")
    sb, mb = g.backward([0.2], gloc_bar=gbar.reshape(-1), n_bar=[0.7])
    sb_o, mb_o = oracle.get().backward(s.H, s.P, s.sigma, s.sigma_inf, s.beta, 0.2, gloc_bar=gbar,
                                       n_bar=0.7)
    assert rel(sb.cpu().numpy(), sb_o.reshape(-1)) < 1e-8
    assert abs(mb[0] - mb_o) / abs(mb_o) < 1e-6


def test_find_mu():
    s = synth.d_toy(nk=32, n_iw=128).systems[0]
    g = make_gf([s], precision="mixed")
    mu, it = g.find_mu([s.n_target], 0.0, tol=1e-10, max_iter=50)
    n_o = oracle.get().density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, float(mu[0]), want_rho=False)["N"]
    assert abs(n_o - s.n_target) < 1e-7 * s.n_target


def test_repeated_calls_are_bitwise_identical():
    """Fixed reduction orders: the same inputs give the same bits."""
    s = synth.ce_like(nk=6, n_iw=32).systems[0]
    g = make_gf([s], precision="mixed")
    a = g.evaluate([0.2], rho=True)
    b = g.evaluate([0.2], rho=True)
    assert np.array_equal(a["N"], b["N"]) and np.array_equal(a["dN_dmu"], b["dN_dmu"])
    assert bool((a["gloc"] == b["gloc"]).all()) and bool((a["rho"] == b["rho"]).all())


def test_ce_like_full_size_sampled():
    s = synth.ce_like().systems[0]
    mu = 0.15
    g = make_gf([s], precision="mixed")
    out = g.evaluate([mu], gloc=True, rho=True)
    gl = out["gloc"].cpu().numpy().reshape(s.n_iw, s.m, s.m)
    rho = out["rho"].cpu().numpy().reshape(s.nk, 40, 40)
    o = oracle.get()
    idx = [0, 3, 511, 1023]
    assert rel(gl[idx], o.local(s.H, s.P, s.sigma, s.beta, mu, n_idx=idx)) < TOL["G_loc"]
    ks = [7, 500]
    r = o.density(s.H[ks], s.P[ks], s.sigma, s.sigma_inf, s.beta, mu, weights=np.full(2, 1e-3))
    assert rel(rho[ks], r["rho"]) < TOL["rho"]


def test_nio_like_full_size_sampled():
    """Full NiO-like size (N_k = 4096, N_b = 96, m = 20, N_w = 2048) in the launch configuration
    that bench.py times: G_loc at four frequencies over all k against the oracle; N_k = Tr rho_k
    at sampled k (every frequency) against the oracle's; N(mu) against the FP64 GPU path, which
    the FP64 tests hold to the oracle."""
    s = synth.nio_like().systems[0]
    mu = 0.1
    g = make_gf([s], precision="mixed")
    out = g.evaluate([mu], gloc=True, rho=True, occupation=True, n_corr=False)
    gl = out["gloc"].cpu().numpy().reshape(s.n_iw, s.m, s.m)
    o = oracle.get()
    idx = [0, 1, 1000, 2047]
    assert rel(gl[idx], o.local(s.H, s.P, s.sigma, s.beta, mu, n_idx=idx)) < TOL["G_loc"]
    ks = [11, 2047, 4000]
    rho = out["rho"].cpu().numpy().reshape(s.nk, 96, 96)
    r = o.density(s.H[ks], s.P[ks], s.sigma, s.sigma_inf, s.beta, mu, weights=np.full(3, 1.0))
    for j, k in enumerate(ks):
        n_k = float(np.trace(rho[k]).real)
        assert abs(n_k - float(np.trace(r["rho"][j]).real)) < 1e-7 * s.nb[0] / 2
    assert rel(rho[ks], r["rho"]) < TOL["rho"]
    g.close()
    g64 = make_gf([s], precision="fp64")
    n64, _ = g64.occupation([mu])
    assert abs(out["N"][0] - n64[0]) < TOL["N"] * n64[0]
