"""FP32-pair path (GF_PREC_PAIR: Gauss-Jordan in FP32 pairs on the FP32 pipes, FP64
reductions) against the FP64 oracle.

The FP32-pair arithmetic carries about 2^-48 relative precision per operation, so
every output is held to 1e-9 of the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1111_2157_gb300 import synth
from tests.parity import check_system_set, make_gf, rel

pytestmark = pytest.mark.gpu
TOL = {"G_loc": 1e-9, "N": 1e-9, "dN_dmu": 1e-9, "n_corr": 1e-9, "rho": 1e-9}


def test_d_toy_full_size():
    check_system_set([synth.d_toy().systems[0]], [0.3], TOL, precision="pair")


def test_ce_like_small():
    check_system_set([synth.ce_like(nk=5, n_iw=48).systems[0]], [0.1], TOL, precision="pair")


def test_nio_like_small():
    """N_b = 96, m = 20, block AFM Sigma, beta = 40."""
    check_system_set([synth.nio_like(nk=3, n_iw=40).systems[0]], [0.2], TOL, precision="pair")


def test_ragged_multi_system():
    rng = synth.rng_for(4242)
    systems = []
    for sidx, (m, nbs) in enumerate([(3, [1, 2, 7, 33, 5]), (5, [6, 17, 40]), (2, [64, 3])]):
        H = [synth.hamiltonian_dense(rng, 1, n, -4, 4, 0.3)[0] for n in nbs]
        P = [(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(n) for n in nbs]
        pole = synth.sigma_two_pole(rng, m, 3.0)
        systems.append(synth.System(H, P, pole, pole.sample(8.0 + 4 * sidx, 40), 8.0 + 4 * sidx, 1.0))
    check_system_set(systems, [0.2, -0.4, 1.1], TOL, precision="pair")


def test_large_window_matrix_in_global_memory():
    check_system_set([synth.random_system(12, 2, 130, 4, 3, 10.0)], [0.0], TOL, precision="pair")


def test_complex64_inputs():
    s = synth.random_system(11, 4, 12, 4, 24, 10.0)
    r = synth.System(s.H.astype(np.complex64).astype(np.complex128),
                     s.P.astype(np.complex64).astype(np.complex128),
                     synth.PoleSigma(s.pole.sigma_inf.astype(np.complex64).astype(np.complex128),
                                     s.pole.p, s.pole.V),
                     s.sigma.astype(np.complex64).astype(np.complex128), s.beta, s.n_target)
    check_system_set([r], [0.1], TOL, precision="pair", input_dtype="c64")


def test_tail_order_one():
    check_system_set([synth.random_system(5, 4, 9, 3, 32, 10.0)], [0.05], TOL, precision="pair",
                     tail_order=1)


def test_backward():
    s = synth.random_system(13, 3, 10, 4, 20, 6.0)
    rng = np.random.default_rng(1)
    gbar = rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)
    g = make_gf([s], precision="pair")
    sb, mb = g.backward([0.2], gloc_bar=gbar.reshape(-1), n_bar=[0.7])
    sb_o, mb_o = oracle.get().backward(s.H, s.P, s.sigma, s.sigma_inf, s.beta, 0.2, gloc_bar=gbar,
                                       n_bar=0.7)
    assert rel(sb.cpu().numpy(), sb_o.reshape(-1)) < 1e-9
    assert abs(mb[0] - mb_o) / abs(mb_o) < 1e-9


def test_find_mu():
    s = synth.d_toy(nk=32, n_iw=128).systems[0]
    g = make_gf([s], precision="pair")
    mu, it = g.find_mu([s.n_target], 0.0, tol=1e-10, max_iter=50)
    mu_o, _, _ = oracle.get().find_mu(s.H, s.P, s.sigma, s.sigma_inf, s.beta, s.n_target, -1, 1)
    assert abs(mu[0] - mu_o) < 1e-8


def test_ce_like_full_size_sampled():
    s = synth.ce_like().systems[0]
    mu = 0.15
    g = make_gf([s], precision="pair")
    gl = g.local([mu]).cpu().numpy().reshape(s.n_iw, s.m, s.m)
    rho, _ = g.density_matrix([mu])
    rho = rho.cpu().numpy().reshape(s.nk, 40, 40)
    o = oracle.get()
    idx = [0, 3, 511, 1023]
    assert rel(gl[idx], o.local(s.H, s.P, s.sigma, s.beta, mu, n_idx=idx)) < 1e-9
    ks = [7, 500]
    r = o.density(s.H[ks], s.P[ks], s.sigma, s.sigma_inf, s.beta, mu, weights=np.full(2, 1e-3))
    assert rel(rho[ks], r["rho"]) < 1e-9


def test_nio_like_full_size_sampled():
    """Full NiO-like size (N_k=4096, N_b=96, m=20, N_w=2048) in the launch configuration of
    bench.py --workload nio_like: G_loc at four frequencies over all k, and rho_k at two k."""
    s = synth.nio_like().systems[0]
    mu = 0.1
    g = make_gf([s], precision="pair")
    out = g.evaluate([mu], gloc=True, rho=True, occupation=False, n_corr=False)
    gl = out["gloc"].cpu().numpy().reshape(s.n_iw, s.m, s.m)
    o = oracle.get()
    idx = [0, 1, 1000, 2047]
    assert rel(gl[idx], o.local(s.H, s.P, s.sigma, s.beta, mu, n_idx=idx)) < 1e-9
    ks = [11, 4000]
    rho = out["rho"].cpu().numpy().reshape(s.nk, 96, 96)
    r = o.density(s.H[ks], s.P[ks], s.sigma, s.sigma_inf, s.beta, mu, weights=np.full(2, 0.5))
    assert rel(rho[ks], r["rho"]) < 1e-9
