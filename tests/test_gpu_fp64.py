"""FP64 CUDA path against the FP64 oracle, element by element (tolerance 1e-10 relative)."""
import numpy as np
import pytest

import oracle
from paper_1111_2157_gb300 import synth
from tests.parity import make_gf, oracle_all, pack, rel, split_sys

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _check_system_set(systems, mus, tail_order=2, input_dtype="c128"):
    g = make_gf(systems, tail_order=tail_order, input_dtype=input_dtype)
    gl = g.local(mus).cpu().numpy()
    n, dn = g.occupation(mus)
    rho, nc = g.density_matrix(mus)
    rho = rho.cpu().numpy()
    gls = split_sys(gl, systems, lambda s: s.n_iw * s.m * s.m)
    rhos = split_sys(rho, systems, lambda s: int(np.sum(s.nb.astype(np.int64) ** 2)))
    for i, s in enumerate(systems):
        r, glo = oracle_all(s, mus[i], tail_order=tail_order)
        assert rel(gls[i], glo.reshape(-1)) < TOL, f"G_loc system {i}"
        assert abs(n[i] - r["N"]) / max(1.0, abs(r["N"])) < TOL, f"N system {i}"
        assert abs(dn[i] - r["dN_dmu"]) / abs(r["dN_dmu"]) < TOL, f"dN/dmu system {i}"
        assert abs(nc[i] - r["n_corr"]) / max(1.0, abs(r["n_corr"])) < TOL, f"n_corr system {i}"
        assert rel(rhos[i], pack(r["rho"])) < TOL, f"rho system {i}"
    g.close()


def test_d_toy_full_size():
    s = synth.d_toy().systems[0]
    _check_system_set([s], [0.3])


def test_ce_like_small_spans_tiles():
    s = synth.ce_like(nk=5, n_iw=48).systems[0]
    _check_system_set([s], [0.1])


def test_ragged_multi_system():
    rng = synth.rng_for(777)
    systems = []
    for sidx, (m, nbs) in enumerate([(3, [1, 2, 7, 33, 5]), (5, [6, 17, 40]), (2, [64, 3])]):
        H = [synth.hamiltonian_dense(rng, 1, n, -4, 4, 0.3)[0] for n in nbs]
        P = [rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)) for n in nbs]
        P = [p / np.sqrt(n) for p, n in zip(P, nbs)]
        pole = synth.sigma_two_pole(rng, m, 3.0)
        systems.append(synth.System(H, P, pole, pole.sample(8.0 + 4 * sidx, 40), 8.0 + 4 * sidx, 1.0))
    _check_system_set(systems, [0.2, -0.4, 1.1])


def test_tail_order_one():
    s = synth.random_system(5, 4, 9, 3, 32, 10.0)
    _check_system_set([s], [0.05], tail_order=1)


def test_single_band_single_orbital():
    s = synth.random_system(6, 3, 1, 1, 16, 5.0)
    _check_system_set([s], [0.0])


def test_more_orbitals_than_bands():
    rng = synth.rng_for(8)
    nk, nb, m = 3, 2, 5
    H = synth.hamiltonian_dense(rng, nk, nb, -2, 2, 0.3)
    P = (rng.standard_normal((nk, m, nb)) + 1j * rng.standard_normal((nk, m, nb))) * 0.4
    pole = synth.sigma_two_pole(rng, m, 2.0)
    s = synth.System(H, P, pole, pole.sample(6.0, 24), 6.0, 1.0)
    _check_system_set([s], [0.3])


def test_mu_far_outside_band():
    s = synth.random_system(9, 3, 6, 2, 32, 10.0)
    _check_system_set([s], [40.0])


def test_single_frequency():
    s = synth.random_system(10, 4, 8, 3, 1, 10.0)
    _check_system_set([s], [0.1])


def test_complex64_inputs_are_upcast():
    s = synth.random_system(11, 4, 12, 4, 24, 10.0)
    rounded = synth.System(s.H.astype(np.complex64).astype(np.complex128),
                           s.P.astype(np.complex64).astype(np.complex128),
                           synth.PoleSigma(s.pole.sigma_inf.astype(np.complex64).astype(np.complex128),
                                           s.pole.p, s.pole.V),
                           s.sigma.astype(np.complex64).astype(np.complex128), s.beta, s.n_target)
    _check_system_set([rounded], [0.1], input_dtype="c64")


def test_large_window_matrix_in_global_memory():
    """N_b = 130 does not fit in shared memory: the matrix lives in a global scratch slice."""
    s = synth.random_system(12, 2, 130, 4, 3, 10.0)
    _check_system_set([s], [0.0])


def test_find_mu_matches_oracle():
    s = synth.d_toy(nk=32, n_iw=128).systems[0]
    g = make_gf([s])
    mu, it = g.find_mu([s.n_target], 0.0, tol=1e-11, max_iter=50)
    n, _ = g.occupation(mu)
    assert abs(n[0] - s.n_target) <= 1e-11
    mu_o, n_o, _ = oracle.get().find_mu(s.H, s.P, s.sigma, s.sigma_inf, s.beta, s.n_target, -1, 1)
    # N is strictly increasing: equal N means equal mu to |dN| / (dN/dmu)
    assert abs(mu[0] - mu_o) < 1e-8
    assert it < 15


def test_backward_matches_oracle():
    s = synth.random_system(13, 3, 10, 4, 20, 6.0)
    rng = np.random.default_rng(1)
    gbar = rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)
    g = make_gf([s])
    sb, mb = g.backward([0.2], gloc_bar=gbar.reshape(-1), n_bar=[0.7])
    sb_o, mb_o = oracle.get().backward(s.H, s.P, s.sigma, s.sigma_inf, s.beta, 0.2, gloc_bar=gbar,
                                       n_bar=0.7)
    assert rel(sb.cpu().numpy(), sb_o.reshape(-1)) < TOL
    assert abs(mb[0] - mb_o) / abs(mb_o) < TOL
    sb2, mb2 = g.backward([0.2], gloc_bar=None, n_bar=[1.0])
    sb2_o, mb2_o = oracle.get().backward(s.H, s.P, s.sigma, s.sigma_inf, s.beta, 0.2, n_bar=1.0)
    assert rel(sb2.cpu().numpy(), sb2_o.reshape(-1)) < TOL
    assert abs(mb2[0] - mb2_o) / abs(mb2_o) < TOL


def test_singular_point_reports_error():
    """A = 0 exactly at w_0 (Sigma(i w_0) = i w_0 + mu, H = 0, P = 1): GF_ESINGULAR, no fault."""
    from paper_1111_2157_gb300.gf import GFError, GF_ESINGULAR
    beta, mu = 10.0, 0.25
    w0 = np.pi / beta
    H = np.zeros((1, 1, 1), np.complex128)
    P = np.ones((1, 1, 1), np.complex128)
    sig = np.full((2, 1, 1), 1j * w0 + mu)
    pole = synth.PoleSigma(np.zeros((1, 1), np.complex128), np.zeros(0), np.zeros((0, 1)))
    s = synth.System(H, P, pole, sig, beta, 0.5)
    g = make_gf([s])
    with pytest.raises(GFError) as ei:
        g.occupation([mu])
    assert ei.value.status == GF_ESINGULAR
    # the context stays usable
    g.set_sigma(np.zeros((2, 1, 1), np.complex128), np.zeros((1, 1), np.complex128))
    n, _ = g.occupation([mu])
    assert np.isfinite(n[0])


def test_state_error_before_sigma():
    from paper_1111_2157_gb300.gf import GFError, GF_ESTATE, GreensFunction
    g = GreensFunction(4, 2, 8, 10.0, n_k=3)
    g.set_hamiltonian(np.zeros((3, 4, 4), np.complex128))
    with pytest.raises(GFError) as ei:
        g.occupation([0.0])
    assert ei.value.status == GF_ESTATE


def test_ce_like_full_size_sampled():
    """Ce-like workload at full size (1000 k, N_b=40, m=14, 1024 w): G_loc at sampled
    frequencies over all k and rho_k at sampled k over all frequencies, one by one on the oracle."""
    s = synth.ce_like().systems[0]
    mu = 0.15
    g = make_gf([s])
    gl = g.local([mu]).cpu().numpy().reshape(s.n_iw, s.m, s.m)
    rho, nc = g.density_matrix([mu])
    rho = rho.cpu().numpy().reshape(s.nk, 40, 40)
    n, dn = g.occupation([mu])
    o = oracle.get()
    idx = [0, 1, 17, 511, 1023]
    glo = o.local(s.H, s.P, s.sigma, s.beta, mu, n_idx=idx)
    assert rel(gl[idx], glo) < TOL
    ks = [0, 123, 999]
    r = o.density(s.H[ks], s.P[ks], s.sigma, s.sigma_inf, s.beta, mu, weights=np.full(3, 1.0 / s.nk))
    assert rel(rho[ks], r["rho"]) < TOL
    # N = sum_k w_k Tr rho_k holds for the GPU's own outputs
    assert abs(n[0] - np.trace(rho, axis1=1, axis2=2).real.sum() / s.nk) < 1e-10 * n[0]


def test_evaluate_fused_pass():
    s = synth.ce_like(nk=4, n_iw=40).systems[0]
    mu = 0.1
    g = make_gf([s])
    out = g.evaluate([mu])
    r, glo = oracle_all(s, mu)
    assert rel(out["gloc"].cpu().numpy(), glo.reshape(-1)) < TOL
    assert rel(out["rho"].cpu().numpy(), r["rho"].reshape(-1)) < TOL
    assert abs(out["N"][0] - r["N"]) < TOL * r["N"]
    assert abs(out["dN_dmu"][0] - r["dN_dmu"]) < TOL * r["dN_dmu"]
    assert abs(out["n_corr"][0] - r["n_corr"]) < TOL * r["n_corr"]
    only_n = g.evaluate([mu], gloc=False, rho=False, n_corr=False)
    assert only_n["gloc"] is None and only_n["rho"] is None
    assert abs(only_n["N"][0] - r["N"]) < TOL * r["N"]
    st = g.stats()
    assert st["points"] == s.nk * s.n_iw and st["kernel_ms"] > 0 and st["flops"] > 0


@pytest.mark.parametrize("beta", [0.5, 400.0])
def test_extreme_temperatures(beta):
    """beta = 0.5 (hot: the tail terms dominate) and beta = 400 (cold: w_0 = 0.008 eV)."""
    s = synth.random_system(41, 4, 10, 3, 96, beta)
    _check_system_set([s], [0.2])


def test_mu_search_iteration_cap_reports_non_convergence():
    from paper_1111_2157_gb300.gf import GFError
    s = synth.random_system(42, 3, 8, 3, 32, 10.0)
    g = make_gf([s])
    with pytest.raises(GFError, match="ENOTCONV"):
        g.find_mu([s.n_target], mu0=3.0, tol=1e-14, max_iter=1)
    mu, it = g.find_mu([s.n_target], mu0=3.0, tol=1e-10)  # the context is still usable
    assert it > 1
