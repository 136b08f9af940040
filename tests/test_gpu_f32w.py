"""Fused passes (G_loc, rho_k, the adjoint) of windows up to 40 bands on the warp-batched
kernel (k_point_f32w) against the oracle.

Each warp of the CTA inverts one frequency in FP32 with the matrix in its registers (the
one-warp Gauss-Jordan of the N(mu) kernel), then the CTA refines G P^+ (and P G for the
adjoint) once with an FP32-pair residual and forms the projections, frequency after
frequency.  GF_KERNEL=w32 leaves it the only mixed candidate for these passes (windows
above 40 bands take the FP32-pair kernels).  The mixed path's bounds apply: N 1e-7,
G_loc 1e-8 (the refinement; the contract is 1e-6), rho_k 1e-5, Sigma_bar 1e-8.
"""
import numpy as np
import pytest

import oracle
from paper_1111_2157_gb300 import synth
from tests.parity import check_system_set, make_gf, rel

pytestmark = pytest.mark.gpu
TOL = {"G_loc": 1e-8, "N": 1e-7, "dN_dmu": 1e-5, "n_corr": 1e-6, "rho": 1e-5}


@pytest.fixture
def warp_kernels(monkeypatch):
    monkeypatch.setenv("GF_KERNEL", "w32")


def ragged_systems():
    rng = synth.rng_for(99)
    systems = []
    for sidx, (m, nbs) in enumerate([(3, [1, 2, 7, 33, 5]), (5, [6, 17, 40]), (2, [16, 3, 24, 29])]):
        H = [synth.hamiltonian_dense(rng, 1, n, -4, 4, 0.3)[0] for n in nbs]
        P = [(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(n) for n in nbs]
        pole = synth.sigma_two_pole(rng, m, 3.0)
        systems.append(synth.System(H, P, pole, pole.sample(8.0 + 4 * sidx, 37), 8.0 + 4 * sidx, 1.0))
    return systems


CASES = {
    "d_toy": (lambda: [synth.d_toy().systems[0]], [0.3]),
    "ce_like_small": (lambda: [synth.ce_like(nk=5, n_iw=48).systems[0]], [0.1]),
    "window_13": (lambda: [synth.random_system(5, 4, 13, 3, 30, 10.0)], [0.05]),
    "window_29": (lambda: [synth.random_system(6, 3, 29, 5, 22, 10.0)], [0.15]),
    "window_35_split_rows": (lambda: [synth.random_system(8, 3, 35, 4, 21, 10.0)], [-0.1]),
    "ragged_three_systems": (ragged_systems, [0.2, -0.4, 1.1]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fused_passes_match_oracle(warp_kernels, name):
    make, mus = CASES[name]
    check_system_set(make(), mus, TOL, precision="mixed")


def test_the_warp_batched_kernel_runs(warp_kernels):
    s = synth.ce_like(nk=3, n_iw=16).systems[0]
    g = make_gf([s], precision="mixed")
    g.local([0.1])
    log = g.tuning_log()
    g.close()
    assert "one warp per matrix + CTA projections" in log, log


def test_tail_order_one(warp_kernels):
    check_system_set([synth.random_system(5, 4, 9, 3, 32, 10.0)], [0.05], TOL, precision="mixed",
                     tail_order=1)


def test_backward(warp_kernels):
    """Sigma_bar from the refined A_k = P G P^+ and B_k = P G^2 P^+; several k-points, a
    frequency count that leaves a partial last batch of warps."""
    s = synth.random_system(13, 3, 38, 4, 23, 6.0)
    rng = np.random.default_rng(1)
    gbar = rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)
    g = make_gf([s], precision="mixed")
    sb, mb = g.backward([0.2], gloc_bar=gbar.reshape(-1), n_bar=[0.7])
    g.close()
    sb_o, mb_o = oracle.get().backward(s.H, s.P, s.sigma, s.sigma_inf, s.beta, 0.2, gloc_bar=gbar,
                                       n_bar=0.7)
    assert rel(sb.cpu().numpy(), sb_o.reshape(-1)) < 1e-8
    assert abs(mb[0] - mb_o) / abs(mb_o) < 1e-6


def test_repeated_calls_are_bitwise_identical(warp_kernels):
    s = synth.ce_like(nk=6, n_iw=32).systems[0]
    g = make_gf([s], precision="mixed")
    a = g.evaluate([0.2], rho=True)
    b = g.evaluate([0.2], rho=True)
    g.close()
    assert np.array_equal(a["N"], b["N"]) and np.array_equal(a["dN_dmu"], b["dN_dmu"])
    assert bool((a["gloc"] == b["gloc"]).all()) and bool((a["rho"] == b["rho"]).all())


def test_ce_like_full_size_sampled(warp_kernels):
    s = synth.ce_like().systems[0]
    mu = 0.15
    g = make_gf([s], precision="mixed")
    out = g.evaluate([mu], gloc=True, rho=True)
    g.close()
    gl = out["gloc"].cpu().numpy().reshape(s.n_iw, s.m, s.m)
    rho = out["rho"].cpu().numpy().reshape(s.nk, 40, 40)
    o = oracle.get()
    idx = [0, 3, 511, 1023]
    assert rel(gl[idx], o.local(s.H, s.P, s.sigma, s.beta, mu, n_idx=idx)) < TOL["G_loc"]
    ks = [7, 500]
    r = o.density(s.H[ks], s.P[ks], s.sigma, s.sigma_inf, s.beta, mu, weights=np.full(2, 1e-3))
    assert rel(rho[ks], r["rho"]) < TOL["rho"]
