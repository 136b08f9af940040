"""Pins of the pole-path oracle (oracle/pole.py, Sec. 3.3) against independent routes.

The Matsubara-sum oracle (LU per (k, i w_n), itself pinned in test_oracle_pins)
fixes G_loc exactly and, extrapolated in N_w, rho_k, N and n_corr; central
differences fix dN/dmu; band eigenvalues fix the pole-free limit.
"""
import numpy as np

import oracle
from oracle import pole
from paper_1111_2157_gb300 import synth


def _ragged(seed=31, nk=4, m=3, beta=8.0):
    rng = synth.rng_for(seed)
    nbs = [5, 8, 6, 7][:nk]
    H = [synth.hamiltonian_dense(rng, 1, n, -3.0, 3.0, 0.4)[0] for n in nbs]
    P = [synth.projectors(rng, 1, n, m)[0] for n in nbs]
    ps = synth.sigma_two_pole(rng, m, 3.0)
    w = rng.uniform(0.5, 1.5, size=nk)
    return H, P, ps, w / w.sum(), beta


def test_local_equals_matsubara_oracle():
    H, P, ps, w, beta = _ragged()
    mu, n_iw = 0.27, 40
    got = pole.local(H, P, ps.sigma_inf, ps.p, ps.V, beta, mu, n_iw, weights=w)
    ref = oracle.get().local(H, P, ps.sample(beta, n_iw), beta, mu, weights=w)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_density_is_the_infinite_matsubara_limit():
    """Richardson (8 X(800) - X(400)) / 7 of the truncated sums removes the N_w^-3 term."""
    H, P, ps, w, beta = _ragged(beta=6.0)
    mu = 0.3
    ex = pole.density(H, P, ps.sigma_inf, ps.p, ps.V, beta, mu, weights=w)
    o = oracle.get()
    r = {n: o.density(H, P, ps.sample(beta, n), ps.sigma_inf, beta, mu, weights=w) for n in (400, 800)}
    rich = lambda key: (8 * r[800][key] - r[400][key]) / 7  # noqa: E731
    assert abs(rich("N") - ex["N"]) < 1e-8
    assert abs(rich("n_corr") - ex["n_corr"]) < 1e-8
    for k in range(len(H)):
        rr = (8 * r[800]["rho"][k] - r[400]["rho"][k]) / 7
        assert np.max(np.abs(rr - ex["rho"][k])) < 1e-8


def test_dn_dmu_central_difference():
    H, P, ps, w, beta = _ragged(seed=32, beta=10.0)
    mu, h = 0.1, 1e-5
    d = pole.density(H, P, ps.sigma_inf, ps.p, ps.V, beta, mu, weights=w)["dN_dmu"]
    up = pole.density(H, P, ps.sigma_inf, ps.p, ps.V, beta, mu + h, weights=w)["N"]
    dn = pole.density(H, P, ps.sigma_inf, ps.p, ps.V, beta, mu - h, weights=w)["N"]
    fd = (up - dn) / (2 * h)
    assert d > 0
    assert abs(d - fd) <= 1e-7 * abs(fd)


def test_pole_free_limit_is_the_band_fermi_sum():
    H, P, ps, w, beta = _ragged(seed=33)
    mu = -0.4
    m = P[0].shape[0]
    zero = np.zeros((m, m), np.complex128)
    got = pole.density(H, P, zero, np.zeros(0), np.zeros((0, m)), beta, mu, weights=w)
    ref = sum(w[k] * np.sum(pole.fermi(np.linalg.eigvalsh(H[k]) - mu, beta)) for k in range(len(H)))
    assert abs(got["N"] - ref) < 1e-13


def test_find_mu_hits_the_target():
    H, P, ps, w, beta = _ragged(seed=34)
    target = 3.0
    mu = pole.find_mu(H, P, ps.sigma_inf, ps.p, ps.V, beta, target, -10.0, 10.0, weights=w)
    n = pole.density(H, P, ps.sigma_inf, ps.p, ps.V, beta, mu, weights=w)["N"]
    assert abs(n - target) < 1e-11


def test_spectral_without_self_energy_is_the_band_lorentzian_sum():
    H, P, ps, w, beta = _ragged(seed=35)
    m = P[0].shape[0]
    mu, eta = 0.2, 0.05
    eps = np.linspace(-4, 4, 41)
    dos, pdos = pole.spectral(H, P, np.zeros((m, m)), np.zeros(0), np.zeros((0, m)), mu, eps, eta, w)
    ref = np.zeros_like(eps)
    pref = np.zeros((len(eps), m))
    for k in range(len(H)):
        e, U = np.linalg.eigh(H[k])
        lor = (eta / np.pi) / ((eps[:, None] + mu - e[None, :]) ** 2 + eta ** 2)
        ref += w[k] * lor.sum(axis=1)
        pref += w[k] * lor @ (np.abs(P[k] @ U) ** 2).T
    assert np.max(np.abs(dos - ref)) < 1e-12
    assert np.max(np.abs(pdos - pref)) < 1e-12


def test_spectral_weight_integrates_to_the_band_count():
    """A Lorentzian integrates to 1: int D = sum_k w_k N_b(k) up to the tails outside the grid."""
    H, P, ps, w, beta = _ragged(seed=36)
    eta, L = 0.05, 400.0
    eps = np.linspace(-L, L, 400001)
    dos, pdos = pole.spectral(H, P, ps.sigma_inf, ps.p, ps.V, 0.0, eps, eta, w)
    total = np.trapezoid(dos, eps)
    nb = sum(w[k] * H[k].shape[0] for k in range(len(H)))
    tail = 2 * eta / (np.pi * (L - 20.0)) * nb
    assert abs(total - nb) < tail + 1e-6
    # with orthonormal projector rows the orbital weights add up to m
    assert abs(np.trapezoid(pdos.sum(axis=1), eps) - P[0].shape[0]) < tail * 2 + 1e-6


def test_energy_without_self_energy():
    """Sigma = 0: e_ps + mu N = Tr(H rho) summed over k."""
    H, P, ps, w, beta = _ragged(seed=37)
    m = P[0].shape[0]
    mu = 0.15
    z = (np.zeros((m, m)), np.zeros(0), np.zeros((0, m)))
    hks, eps_sum = pole.energy(H, P, *z, beta, mu, w)
    n = pole.density(H, P, *z, beta, mu, weights=w)["N"]
    assert abs(eps_sum + mu * n - hks) < 1e-12


def test_energy_h_ks_from_the_matsubara_density():
    """Tr(H rho) with rho from the Matsubara-sum oracle (Richardson in N_w) matches."""
    H, P, ps, w, beta = _ragged(seed=38, beta=6.0)
    mu = 0.1
    hks, _ = pole.energy(H, P, ps.sigma_inf, ps.p, ps.V, beta, mu, w)
    o = oracle.get()
    r = {n: o.density(H, P, ps.sample(beta, n), ps.sigma_inf, beta, mu, weights=w) for n in (400, 800)}
    ref = 0.0
    for k in range(len(H)):
        rho = (8 * r[800]["rho"][k] - r[400]["rho"][k]) / 7
        ref += w[k] * np.trace(H[k] @ rho).real
    assert abs(hks - ref) < 1e-8
