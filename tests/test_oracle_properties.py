"""Property checks of the oracle over random shapes and seeds (hypothesis, CPU)."""
import numpy as np
import pytest

import oracle
from oracle import pole
from paper_1111_2157_gb300 import synth

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


@settings(max_examples=25, deadline=None)
@given(seed=st.integers(0, 10_000), nk=st.integers(1, 4), nb=st.integers(1, 9), m=st.integers(1, 4),
       beta=st.sampled_from([2.0, 10.0, 40.0]), mu=st.floats(-3.0, 3.0))
def test_density_invariants(seed, nk, nb, m, beta, mu):
    """rho_k Hermitian with eigenvalues in [0, 1] up to the truncation remainder, 0 <= N <= N_b,
    dN/dmu > 0, n_corr <= trace of P P^+ (the Matsubara sum at 512 frequencies)."""
    m = min(m, nb)
    s = synth.random_system(seed, nk, nb, m, 512, beta)
    r = oracle.get().density(s.H, s.P, s.sigma, s.sigma_inf, beta, mu)
    for rho in r["rho"]:
        assert np.max(np.abs(rho - np.conj(rho.T))) < 1e-12
        ev = np.linalg.eigvalsh(rho)
        assert ev.min() > -2e-3 and ev.max() < 1 + 2e-3
    assert -1e-3 <= r["N"] <= nb + 1e-3
    assert r["dN_dmu"] > 0
    tr_pp = np.mean([np.trace(p @ np.conj(p.T)).real for p in s.P])
    assert r["n_corr"] <= tr_pp + 1e-3


@settings(max_examples=25, deadline=None)
@given(seed=st.integers(0, 10_000), nb=st.integers(1, 8), m=st.integers(1, 4),
       n=st.integers(0, 200), mu=st.floats(-3.0, 3.0))
def test_green_matches_the_pseudo_hamiltonian_resolvent(seed, nb, m, n, mu):
    """For pole-form Sigma, G(k, i w) from the LU inverse equals the band block of
    [(i w + mu) - H_ps]^{-1} of Sec. 3.3, an independent construction."""
    m = min(m, nb)
    s = synth.random_system(seed, 1, nb, m, n + 1, 10.0)
    wn = (2 * n + 1) * np.pi / s.beta
    G = oracle.get().green(s.H[0], s.P[0], s.sigma[n], wn, mu)
    Hps = pole.pseudo_hamiltonian(s.H[0], s.P[0], s.pole.sigma_inf, s.pole.p, s.pole.V, mu)
    R = np.linalg.inv((1j * wn + mu) * np.eye(Hps.shape[0]) - Hps)[:nb, :nb]
    assert np.max(np.abs(G - R)) <= 1e-11 * max(1.0, np.max(np.abs(R)))


@settings(max_examples=25, deadline=None)
@given(seed=st.integers(0, 10_000), nk=st.integers(1, 3), nb=st.integers(1, 8), m=st.integers(1, 4),
       beta=st.sampled_from([2.0, 10.0, 40.0]), mu=st.floats(-3.0, 3.0))
def test_pole_density_invariants(seed, nk, nb, m, beta, mu):
    """Pole path (Sec. 3.3): rho_k is the band block of n_F(H_ps - mu), a compression of a matrix
    with spectrum in [0, 1], so it is Hermitian with eigenvalues in [0, 1] exactly (no truncation
    remainder); dN/dmu >= 0 and N rises with mu; the Lorentzian DOS and PDOS are non-negative."""
    m = min(m, nb)
    s = synth.random_system(seed, nk, nb, m, 1, beta)
    args = (s.H, s.P, s.pole.sigma_inf, s.pole.p, s.pole.V)
    r = pole.density(*args, beta, mu)
    for rho in r["rho"]:
        assert np.max(np.abs(rho - np.conj(rho.T))) < 1e-13
        ev = np.linalg.eigvalsh(rho)
        assert ev.min() > -1e-13 and ev.max() < 1 + 1e-13
    assert -1e-13 <= r["N"] <= nb + 1e-13
    assert r["dN_dmu"] >= 0.0
    assert pole.density(*args, beta, mu + 0.05)["N"] >= r["N"] - 1e-13
    dos, pdos = pole.spectral(*args, mu, np.linspace(-6.0, 6.0, 41), 0.1)
    assert dos.min() >= 0.0 and pdos.min() >= 0.0
