"""Host-side behaviour of the oracle: mu search, ragged windows, weights."""
import numpy as np

import oracle
from paper_1111_2157_gb300 import synth


def test_find_mu_d_toy():
    s = synth.d_toy(nk=16, n_iw=128).systems[0]
    o = oracle.get()
    mu, n, it = o.find_mu(s.H, s.P, s.sigma, s.sigma_inf, s.beta, s.n_target, -1.0, 1.0)
    assert abs(n - s.n_target) <= 1e-11
    r = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu, want_rho=False)
    assert abs(r["N"] - s.n_target) <= 1e-11
    assert r["dN_dmu"] > 0


def test_occupation_monotone():
    s = synth.random_system(3, 4, 6, 2, 64, 10.0)
    o = oracle.get()
    ns = [o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu, want_rho=False)["N"]
          for mu in np.linspace(-3, 3, 7)]
    assert np.all(np.diff(ns) > 0)


def test_ragged_equals_per_k_sum():
    """A ragged system is the weighted sum of its k-points taken one at a time."""
    rng = synth.rng_for(99)
    m, beta, n_iw = 3, 8.0, 32
    nbs = [4, 7, 5]
    H = [synth.hamiltonian_dense(rng, 1, n, -3, 3, 0.3)[0] for n in nbs]
    P = [synth.projectors(rng, 1, n, m)[0] for n in nbs]
    pole = synth.sigma_two_pole(rng, m, 3.0)
    sig = pole.sample(beta, n_iw)
    w = np.array([0.5, 0.3, 0.2])
    o = oracle.get()
    mu = 0.1
    gl = o.local(H, P, sig, beta, mu, weights=w)
    r = o.density(H, P, sig, pole.sigma_inf, beta, mu, weights=w)
    gl_ref = sum(w[k] * o.local(H[k][None], P[k][None], sig, beta, mu, weights=[1.0]) for k in range(3))
    n_ref = sum(w[k] * o.density(H[k][None], P[k][None], sig, pole.sigma_inf, beta, mu,
                                 weights=[1.0])["N"] for k in range(3))
    assert np.max(np.abs(gl - gl_ref)) < 1e-14
    assert abs(r["N"] - n_ref) < 1e-13
    for k in range(3):
        rk = o.density(H[k][None], P[k][None], sig, pole.sigma_inf, beta, mu, weights=[1.0])["rho"][0]
        assert np.max(np.abs(r["rho"][k] - rk)) < 1e-14


def test_thread_count_independent():
    s = synth.random_system(4, 9, 6, 3, 32, 10.0)
    o = oracle.get()
    o.set_threads(1)
    a = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, 0.2)
    o.set_threads(4)
    b = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, 0.2)
    o.set_threads(0)
    assert np.array_equal(a["rho"], b["rho"])
    assert abs(a["N"] - b["N"]) < 1e-13
