"""Pins of oracle/dmft.py: closed forms, invariants and library routines."""
import numpy as np
import scipy.linalg

import oracle
from oracle import dmft
from paper_1111_2157_gb300 import synth


def _lattice(seed=71, nk=6, nb=7, m=3, n_iw=64, beta=10.0):
    s = synth.random_system(seed, nk, nb, m, n_iw, beta)
    return s


def test_single_k_with_identity_projector_gives_v_dc():
    """N_k = 1, P = I: G_loc = G, so Delta = (H - E_imp) = V_DC I at every frequency."""
    rng = synth.rng_for(72)
    m, beta, n_iw, vdc = 4, 8.0, 32, 1.7
    H = synth.hamiltonian_dense(rng, 1, m, -2.0, 2.0, 0.5)
    P = np.eye(m, dtype=np.complex128)[None]
    ps = synth.sigma_two_pole(rng, m, 3.0)
    sig = ps.sample(beta, n_iw)
    mu = 0.3
    gl = oracle.get().local(H, P, sig, beta, mu)
    E = dmft.impurity_levels(H, P, v_dc=vdc)
    D = dmft.hybridization(gl, sig, E, beta, mu)
    assert np.max(np.abs(D - vdc * np.eye(m)[None])) < 1e-12


def test_high_frequency_decay_and_causality():
    """P P^+ = I: Delta - V_DC = O(1/w) and -Im Delta >= 0 (a bath hybridization)."""
    s = _lattice(n_iw=4000)
    mu, vdc = 0.2, 0.5
    idx = [10, 1000, 3999]
    gl = oracle.get().local(s.H, s.P, s.sigma, s.beta, mu, n_idx=idx)
    E = dmft.impurity_levels(s.H, s.P, v_dc=vdc)
    m = s.m
    D = np.array([(1j * (2 * n + 1) * np.pi / s.beta + mu) * np.eye(m) - E - s.sigma[n]
                  - np.linalg.inv(gl[i]) for i, n in enumerate(idx)])
    w = (2 * np.array(idx) + 1) * np.pi / s.beta
    r = [np.max(np.abs(D[i] - vdc * np.eye(m))) * w[i] for i in range(3)]
    assert abs(r[2] / r[1] - 1.0) < 0.05
    for i in range(3):
        herm_im = (D[i] - np.conj(D[i].T)) / 2j
        assert np.max(np.linalg.eigvalsh(herm_im)) < 1e-12


def test_hybridization_numbering_matches_direct_formula():
    s = _lattice(n_iw=16)
    mu = -0.1
    gl = oracle.get().local(s.H, s.P, s.sigma, s.beta, mu)
    E = dmft.impurity_levels(s.H, s.P)
    D = dmft.hybridization(gl, s.sigma, E, s.beta, mu)
    n = 7
    ref = (1j * (2 * n + 1) * np.pi / s.beta + mu) * np.eye(s.m) - E - s.sigma[n] - np.linalg.inv(gl[n])
    assert np.max(np.abs(D[n] - ref)) < 1e-13


def test_lowdin_against_library_sqrtm_and_special_cases():
    rng = np.random.default_rng(73)
    W = [rng.standard_normal((4, 9)) + 1j * rng.standard_normal((4, 9)) for _ in range(3)]
    P = dmft.lowdin(W)
    for Wk, Pk in zip(W, P):
        assert np.max(np.abs(Pk @ np.conj(Pk.T) - np.eye(4))) < 1e-13
        ref = np.linalg.inv(scipy.linalg.sqrtm(Wk @ np.conj(Wk.T))) @ Wk
        assert np.max(np.abs(Pk - ref)) < 1e-12
    Q = synth.projectors(synth.rng_for(74), 2, 9, 4)
    assert np.max(np.abs(np.array(dmft.lowdin(Q)) - Q)) < 1e-13
    D = np.diag([0.5, 2.0, 1.3, 0.9])
    assert np.max(np.abs(np.array(dmft.lowdin([D @ Q[0]]))[0] - Q[0])) < 1e-13


def test_double_counting_special_cases():
    assert abs(dmft.double_counting(6.0, 0.0, 3, 1.0)[0] - 6.0) < 1e-15   # J = 0
    assert abs(dmft.double_counting(6.0, 0.7, 0, 1.0)[0] - 6.0) < 1e-15   # s shell: U_bar = U
    ub, vdc, edc = dmft.double_counting(8.0, 1.0, 2, 8.0)                  # d shell, U = 8, J = 1
    assert abs(ub - 52.0 / 9.0) < 1e-14
    assert abs(vdc - ub * 7.5) < 1e-13 and abs(edc - ub * 28.0) < 1e-12
