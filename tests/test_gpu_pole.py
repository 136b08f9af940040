"""Pole (pseudo-Hamiltonian) path on the GPU against oracle/pole.py and the Matsubara oracle."""
import numpy as np
import pytest

import oracle
from oracle import pole as pole_oracle
from paper_1111_2157_gb300 import gf as gfm
from paper_1111_2157_gb300 import synth
from tests.parity import make_gf, pack, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 2, 7, 68, 100, 256])
def test_heev_batched_matches_eigh(n):
    import torch
    rng = np.random.default_rng(n)
    n_mat = 5
    X = rng.standard_normal((n_mat, n, n)) + 1j * rng.standard_normal((n_mat, n, n))
    A = 0.5 * (X + np.conj(np.swapaxes(X, 1, 2)))
    if n >= 2:
        A[0] = np.diag(np.repeat(rng.standard_normal(1), n))  # fully degenerate, already diagonal
    w, V = gfm.heev_batched(torch.as_tensor(A, device="cuda"))
    w, V = w.cpu().numpy(), V.cpu().numpy()
    for i in range(n_mat):
        ref = np.linalg.eigvalsh(A[i])
        scale = max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(w[i] - ref)) <= 1e-12 * scale * max(1, n // 16)
        assert np.all(np.diff(w[i]) >= 0)
        res = A[i] @ V[i] - V[i] * w[i][None, :]
        assert np.max(np.abs(res)) <= 1e-12 * scale * max(1, n // 16)
        assert np.max(np.abs(np.conj(V[i].T) @ V[i] - np.eye(n))) <= 1e-12 * max(1, n // 16)


def test_heev_rejects_bad_sizes():
    import torch
    A = torch.zeros((1, 257, 257), dtype=torch.complex128, device="cuda")
    with pytest.raises(gfm.GFError):
        gfm.heev_batched(A)


def _pole_gf(systems, precision="fp64"):
    g = make_gf(systems, precision=precision)
    g.set_sigma_poles([len(s.pole.p) for s in systems],
                      np.concatenate([s.pole.p for s in systems]),
                      np.concatenate([s.pole.V.reshape(-1) for s in systems]),
                      np.concatenate([s.pole.sigma_inf.reshape(-1) for s in systems]))
    return g


def _ce_small(nk=6, n_iw=48):
    return synth.ce_like(nk=nk, n_iw=n_iw).systems[0]


def test_ce_like_occupation_density_local():
    s = _ce_small()
    g = _pole_gf([s])
    mu = 0.35
    n, dn = g.pole_occupation(mu)
    rho, nc = g.pole_density_matrix(mu)
    gl = g.pole_local(mu).cpu().numpy()
    ref = pole_oracle.density(s.H, s.P, s.sigma_inf, s.pole.p, s.pole.V, s.beta, mu)
    assert abs(n[0] - ref["N"]) <= 1e-10 * ref["N"]
    assert abs(dn[0] - ref["dN_dmu"]) <= 1e-10 * ref["dN_dmu"]
    assert abs(nc[0] - ref["n_corr"]) <= 1e-10 * ref["n_corr"]
    assert rel(rho.cpu().numpy(), pack(ref["rho"])) <= 1e-10
    glo = oracle.get().local(s.H, s.P, s.sigma, s.beta, mu)
    assert rel(gl, glo.reshape(-1)) <= 1e-10


def test_pole_local_equals_matsubara_path_on_gpu():
    s = _ce_small(nk=4, n_iw=64)
    g = _pole_gf([s])
    mu = -0.2
    a = g.pole_local(mu).cpu().numpy()
    b = g.local(mu).cpu().numpy()
    assert rel(a, b) <= 1e-12


def _ragged_systems():
    """Two systems; the second has N_b + n_poles up to 98 (matrix in global memory)."""
    out = []
    for seed, nbs, m in ((41, [12, 20, 9], 4), (42, [60, 70, 66, 64], 14)):
        rng = synth.rng_for(seed)
        H = [synth.hamiltonian_dense(rng, 1, n, -6.0, 6.0, 0.3)[0] for n in nbs]
        P = [synth.projectors(rng, 1, n, m)[0] for n in nbs]
        ps = synth.sigma_two_pole(rng, m, 5.0)
        out.append(synth.System(H, P, ps, ps.sample(30.0, 24), 30.0, float(np.mean(nbs)) / 2))
    return out


def test_ragged_systems_and_global_workspace():
    systems = _ragged_systems()
    g = _pole_gf(systems)
    mus = [0.1, -0.3]
    n, dn = g.pole_occupation(mus)
    rho, nc = g.pole_density_matrix(mus)
    gl = g.pole_local(mus).cpu().numpy()
    rho = rho.cpu().numpy()
    off_r, off_g = 0, 0
    for i, s in enumerate(systems):
        ref = pole_oracle.density(s.H, s.P, s.sigma_inf, s.pole.p, s.pole.V, s.beta, mus[i])
        assert abs(n[i] - ref["N"]) <= 1e-10 * ref["N"]
        assert abs(dn[i] - ref["dN_dmu"]) <= 1e-10 * ref["dN_dmu"]
        assert abs(nc[i] - ref["n_corr"]) <= 1e-10 * ref["n_corr"]
        pr = pack(ref["rho"])
        assert rel(rho[off_r:off_r + pr.size], pr) <= 1e-10
        off_r += pr.size
        glo = pole_oracle.local(s.H, s.P, s.sigma_inf, s.pole.p, s.pole.V, s.beta, mus[i], s.n_iw)
        assert rel(gl[off_g:off_g + glo.size], glo.reshape(-1)) <= 1e-10
        off_g += glo.size


def test_pole_find_mu():
    s = _ce_small(nk=5)
    g = _pole_gf([s])
    mu, it = g.pole_find_mu(s.n_target, mu0=0.0, tol=1e-10)
    ref = pole_oracle.density(s.H, s.P, s.sigma_inf, s.pole.p, s.pole.V, s.beta, mu[0])
    assert abs(ref["N"] - s.n_target) <= 1e-9
    assert it <= 12


def test_pole_state_and_size_errors():
    s = _ce_small(nk=2, n_iw=8)
    g = make_gf([s])
    with pytest.raises(gfm.GFError, match="ESTATE"):
        g.pole_occupation(0.0)
    with pytest.raises(gfm.GFError, match="EINVAL"):
        g.set_sigma_poles([300], np.zeros(300), np.zeros(300 * s.m, np.complex128), s.sigma_inf)


def test_pole_spectral_and_energy():
    systems = _ragged_systems()
    g = _pole_gf(systems)
    mus = [0.1, -0.3]
    eps = np.linspace(-6.0, 6.0, 97)
    eta = 0.08
    dos, pdos = g.pole_spectral(mus, eps, eta)
    hks, eps_sum = g.pole_energy(mus)
    for i, s in enumerate(systems):
        d_ref, p_ref = pole_oracle.spectral(s.H, s.P, s.sigma_inf, s.pole.p, s.pole.V, mus[i], eps, eta)
        assert np.max(np.abs(dos[i] - d_ref)) <= 1e-10 * np.max(d_ref)
        assert np.max(np.abs(pdos[i] - p_ref)) <= 1e-10 * np.max(p_ref)
        h_ref, e_ref = pole_oracle.energy(s.H, s.P, s.sigma_inf, s.pole.p, s.pole.V, s.beta, mus[i])
        assert abs(hks[i] - h_ref) <= 1e-10 * max(1.0, abs(h_ref))
        assert abs(eps_sum[i] - e_ref) <= 1e-10 * max(1.0, abs(e_ref))


def test_warm_started_mu_search_matches_a_cold_evaluation():
    """pole_find_mu restarts Jacobi from the previous eigenpairs; a cold evaluation at its mu agrees."""
    systems = _ragged_systems()
    g = _pole_gf(systems)
    targets = [s.n_target for s in systems]
    mu, it = g.pole_find_mu(targets, mu0=0.0, tol=1e-11)
    n_cold, _ = g.pole_occupation(mu)
    assert np.max(np.abs(n_cold - np.array(targets))) <= 1e-10
    for i, s in enumerate(systems):
        ref = pole_oracle.density(s.H, s.P, s.sigma_inf, s.pole.p, s.pole.V, s.beta, mu[i])
        assert abs(ref["N"] - targets[i]) <= 1e-10


def test_heev_reports_non_convergence_without_a_fault():
    """One sweep cannot diagonalise a dense 40 x 40 matrix: GF_ENOTCONV, and the context stays usable."""
    import torch
    rng = np.random.default_rng(9)
    X = rng.standard_normal((2, 40, 40)) + 1j * rng.standard_normal((2, 40, 40))
    A = torch.as_tensor(0.5 * (X + np.conj(np.swapaxes(X, 1, 2))), device="cuda")
    with pytest.raises(gfm.GFError, match="ENOTCONV"):
        gfm.heev_batched(A, max_sweeps=1)
    w, V = gfm.heev_batched(A)
    assert np.max(np.abs(w.cpu().numpy()[0] - np.linalg.eigvalsh(A.cpu().numpy()[0]))) < 1e-11


def test_zero_poles_is_the_static_self_energy_limit():
    """n_poles = 0: H_ps = H + P^+ Sigma_inf P, N = band Fermi sum of its eigenvalues."""
    s = _ce_small(nk=3, n_iw=8)
    g = make_gf([s])
    g.set_sigma_poles([0], np.zeros(0), np.zeros(0, np.complex128), s.sigma_inf.reshape(-1))
    mu = 0.5
    n, dn = g.pole_occupation(mu)
    m = s.m
    ref = pole_oracle.density(s.H, s.P, s.sigma_inf, np.zeros(0), np.zeros((0, m)), s.beta, mu)
    assert abs(n[0] - ref["N"]) <= 1e-10 * ref["N"]
    assert abs(dn[0] - ref["dN_dmu"]) <= 1e-10 * ref["dN_dmu"]


def test_ce_like_full_size():
    """Full Ce-like size (N_k=1000, 28 poles, matrices of 68): N, dN/dmu, n_corr against the pole
    oracle over every k, G_loc at four frequencies against the Matsubara oracle."""
    s = synth.ce_like().systems[0]
    g = _pole_gf([s])
    mu = 0.9
    n, dn = g.pole_occupation(mu)
    _, nc = g.pole_density_matrix(mu, want_rho=False)
    gl = g.pole_local(mu).cpu().numpy().reshape(s.n_iw, s.m, s.m)
    ref = pole_oracle.density(s.H, s.P, s.sigma_inf, s.pole.p, s.pole.V, s.beta, mu)
    assert abs(n[0] - ref["N"]) <= 1e-10 * ref["N"]
    assert abs(dn[0] - ref["dN_dmu"]) <= 1e-10 * ref["dN_dmu"]
    assert abs(nc[0] - ref["n_corr"]) <= 1e-10 * ref["n_corr"]
    idx = [0, 5, 700, 1023]
    assert rel(gl[idx], oracle.get().local(s.H, s.P, s.sigma, s.beta, mu, n_idx=idx)) <= 1e-10
