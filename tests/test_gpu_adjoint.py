"""Adjoint through torch.autograd: oracle gradient, central finite differences, Newton mu, mixing."""
import numpy as np
import pytest

import oracle
from paper_1111_2157_gb300 import synth
from tests.parity import make_gf, rel

pytestmark = pytest.mark.gpu


def _case(nk=3, n_iw=12):
    # adjoint-workload shapes (N_b = 64, m = 14, beta = 100), few k-points and frequencies
    return synth.adjoint_case(nk=nk, n_iw=n_iw).systems[0]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autograd_matches_oracle_gradient(precision):
    import torch
    from paper_1111_2157_gb300.autograd import lattice_green
    s = _case()
    g = make_gf([s], precision=precision)
    rng = np.random.default_rng(7)
    gbar = rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)
    sigma = torch.tensor(s.sigma, dtype=torch.complex128, device="cuda", requires_grad=True)
    mu = torch.tensor([0.3], dtype=torch.float64, requires_grad=True)
    gl, n = lattice_green(g, sigma, mu, s.sigma_inf)
    loss = (torch.conj(torch.from_numpy(gbar).cuda()) * gl).real.sum() + 0.7 * n.sum()
    loss.backward()
    sb, mb = oracle.get().backward(s.H, s.P, s.sigma, s.sigma_inf, s.beta, 0.3, gloc_bar=gbar, n_bar=0.7)
    # mixed: Sigma_bar from the refined projections; mu_bar also carries dN/dmu from
    # unrefined FP32 inverses
    tol, tol_mu = (1e-10, 1e-10) if precision == "fp64" else (1e-8, 1e-6)
    assert rel(sigma.grad.cpu().numpy(), sb) < tol
    assert abs(mu.grad.item() - mb) / abs(mb) < tol_mu


def test_gradient_central_differences():
    """Sigma_bar and mu_bar of the GPU path against central differences of its own forward (h = 1e-6)."""
    import torch
    from paper_1111_2157_gb300.autograd import lattice_green
    s = _case(nk=2, n_iw=8)
    g = make_gf([s])
    rng = np.random.default_rng(8)
    gbar = torch.from_numpy(rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)).cuda()

    def loss_of(sig_np, mu_val):
        sig = torch.tensor(sig_np, dtype=torch.complex128, device="cuda")
        gl, n = lattice_green(g, sig, torch.tensor([mu_val], dtype=torch.float64), s.sigma_inf)
        return float(((torch.conj(gbar) * gl).real.sum() + 0.7 * n.sum()).item())

    sigma = torch.tensor(s.sigma, dtype=torch.complex128, device="cuda", requires_grad=True)
    mu = torch.tensor([0.3], dtype=torch.float64, requires_grad=True)
    gl, n = lattice_green(g, sigma, mu, s.sigma_inf)
    ((torch.conj(gbar) * gl).real.sum() + 0.7 * n.sum()).backward()
    h = 1e-6
    for (w, a, b) in [(0, 0, 0), (0, 3, 7), (5, 13, 2), (7, 6, 6)]:
        fd = 0j
        for unit in (1.0, 1j):
            sp, sm = s.sigma.copy(), s.sigma.copy()
            sp[w, a, b] += h * unit
            sm[w, a, b] -= h * unit
            fd += unit * (loss_of(sp, 0.3) - loss_of(sm, 0.3)) / (2 * h)
        got = sigma.grad[w, a, b].item()
        assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (w, a, b, got, fd)
    fd_mu = (loss_of(s.sigma, 0.3 + h) - loss_of(s.sigma, 0.3 - h)) / (2 * h)
    assert abs(mu.grad.item() - fd_mu) <= 1e-6 * abs(fd_mu)


def test_newton_mu_from_adjoint():
    from paper_1111_2157_gb300.autograd import newton_mu
    import torch
    s = _case(nk=4, n_iw=64)
    g = make_gf([s])
    sigma = torch.tensor(s.sigma, dtype=torch.complex128, device="cuda")
    mu, it = newton_mu(g, sigma, s.sigma_inf, s.n_target, mu0=0.0, tol=1e-10)
    mu_lib, _ = g.find_mu([s.n_target], 0.0, tol=1e-10)
    assert abs(mu - mu_lib[0]) < 1e-8
    assert it <= 12


def test_mixed_forward_backward_pair():
    """Mixed-precision forward/backward against the FP64 GPU pair, at the contract's
    tolerances for G_loc (1e-6) and N (1e-7) and the same for the gradients."""
    import torch
    from paper_1111_2157_gb300.autograd import lattice_green
    s = _case()
    outs = {}
    for prec in ("fp64", "mixed"):
        g = make_gf([s], precision=prec)
        sigma = torch.tensor(s.sigma, dtype=torch.complex128, device="cuda", requires_grad=True)
        mu = torch.tensor([0.1], dtype=torch.float64, requires_grad=True)
        gl, n = lattice_green(g, sigma, mu, s.sigma_inf)
        (gl.abs().pow(2).sum() + n.sum()).backward()
        outs[prec] = (gl.detach().cpu().numpy(), n.item(), sigma.grad.cpu().numpy(), mu.grad.item())
    a, b = outs["fp64"], outs["mixed"]
    assert rel(b[0], a[0]) < 1e-6 and abs(b[1] - a[1]) < 1e-7 * abs(a[1])
    assert rel(b[2], a[2]) < 1e-6 and abs(b[3] - a[3]) < 1e-6 * abs(a[3])


def test_self_energy_mixing_step_reduces_mismatch():
    """One adjoint-driven update of Sigma toward a target G_loc lowers the mismatch."""
    import torch
    from paper_1111_2157_gb300.autograd import lattice_green
    s = _case(nk=3, n_iw=10)
    g = make_gf([s])
    target = torch.tensor(synth.adjoint_case(nk=3, n_iw=10, seed=77).systems[0].sigma * 0.0,
                          dtype=torch.complex128, device="cuda")
    mu = torch.tensor([0.0], dtype=torch.float64)
    sigma = torch.tensor(s.sigma, dtype=torch.complex128, device="cuda", requires_grad=True)
    gl, _ = lattice_green(g, sigma, mu, s.sigma_inf)
    target = gl.detach() * 0.9
    loss0 = (gl - target).abs().pow(2).sum()
    loss0.backward()
    with torch.no_grad():
        sigma2 = sigma - 1e-2 * sigma.grad / sigma.grad.abs().max()
    gl2, _ = lattice_green(g, sigma2, mu, s.sigma_inf)
    loss1 = (gl2 - target).abs().pow(2).sum()
    assert loss1.item() < loss0.item()


def test_full_size_gradient_against_the_oracle():
    """The differentiation workload at full size (N_k = 2048, N_b = 64, m = 14, N_w = 1024,
    beta = 100), in the launch configuration of the full problem: Sigma_bar and mu_bar of the
    whole k-set equal the sum of the same VJP over eight k-blocks (each a context whose k-points
    carry the full set's weight 1/2048), and one block's VJP equals the oracle's (1e-10).  The
    mixed forward/backward pair matches the FP64 one to the contract's tolerance."""
    import torch
    s = synth.adjoint_case().systems[0]
    assert (s.nk, s.nb[0], s.m, s.n_iw) == (2048, 64, 14, 1024)
    rng = np.random.default_rng(31)
    gbar = (rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)) * 1e-2
    mu, nbar = 0.25, 0.6
    g = make_gf([s])
    sb_full, mb_full = g.backward([mu], gloc_bar=gbar.reshape(-1), n_bar=[nbar])
    sb_full = sb_full.cpu().numpy().reshape(s.sigma.shape)
    g.close()
    nblk, kb = 8, s.nk // 8
    w_full = np.full(kb, 1.0 / s.nk)
    acc_sb, acc_mb = np.zeros_like(sb_full), 0.0
    block0 = None
    for b in range(nblk):
        ks = slice(b * kb, (b + 1) * kb)
        sub = synth.System(s.H[ks], s.P[ks], s.pole, s.sigma, s.beta, s.n_target, weights=w_full)
        from paper_1111_2157_gb300.gf import GreensFunction
        gb = GreensFunction(64, 14, s.n_iw, s.beta, n_k=kb, k_weight=w_full)
        gb.set_hamiltonian(s.H[ks])
        gb.set_projectors(s.P[ks])
        gb.set_sigma(s.sigma, s.sigma_inf)
        sb_b, mb_b = gb.backward([mu], gloc_bar=gbar.reshape(-1), n_bar=[nbar])
        sb_b = sb_b.cpu().numpy().reshape(s.sigma.shape)
        gb.close()
        acc_sb += sb_b
        acc_mb += mb_b[0]
        if b == 0:
            block0 = (sub, sb_b, mb_b[0])
    assert rel(sb_full, acc_sb) < 1e-12
    assert abs(mb_full[0] - acc_mb) <= 1e-12 * abs(mb_full[0])
    sub, sb_0, mb_0 = block0
    sb_o, mb_o = oracle.get().backward(sub.H, sub.P, sub.sigma, sub.sigma_inf, sub.beta, mu,
                                       gloc_bar=gbar, n_bar=nbar, weights=w_full)
    assert rel(sb_0, sb_o) < 1e-10
    assert abs(mb_0 - mb_o) <= 1e-10 * abs(mb_o)
    # sampled entries of the full gradient are finite and carry both terms of the VJP
    for (w, a, b2) in [(0, 0, 0), (3, 5, 9), (511, 13, 2), (1023, 7, 7)]:
        assert np.isfinite(sb_full[w, a, b2])
    gm = make_gf([s], precision="mixed")
    sb_m, mb_m = gm.backward([mu], gloc_bar=gbar.reshape(-1), n_bar=[nbar])
    gm.close()
    assert rel(sb_m.cpu().numpy().reshape(s.sigma.shape), sb_full) < 1e-6
    assert abs(mb_m[0] - mb_full[0]) <= 1e-6 * abs(mb_full[0])
