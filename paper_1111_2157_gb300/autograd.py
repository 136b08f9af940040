"""torch.autograd bridge: (Sigma(i w_n), mu) -> (G_loc(i w_n), N(mu)) through libgf.

The forward pass is one fused evaluation of the CUDA path (gf_evaluate) and the
backward pass is the library's hand-written adjoint (gf_backward): for a real
loss L with upstream gradients Gbar = dL/dRe G_loc + i dL/dIm G_loc and
Nbar = dL/dN,
    Sigma_bar(w_n) = sum_k w_k [A_k^+ Gbar(w_n) A_k^+ + Nbar (2/beta) B_k^+],
    mu_bar         = Nbar dN/dmu - sum_n sum_k w_k Re<Gbar(w_n), B_k>,
with A_k = P_k G P_k^+ and B_k = P_k G G P_k^+ (derived from Eq. dmftloop1 with
dG = G P^+ dSigma P G and dG/dmu = -G^2).  Complex gradients follow PyTorch's
convention (grad z = dL/dRe z + i dL/dIm z).
"""
from __future__ import annotations

import numpy as np
import torch


class LatticeGreen(torch.autograd.Function):
    """Inputs: sigma [n_iw, m, m] complex128 (one system) or packed over systems,
    mu float64 tensor [n_sys]; non-differentiable: the GreensFunction and Sigma(inf)."""

    @staticmethod
    def forward(ctx, sigma, mu, g, sigma_inf):
        sig = sigma.detach().contiguous()
        g.set_sigma(sig, sigma_inf)
        mus = mu.detach().double().cpu().numpy().reshape(-1)
        out = g.evaluate(mus, gloc=True, rho=False, occupation=True, n_corr=False)
        ctx.g, ctx.mus, ctx.sig, ctx.sinf, ctx.shape = g, mus, sig, sigma_inf, sigma.shape
        n = torch.as_tensor(out["N"], dtype=torch.float64, device=mu.device)
        return out["gloc"].view(sigma.shape).to(sigma.device), n.view(mu.shape)

    @staticmethod
    def backward(ctx, gbar, nbar):
        g = ctx.g
        g.set_sigma(ctx.sig, ctx.sinf)  # the forward's Sigma, whatever happened in between
        gb = None if gbar is None else gbar.detach().to(torch.complex128).contiguous().reshape(-1)
        nb = None if nbar is None else nbar.detach().double().cpu().numpy().reshape(-1)
        sbar, mubar = g.backward(ctx.mus, gloc_bar=gb, n_bar=nb)
        mu_grad = torch.as_tensor(np.asarray(mubar), dtype=torch.float64, device=nbar.device
                                  if nbar is not None else sbar.device)
        return sbar.view(ctx.shape).to(ctx.sig.device), mu_grad.view(ctx.mus.shape), None, None


def lattice_green(g, sigma, mu, sigma_inf):
    """(G_loc, N) with gradients w.r.t. sigma and mu; g is a GreensFunction with H and P set."""
    return LatticeGreen.apply(sigma, mu, g, sigma_inf)


def newton_mu(g, sigma, sigma_inf, n_target, mu0=0.0, tol=1e-10, max_iter=50):
    """Newton search for N(mu) = n_target with dN/dmu from the autograd graph (adjoint)."""
    mu = torch.tensor([float(mu0)], dtype=torch.float64, requires_grad=True)
    lo, hi = -np.inf, np.inf
    for it in range(1, max_iter + 1):
        _, n = lattice_green(g, sigma, mu, sigma_inf)
        f = float(n.item()) - n_target
        if abs(f) <= tol:
            return float(mu.item()), it
        (dn,) = torch.autograd.grad(n.sum(), mu)
        m = float(mu.item())
        if f < 0:
            lo = max(lo, m)
        else:
            hi = min(hi, m)
        step = -f / max(float(dn.item()), 1e-300)
        new = m + float(np.clip(step, -4.0, 4.0))
        if np.isfinite(lo) and np.isfinite(hi) and not (lo < new < hi):
            new = 0.5 * (lo + hi)
        mu = torch.tensor([new], dtype=torch.float64, requires_grad=True)
    raise RuntimeError("newton_mu did not converge")
