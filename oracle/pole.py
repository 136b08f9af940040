"""Oracle of the pole (pseudo-Hamiltonian) path, Sec. 3.3 -- test infrastructure.

Only tests, the smoke check and the CPU legs of the benchmark use this module;
the library never does.  It is plain numpy: one ``numpy.linalg.eigh`` per
k-point, then the closed forms written out.

For Sigma in the pole form of Sec. 3.2.4 (Eq. se_pole),
    Sigma(i w) = Sigma_inf + sum_i V_i^+ V_i / (i w - p_i),    V_i = V[i] (1 x m),
the pseudo-Hamiltonian of Eq. pseudo_H_k, with the pole energies shifted by mu
(Sigma is a function of i w, so that the band block of [(i w + mu) - H_ps]^-1
is G(k, i w) of Eq. dmftloop1 exactly),
    H_ps = [[H_k + P^+ Sigma_inf P, W^+], [W, diag(p + mu)]],    W = V P_k,
has eigenpairs (E_l, psi_l).  With psi_l^b the band block (first N_b rows):
    rho_k  = sum_l psi_l^b psi_l^b+ n_F(E_l - mu)       (Eq. rho_LDA+DMFT_componet_final)
    N      = sum_k w_k Tr rho_k                         (Eq. fix_mu)
    n_corr = sum_k w_k Tr(P_k rho_k P_k^+)              (Eq. nf_LDA+DMFT)
    G_loc(i w_n) = sum_k w_k sum_l (P psi_l^b)(P psi_l^b)^+ / (i w_n + mu - E_l)
dN/dmu at fixed Sigma(i w): H_ps(mu) - mu = H_0 - mu Pi_b (H_0 with the poles
unshifted, Pi_b the band projector), so N = Tr[Pi_b n_F(H_0 - mu Pi_b)] and its
derivative is -sum_{l,l'} |<psi_l|Pi_b|psi_l'>|^2 (n_F(E_l) - n_F(E_l'))/(E_l - E_l')
(derivative of a matrix function; n_F' on the diagonal and for equal E).
"""
from __future__ import annotations

import numpy as np


def fermi(x, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * np.asarray(x, dtype=float)))


def pseudo_hamiltonian(H_k, P_k, sigma_inf, poles, V, mu):
    """H_ps of Eq. pseudo_H_k with pole energies p + mu; V is [n_poles, m]."""
    nb = H_k.shape[0]
    npl = len(poles)
    W = np.asarray(V) @ P_k
    Hps = np.zeros((nb + npl, nb + npl), np.complex128)
    Hps[:nb, :nb] = H_k + np.conj(P_k.T) @ sigma_inf @ P_k
    Hps[:nb, nb:] = np.conj(W.T)
    Hps[nb:, :nb] = W
    Hps[nb:, nb:] = np.diag(np.asarray(poles, dtype=float) + mu)
    return Hps


def _weights(nk, weights):
    return np.full(nk, 1.0 / nk) if weights is None else np.asarray(weights, dtype=float)


def density(H, P, sigma_inf, poles, V, beta, mu, weights=None):
    """dict(N, n_corr, dN_dmu, rho [per k]) from the eigenpairs of H_ps per k."""
    nk = len(H)
    w = _weights(nk, weights)
    rhos, N, nc, dn = [], 0.0, 0.0, 0.0
    for k in range(nk):
        nb = H[k].shape[0]
        E, psi = np.linalg.eigh(pseudo_hamiltonian(H[k], P[k], sigma_inf, poles, V, mu))
        pb = psi[:nb]
        f = fermi(E - mu, beta)
        rho = (pb * f) @ np.conj(pb.T)
        rhos.append(rho)
        N += w[k] * np.trace(rho).real
        nc += w[k] * np.trace(P[k] @ rho @ np.conj(P[k].T)).real
        # divided differences of n_F over all pairs of eigenvalues
        dE = E[:, None] - E[None, :]
        df = f[:, None] - f[None, :]
        close = np.abs(dE) < 1e-9
        dd = np.where(close, -beta * f[:, None] * (1.0 - f[:, None]), df / np.where(close, 1.0, dE))
        O = np.conj(pb.T) @ pb
        dn += w[k] * -np.sum(np.abs(O) ** 2 * dd)
    return {"N": N, "n_corr": nc, "dN_dmu": dn, "rho": rhos}


def local(H, P, sigma_inf, poles, V, beta, mu, n_iw, weights=None):
    """G_loc(i w_n) for n = 0..n_iw-1, [n_iw, m, m]."""
    nk = len(H)
    w = _weights(nk, weights)
    wn = (2.0 * np.arange(n_iw) + 1.0) * np.pi / beta
    m = P[0].shape[0]
    out = np.zeros((n_iw, m, m), np.complex128)
    for k in range(nk):
        nb = H[k].shape[0]
        E, psi = np.linalg.eigh(pseudo_hamiltonian(H[k], P[k], sigma_inf, poles, V, mu))
        phi = P[k] @ psi[:nb]
        g = 1.0 / (1j * wn[:, None] + mu - E[None, :])
        out += w[k] * np.einsum("al,nl,bl->nab", phi, g, np.conj(phi))
    return out


def find_mu(H, P, sigma_inf, poles, V, beta, n_target, lo, hi, weights=None, tol=1e-12):
    """Bisection on the monotone N(mu) in [lo, hi]; returns mu."""
    f = lambda x: density(H, P, sigma_inf, poles, V, beta, x, weights)["N"] - n_target  # noqa: E731
    flo, fhi = f(lo), f(hi)
    if flo > 0 or fhi < 0:
        raise ValueError("n_target is not bracketed")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if abs(fm) <= tol or hi - lo < 1e-15:
            return mid
        if fm < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def spectral(H, P, sigma_inf, poles, V, mu, eps, eta, weights=None):
    """(DOS [n_eps], PDOS [n_eps, m]) with a Lorentzian of half width eta (Eqs. DOS, PDOS)."""
    nk = len(H)
    w = _weights(nk, weights)
    eps = np.asarray(eps, dtype=float)
    m = P[0].shape[0]
    dos = np.zeros(len(eps))
    pdos = np.zeros((len(eps), m))
    for k in range(nk):
        nb = H[k].shape[0]
        E, psi = np.linalg.eigh(pseudo_hamiltonian(H[k], P[k], sigma_inf, poles, V, mu))
        wb = np.sum(np.abs(psi[:nb]) ** 2, axis=0)
        phi2 = np.abs(P[k] @ psi[:nb]) ** 2          # [m, l]
        x = eps[:, None] + mu - E[None, :]
        lor = -np.imag(1.0 / (x + 1j * eta)) / np.pi   # [n_eps, l]
        dos += w[k] * lor @ wb
        pdos += w[k] * lor @ phi2.T
    return dos, pdos


def energy(H, P, sigma_inf, poles, V, beta, mu, weights=None):
    """(h_ks, e_ps): sum_k w_k Tr(H_k rho_k) (Eq. H_KS) and
    sum_k w_k sum_l (E_l - mu) |psi_l^b|^2 n_F(E_l - mu) (first term of Eq. H_U_energy)."""
    nk = len(H)
    w = _weights(nk, weights)
    hks, eps_sum = 0.0, 0.0
    for k in range(nk):
        nb = H[k].shape[0]
        E, psi = np.linalg.eigh(pseudo_hamiltonian(H[k], P[k], sigma_inf, poles, V, mu))
        pb = psi[:nb]
        f = fermi(E - mu, beta)
        rho = (pb * f) @ np.conj(pb.T)
        hks += w[k] * np.trace(H[k] @ rho).real
        eps_sum += w[k] * np.sum((E - mu) * np.sum(np.abs(pb) ** 2, axis=0) * f)
    return hks, eps_sum
