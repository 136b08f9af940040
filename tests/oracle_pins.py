"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each ``pin_*`` takes an ``oracle.Oracle`` and returns (error, tolerance).  The
pins are written independently of ``oracle/gf_oracle.c``: closed forms from
band eigenvalues (numpy ``eigh``), the pseudo-Hamiltonian closed form of
Sec. 3.3 (Eqs. pseudo_H_k, rho_LDA+DMFT_componet_final, fix_mu), digamma sums,
the explicit 2 x 2 inverse, and central finite differences.  They are used by
``test_oracle_pins.py`` on the real oracle and by ``test_oracle_mutations.py``
on copies with planted mistakes.
"""
from __future__ import annotations

import numpy as np
from scipy.special import digamma, polygamma

from paper_1111_2157_gb300 import synth


def fermi(x, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * x))


def sigma0_remainder(xi, beta, n_iw):
    """(2/beta) sum_{n >= N} xi^3 / (w_n^2 (w_n^2 + xi^2)) in closed form.

    For one level at xi = eps - mu with Sigma = 0, n_F(xi) = 1/2 - beta xi/4 +
    (2/beta) sum_{n>=0} xi^3/(w_n^2 (w_n^2 + xi^2)); the oracle's truncated sum
    with the 1/(i w) and 1/(i w)^2 tails therefore equals n_F(xi) minus this
    remainder.  With a = pi/beta: sum_{n>=N} 1/w_n^2 = psi'(N+1/2)/(4a^2) and
    sum_{n>=N} 1/(w_n^2 + xi^2) = Im psi(N + 1/2 + i xi/(2a)) / (2 a xi).
    """
    xi = np.asarray(xi, dtype=float)
    a = np.pi / beta
    out = np.zeros_like(xi)
    nz = np.abs(xi) > 1e-300
    x = xi[nz]
    s1 = polygamma(1, n_iw + 0.5) / (4 * a * a)
    s2 = np.imag(digamma(n_iw + 0.5 + 1j * x / (2 * a))) / (2 * a * x)
    out[nz] = (2.0 / beta) * x * (s1 - s2)
    return out


def sigma0_remainder_tail1(xi, beta, n_iw):
    """(2 xi/beta) sum_{n >= N} 1/(w_n^2 + xi^2) = (1/pi) Im psi(N + 1/2 + i beta xi/(2 pi)).

    With only the 1/(i w) moment subtracted, one level at xi = eps - mu and Sigma = 0 gives
    (1/beta) sum_{n<N} [(G - 1/(i w_n)) + c.c.] + 1/2 = 1/2 - (2 xi/beta) sum_{n<N} 1/(w_n^2 + xi^2),
    because Re[1/(i w - xi) - 1/(i w)] = -xi/(w^2 + xi^2); the complete sum is
    n_F(xi) = 1/2 - (2 xi/beta) sum_{n>=0} 1/(w_n^2 + xi^2) (the partial-fraction series of
    tanh(beta xi/2)), so the truncated value is n_F(xi) plus this remainder.
    """
    xi = np.asarray(xi, dtype=float)
    return np.imag(digamma(n_iw + 0.5 + 1j * beta * xi / (2 * np.pi))) / np.pi


def small_system(seed=7, nk=5, nb=7, m=3, n_iw=64, beta=12.0, dense=True):
    return synth.random_system(seed, nk, nb, m, n_iw, beta, dense=dense)


def pin_sigma0_gloc(o):
    """Sigma = 0: G_loc(i w) = sum_k w_k sum_b Pt_ab conj(Pt_cb) / (i w + mu - eps_kb), Pt = P U."""
    s = small_system(seed=11)
    mu = 0.37
    sig = np.zeros_like(s.sigma)
    n_idx = [0, 1, 5, 31, 63]
    got = o.local(s.H, s.P, sig, s.beta, mu, n_idx=n_idx)
    eps, U = np.linalg.eigh(s.H)
    Pt = s.P @ U
    wn = (2 * np.array(n_idx) + 1) * np.pi / s.beta
    ref = np.zeros_like(got)
    for f, w in enumerate(wn):
        g = 1.0 / (1j * w + mu - eps)
        ref[f] = np.einsum("kab,kb,kcb->ac", Pt, g, np.conj(Pt)) / s.nk
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref)), 1e-13


def pin_sigma0_density(o):
    """Sigma = 0: rho_k = U diag(n_F(xi) - R_N(xi)) U^+, N and dN/dmu from the same closed form."""
    s = small_system(seed=12, nb=6, m=2, n_iw=40, beta=9.0)
    mu = -0.41
    sig = np.zeros_like(s.sigma)
    sinf = np.zeros_like(s.sigma_inf)
    r = o.density(s.H, s.P, sig, sinf, s.beta, mu)
    eps, U = np.linalg.eigh(s.H)

    def occ(mu_):
        xi = eps - mu_
        return fermi(xi, s.beta) - sigma0_remainder(xi.ravel(), s.beta, s.n_iw).reshape(xi.shape)

    f = occ(mu)
    rho_ref = np.einsum("kab,kb,kcb->kac", U, f, np.conj(U))
    n_ref = np.sum(f) / s.nk
    # dN/dmu: fourth-order central difference of the closed form (h = 1e-3, error ~ h^4)
    h = 1e-3
    dn_ref = (8 * (np.sum(occ(mu + h)) - np.sum(occ(mu - h)))
              - (np.sum(occ(mu + 2 * h)) - np.sum(occ(mu - 2 * h)))) / (12 * h) / s.nk
    Pt = s.P @ U
    ncorr_ref = np.einsum("kab,kb,kab->", Pt, f, np.conj(Pt)).real / s.nk
    # each part divided by its own tolerance: rho, N, n_corr to 1e-12, dN/dmu to 1e-9 relative
    err = max(np.max(np.abs(r["rho"] - rho_ref)) / 1e-12, abs(r["N"] - n_ref) / 1e-12,
              abs(r["n_corr"] - ncorr_ref) / 1e-12, abs(r["dN_dmu"] - dn_ref) / abs(dn_ref) / 1e-9)
    return err, 1.0


def pin_sigma0_density_tail1(o):
    """tail_order = 1, Sigma = 0: rho_k = U diag(n_F(xi) + R1_N(xi)) U^+ with the remainder of the
    1/(i w)-only tail in closed form; N, n_corr and dN/dmu from the same closed form."""
    s = small_system(seed=13, nb=6, m=2, n_iw=48, beta=7.0)
    mu = 0.23
    sig = np.zeros_like(s.sigma)
    sinf = np.zeros_like(s.sigma_inf)
    r = o.density(s.H, s.P, sig, sinf, s.beta, mu, tail_order=1)
    eps, U = np.linalg.eigh(s.H)

    def occ(mu_):
        xi = eps - mu_
        return fermi(xi, s.beta) + sigma0_remainder_tail1(xi.ravel(), s.beta, s.n_iw).reshape(xi.shape)

    f = occ(mu)
    rho_ref = np.einsum("kab,kb,kcb->kac", U, f, np.conj(U))
    n_ref = np.sum(f) / s.nk
    h = 1e-3
    dn_ref = (8 * (np.sum(occ(mu + h)) - np.sum(occ(mu - h)))
              - (np.sum(occ(mu + 2 * h)) - np.sum(occ(mu - 2 * h)))) / (12 * h) / s.nk
    Pt = s.P @ U
    ncorr_ref = np.einsum("kab,kb,kab->", Pt, f, np.conj(Pt)).real / s.nk
    err = max(np.max(np.abs(r["rho"] - rho_ref)) / 1e-12, abs(r["N"] - n_ref) / 1e-12,
              abs(r["n_corr"] - ncorr_ref) / 1e-12, abs(r["dN_dmu"] - dn_ref) / abs(dn_ref) / 1e-9)
    return err, 1.0


def pseudo_h_density(s, mu):
    """Closed form of Sec. 3.3: rho_k = sum_l psi_l^b psi_l^b+ n_F(E_l - mu) from H_ps(k).

    H_ps = [[H_k + P^+ Sigma(inf) P, W^+], [W, diag(p_i + mu)]] with W_i = V_i P_k, so
    that the band block of [(i w + mu) - H_ps]^{-1} is G(k, i w) for
    Sigma(i w) = Sigma(inf) + sum_i V_i^+ V_i / (i w - p_i).
    """
    pole = s.pole
    npl = len(pole.p)
    rhos, N, ncorr = [], 0.0, 0.0
    for k in range(s.nk):
        Hk, Pk = s.H[k], s.P[k]
        nb = Hk.shape[0]
        W = pole.V @ Pk
        Hps = np.zeros((nb + npl, nb + npl), np.complex128)
        Hps[:nb, :nb] = Hk + np.conj(Pk.T) @ pole.sigma_inf @ Pk
        Hps[:nb, nb:] = np.conj(W.T)
        Hps[nb:, :nb] = W
        Hps[nb:, nb:] = np.diag(pole.p + mu)
        E, psi = np.linalg.eigh(Hps)
        pb = psi[:nb]
        rho = (pb * fermi(E - mu, s.beta)) @ np.conj(pb.T)
        rhos.append(rho)
        N += np.trace(rho).real / s.nk
        ncorr += np.trace(Pk @ rho @ np.conj(Pk.T)).real / s.nk
    return np.array(rhos), N, ncorr


def pin_pseudo_hamiltonian(o):
    """Pole-form Sigma: the truncated Matsubara sum converges to the closed form as N_w^-3.

    The first neglected tail term is 2 M4/w^4 (the 1/(i w)^3 term cancels
    between w and -w), so the error of N_w frequencies is c / N_w^3 + O(N_w^-5);
    the Richardson combination (8 X(2M) - X(M)) / 7 removes the N_w^-3 term.
    """
    beta, mu = 6.0, 0.3
    base = synth.random_system(21, 3, 6, 3, 1, beta)
    rho_ex, n_ex, nc_ex = pseudo_h_density(base, mu)
    res = {}
    for n_iw in (400, 800):
        sig = base.pole.sample(beta, n_iw)
        res[n_iw] = o.density(base.H, base.P, sig, base.sigma_inf, beta, mu)
    e1, e2 = res[400]["N"] - n_ex, res[800]["N"] - n_ex
    ratio = e2 / e1 if e1 != 0 else 0.0
    rich_n = (8 * res[800]["N"] - res[400]["N"]) / 7
    rich_rho = (8 * res[800]["rho"] - res[400]["rho"]) / 7
    rich_nc = (8 * res[800]["n_corr"] - res[400]["n_corr"]) / 7
    err = max(abs(rich_n - n_ex), np.max(np.abs(rich_rho - rho_ex)), abs(rich_nc - nc_ex),
              abs(ratio - 0.125) * 1e-6)
    return err, 1e-8


def pin_two_band_inverse(o):
    """2 x 2: G = [[d, -b], [-c, a]] / (ad - bc) for A = [[a, b], [c, d]] built from the definition."""
    rng = np.random.default_rng(5)
    worst = 0.0
    for trial in range(20):
        H = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        H = H + np.conj(H.T)
        m = 1 + trial % 2
        P = rng.standard_normal((m, 2)) + 1j * rng.standard_normal((m, 2))
        S = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        wn, mu = 0.1 + trial * 0.37, rng.standard_normal()
        emb = np.zeros((2, 2), np.complex128)
        for i in range(2):
            for j in range(2):
                emb[i, j] = sum(np.conj(P[x, i]) * S[x, y] * P[y, j] for x in range(m) for y in range(m))
        A = (1j * wn + mu) * np.eye(2) - H - emb
        a, b, c, d = A[0, 0], A[0, 1], A[1, 0], A[1, 1]
        ref = np.array([[d, -b], [-c, a]]) / (a * d - b * c)
        got = o.green(H, P, S, wn, mu)
        worst = max(worst, np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    return worst, 1e-13


def pin_woodbury_eigenbasis(o):
    """G from the eigenbasis of H_k and an m x m solve (Woodbury), an independent route.

    With H = U diag(eps) U^+, Pt = P U and D = diag(i w + mu - eps):
    U^+ A U = D - Pt^+ Sigma Pt, so G = U [D^-1 + D^-1 Pt^+ (I - Sigma g0)^-1 Sigma Pt D^-1] U^+
    with g0 = Pt D^-1 Pt^+ (m x m), and P G P^+ = (g0^-1 - Sigma)^-1.
    """
    rng = np.random.default_rng(17)
    s = synth.random_system(23, 3, 9, 4, 32, 10.0)
    worst = 0.0
    for k in range(s.nk):
        eps, U = np.linalg.eigh(s.H[k])
        Pt = s.P[k] @ U
        for n in (0, 3, 31):
            mu = rng.uniform(-1.0, 1.0)
            wn = (2 * n + 1) * np.pi / s.beta
            Sig = s.sigma[n]
            dinv = 1.0 / (1j * wn + mu - eps)
            g0 = (Pt * dinv) @ np.conj(Pt.T)
            core = np.linalg.solve(np.eye(s.m) - Sig @ g0, Sig)
            Gp = np.diag(dinv) + (dinv[:, None] * np.conj(Pt.T)) @ core @ (Pt * dinv)
            ref = U @ Gp @ np.conj(U.T)
            got = o.green(s.H[k], s.P[k], Sig, wn, mu)
            worst = max(worst, np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
            ploc = np.linalg.inv(np.linalg.inv(g0) - Sig)
            got_loc = s.P[k] @ got @ np.conj(s.P[k].T)
            worst = max(worst, np.max(np.abs(got_loc - ploc)) / np.max(np.abs(ploc)))
    return worst, 1e-12


def pin_high_frequency_moment(o):
    """w^2 (G - I/(i w)) -> -M2 = -(H + P^+ Sigma(inf) P - mu), with an O(1/w) remainder.

    Returns max(rem(w2) / 1e-3, (rem(w2)/rem(w1)) / 0.2): the remainder is small
    at w2 and falls roughly like 1/w between w1 and w2 = 10 w1.
    """
    s = small_system(seed=31, nk=2)
    mu = 0.2
    rem = {}
    for n in (20000, 200000):
        wn = (2 * n + 1) * np.pi / s.beta
        sig_n = s.pole.sigma_inf + np.einsum("ia,i,ib->ab", np.conj(s.pole.V),
                                            1.0 / (1j * wn - s.pole.p), s.pole.V)
        worst = 0.0
        for k in range(s.nk):
            G = o.green(s.H[k], s.P[k], sig_n, wn, mu)
            M2 = s.H[k] + np.conj(s.P[k].T) @ s.pole.sigma_inf @ s.P[k] - mu * np.eye(s.H.shape[1])
            lhs = wn * wn * (G - np.eye(G.shape[0]) / (1j * wn))
            worst = max(worst, np.max(np.abs(lhs + M2)))
        rem[n] = worst
    return max(rem[200000] / 1e-3, (rem[200000] / rem[20000]) / 0.2), 1.0


def pin_symmetry_and_causality(o):
    """G(-i w) = G(i w)^+ when Sigma(-i w) = Sigma(i w)^+, and -(G - G^+)/(2i) >= 0 for w > 0."""
    s = small_system(seed=41)
    mu = 0.1
    worst_sym, worst_pos = 0.0, 0.0
    for n in (0, 3, 17):
        wn = (2 * n + 1) * np.pi / s.beta
        Gp = o.green(s.H[0], s.P[0], s.sigma[n], wn, mu)
        Gm = o.green(s.H[0], s.P[0], np.conj(s.sigma[n].T), -wn, mu)
        worst_sym = max(worst_sym, np.max(np.abs(Gm - np.conj(Gp.T))) / np.max(np.abs(Gp)))
        spec = -(Gp - np.conj(Gp.T)) / 2j
        worst_pos = max(worst_pos, -np.min(np.linalg.eigvalsh(spec)))
    return max(worst_sym, worst_pos), 1e-12


def pin_density_bounds(o):
    """rho_k Hermitian with eigenvalues in [0, 1] (up to the truncation error), 0 <= N <= N_b."""
    s = small_system(seed=51, n_iw=512, beta=8.0)
    r = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, 0.05)
    herm = max(np.max(np.abs(rk - np.conj(rk.T))) for rk in r["rho"])
    ev = np.concatenate([np.linalg.eigvalsh(0.5 * (rk + np.conj(rk.T))) for rk in r["rho"]])
    out = max(0.0, -np.min(ev), np.max(ev) - 1.0)
    bad_n = 0.0 if 0 <= r["N"] <= s.H.shape[1] else 1.0
    return max(herm, out * 1e-3, bad_n), 1e-12


def pin_dn_dmu_fd(o):
    """dN/dmu from the oracle equals the central difference of its own N(mu) (h = 1e-5)."""
    s = small_system(seed=61, n_iw=128)
    mu, h = 0.15, 1e-5
    r0 = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu, want_rho=False)
    rp = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu + h, want_rho=False)
    rm = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu - h, want_rho=False)
    fd = (rp["N"] - rm["N"]) / (2 * h)
    return abs(fd - r0["dN_dmu"]) / abs(fd), 1e-7


def _loss(o, s, sig, mu, gbar, nbar):
    n_all = np.arange(s.n_iw)
    gl = o.local(s.H, s.P, sig, s.beta, mu, n_idx=n_all)
    r = o.density(s.H, s.P, sig, s.sigma_inf, s.beta, mu, want_rho=False)
    return float(np.sum(np.real(np.conj(gbar) * gl)) + nbar * r["N"])


def pin_backward_fd(o):
    """Sigma_bar and mu_bar against central finite differences (h = 1e-6) of L = Re<gbar, G_loc> + nbar N."""
    s = small_system(seed=71, nk=3, nb=5, m=3, n_iw=16, beta=5.0)
    mu = 0.2
    rng = np.random.default_rng(3)
    gbar = rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)
    nbar = 0.7
    sbar, mubar = o.backward(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu, gloc_bar=gbar, n_bar=nbar)
    h = 1e-6
    worst = 0.0
    for (n, a, b) in [(0, 0, 0), (0, 1, 2), (3, 2, 1), (15, 0, 2)]:
        g = 0j
        for unit in (1.0, 1j):
            sp, sm = s.sigma.copy(), s.sigma.copy()
            sp[n, a, b] += h * unit
            sm[n, a, b] -= h * unit
            d = (_loss(o, s, sp, mu, gbar, nbar) - _loss(o, s, sm, mu, gbar, nbar)) / (2 * h)
            g += d * unit
        worst = max(worst, abs(g - sbar[n, a, b]) / max(abs(g), 1e-3))
    dmu = (_loss(o, s, s.sigma, mu + h, gbar, nbar) - _loss(o, s, s.sigma, mu - h, gbar, nbar)) / (2 * h)
    worst = max(worst, abs(dmu - mubar) / abs(dmu))
    return worst, 1e-6


ALL_PINS = [pin_sigma0_gloc, pin_sigma0_density, pin_sigma0_density_tail1, pin_pseudo_hamiltonian, pin_two_band_inverse,
            pin_woodbury_eigenbasis,
            pin_high_frequency_moment, pin_symmetry_and_causality, pin_density_bounds,
            pin_dn_dmu_fd, pin_backward_fd]
