"""Oracle of the steps around the lattice sums -- test infrastructure.

Only tests, the smoke check and the CPU legs of the benchmark use this module;
the library never does.  Plain numpy, one function per equation:

* Lowdin-orthonormal projectors (Eqs. 6 and 7): O_k = W_k W_k^+ is the overlap
  of the projected orbitals (rows of W_k), P_k = O_k^{-1/2} W_k.
* Impurity levels (Eq. E^imp): E_imp = sum_k w_k P_k H_k P_k^+ - V_DC I.
* Hybridization (Eq. dmftloop2): Delta(i w_n) = i w_n + mu - E_imp - Sigma(i w_n)
  - G_loc(i w_n)^{-1}, with G_loc the weighted k-sum of Eq. dmftloop1 projected.
* Double counting (Eqs. U_eff, V_DC_component, E_DC).
"""
from __future__ import annotations

import numpy as np


def lowdin(W):
    """P_k = (W_k W_k^+)^{-1/2} W_k for every k (list or array of m x N_b)."""
    out = []
    for Wk in W:
        O = Wk @ np.conj(Wk.T)
        lam, V = np.linalg.eigh(O)
        inv_sqrt = (V * (1.0 / np.sqrt(lam))) @ np.conj(V.T)
        out.append(inv_sqrt @ Wk)
    return out


def impurity_levels(H, P, weights=None, v_dc=0.0):
    nk = len(H)
    w = np.full(nk, 1.0 / nk) if weights is None else np.asarray(weights, dtype=float)
    m = P[0].shape[0]
    E = np.zeros((m, m), np.complex128)
    for k in range(nk):
        E += w[k] * (P[k] @ H[k] @ np.conj(P[k].T))
    return E - v_dc * np.eye(m)


def hybridization(gloc, sigma, e_imp, beta, mu):
    """Delta for every frequency of gloc / sigma ([n_iw, m, m])."""
    n_iw, m = gloc.shape[0], gloc.shape[1]
    out = np.empty_like(gloc)
    for n in range(n_iw):
        wn = (2 * n + 1) * np.pi / beta
        out[n] = (1j * wn + mu) * np.eye(m) - e_imp - sigma[n] - np.linalg.inv(gloc[n])
    return out


def double_counting(U, J, l, n):
    """(U_bar, V_DC, E_DC)."""
    M = 2 * l + 1
    ub = (U + 2 * (M - 1) * (U - 2 * J) - (M - 1) * J) / (2 * M - 1)
    return ub, ub * (n - 0.5), 0.5 * ub * n * (n - 1)
