"""Plausible mistakes planted in oracle/pole.py and oracle/dmft.py; a pin must catch each.

Every mutation replaces one function of the oracle module (monkeypatch) by a variant with
one mistake; the pins of test_pole_oracle.py / test_dmft_oracle.py then run against it and
at least one of them must fail.
"""
import numpy as np
import pytest

from oracle import dmft, pole
from tests import test_dmft_oracle as dpins
from tests import test_golden_double_counting as gpins
from tests import test_pole_oracle as ppins

POLE_PINS = [ppins.test_local_equals_matsubara_oracle, ppins.test_density_is_the_infinite_matsubara_limit,
             ppins.test_dn_dmu_central_difference, ppins.test_pole_free_limit_is_the_band_fermi_sum,
             ppins.test_spectral_without_self_energy_is_the_band_lorentzian_sum,
             ppins.test_spectral_weight_integrates_to_the_band_count,
             ppins.test_energy_without_self_energy, ppins.test_energy_h_ks_from_the_matsubara_density]
DMFT_PINS = [dpins.test_single_k_with_identity_projector_gives_v_dc,
             dpins.test_high_frequency_decay_and_causality,
             dpins.test_hybridization_numbering_matches_direct_formula,
             dpins.test_lowdin_against_library_sqrtm_and_special_cases,
             dpins.test_double_counting_special_cases,
             gpins.test_u_bar_is_the_pair_average_of_h_u,
             gpins.test_e_dc_is_the_mean_configuration_energy,
             gpins.test_v_dc_is_the_central_difference_of_the_mean_energy]

_ph, _dens, _spec, _energy = pole.pseudo_hamiltonian, pole.density, pole.spectral, pole.energy
_lowdin, _eimp, _hyb, _dc = dmft.lowdin, dmft.impurity_levels, dmft.hybridization, dmft.double_counting


def ph_no_mu_shift(H_k, P_k, sigma_inf, poles, V, mu):
    A = _ph(H_k, P_k, sigma_inf, poles, V, mu)
    nb = H_k.shape[0]
    A[nb:, nb:] -= mu * np.eye(len(poles))
    return A


def ph_conjugated_coupling(H_k, P_k, sigma_inf, poles, V, mu):
    return _ph(H_k, P_k, sigma_inf, poles, np.conj(V), mu)


def ph_drops_static(H_k, P_k, sigma_inf, poles, V, mu):
    return _ph(H_k, P_k, np.zeros_like(sigma_inf), poles, V, mu)


def dens_dn_sign(*a, **k):
    r = _dens(*a, **k)
    return {**r, "dN_dmu": -r["dN_dmu"]}


def dens_rho_transposed(*a, **k):
    r = _dens(*a, **k)
    return {**r, "rho": [x.T for x in r["rho"]]}


def spec_sign(*a, **k):
    d, p = _spec(*a, **k)
    return -d, -p


def energy_no_mu(H, P, sigma_inf, poles, V, beta, mu, weights=None):
    hks, e = _energy(H, P, sigma_inf, poles, V, beta, mu, weights)
    n = _dens(H, P, sigma_inf, poles, V, beta, mu, weights)["N"]
    return hks, e + mu * n  # forgets the -mu of (E_l - mu)


def lowdin_cholesky(W):
    # orthonormal too, but Gram-Schmidt-like (Cholesky) instead of the symmetric O^{-1/2}
    return [np.linalg.inv(np.linalg.cholesky(w @ np.conj(w.T))) @ w for w in W]


def eimp_plus_vdc(H, P, weights=None, v_dc=0.0):
    return _eimp(H, P, weights, -v_dc)


def hyb_plus_inverse(gloc, sigma, e_imp, beta, mu):
    return _hyb(gloc, sigma, e_imp, beta, mu) + 2 * np.linalg.inv(gloc)


def dc_sign(U, J, l, n):
    M = 2 * l + 1
    ub = (U + 2 * (M - 1) * (U - 2 * J) + (M - 1) * J) / (2 * M - 1)
    return ub, ub * (n - 0.5), 0.5 * ub * n * (n - 1)


def dc_hund_all_orbitals(U, J, l, n):
    ub, _, _ = _dc(U, J, l, n)
    M = 2 * l + 1
    ub = ub - J / (2 * M - 1)
    return ub, ub * (n - 0.5), 0.5 * ub * n * (n - 1)


def dc_energy_n_squared(U, J, l, n):
    ub, vdc, _ = _dc(U, J, l, n)
    return ub, vdc, 0.5 * ub * n * n


MUTATIONS = [
    (pole, "pseudo_hamiltonian", ph_no_mu_shift, POLE_PINS),
    (pole, "pseudo_hamiltonian", ph_conjugated_coupling, POLE_PINS),
    (pole, "pseudo_hamiltonian", ph_drops_static, POLE_PINS),
    (pole, "density", dens_dn_sign, POLE_PINS),
    (pole, "density", dens_rho_transposed, POLE_PINS),
    (pole, "spectral", spec_sign, POLE_PINS),
    (pole, "energy", energy_no_mu, POLE_PINS),
    (dmft, "lowdin", lowdin_cholesky, DMFT_PINS),
    (dmft, "impurity_levels", eimp_plus_vdc, DMFT_PINS),
    (dmft, "hybridization", hyb_plus_inverse, DMFT_PINS),
    (dmft, "double_counting", dc_sign, DMFT_PINS),
    (dmft, "double_counting", dc_hund_all_orbitals, DMFT_PINS),
    (dmft, "double_counting", dc_energy_n_squared, DMFT_PINS),
]


@pytest.mark.parametrize("module,name,bad,pins", MUTATIONS, ids=[m[2].__name__ for m in MUTATIONS])
def test_a_pin_catches_the_mutation(monkeypatch, module, name, bad, pins):
    monkeypatch.setattr(module, name, bad)
    caught = 0
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, np.linalg.LinAlgError):
            caught += 1
    assert caught >= 1, f"no pin caught {bad.__name__}"


def test_the_pins_pass_on_the_real_oracle():
    for pin in POLE_PINS + DMFT_PINS:
        pin()
