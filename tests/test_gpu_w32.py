"""N(mu) passes on the warp-per-matrix kernels (GF_KERNEL=w32: one warp per matrix for
windows up to 40 bands, two or three warps per matrix up to 96) against the oracle.

One warp (or a few) inverts one A = (i w_n + mu) I - H_k - P_k^+ Sigma P_k in FP32 with the matrix in
its registers (Gauss-Jordan in exchange form, rows rotated by one column per pivot, lazy
row scales; rows 32 to 39 of a 33- to 40-band window split over four lanes each); the
traces are summed in FP64.  It computes the same single-word FP32 inverse
as the register-tile kernel, so the mixed path's contract tolerances hold: N within 1e-7 of
the FP64 oracle (it reaches 1e-9 to 1e-8 here), dN/dmu within 1e-5.  Cases: windows of 1 to
40 bands (one row per lane for 16- and 32-column instances, split rows from 33 bands on, a
window of exactly 40), ragged windows and
several systems in one launch, the d-shell toy and small Ce-like and NiO-like cases, and
windows of 41 to 96 bands on two or three warps.
"""
import numpy as np
import pytest

import oracle
from paper_1111_2157_gb300 import synth
from tests.parity import make_gf

pytestmark = pytest.mark.gpu
TOL_N, TOL_DN = 1e-7, 1e-5


@pytest.fixture
def w32_kernel(monkeypatch):
    monkeypatch.setenv("GF_KERNEL", "w32")


def ragged_systems():
    rng = synth.rng_for(4242)
    systems = []
    for sidx, (m, nbs) in enumerate([(3, [1, 2, 7, 33, 5]), (5, [6, 17, 40]), (2, [16, 3, 24])]):
        H = [synth.hamiltonian_dense(rng, 1, n, -4, 4, 0.3)[0] for n in nbs]
        P = [(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(n) for n in nbs]
        pole = synth.sigma_two_pole(rng, m, 3.0)
        systems.append(synth.System(H, P, pole, pole.sample(8.0 + 4 * sidx, 40), 8.0 + 4 * sidx, 1.0))
    return systems


def ragged_wide_systems():
    rng = synth.rng_for(77)
    systems = []
    for sidx, (m, nbs) in enumerate([(3, [41, 64, 50]), (5, [65, 96, 70, 90]), (2, [44, 88])]):
        H = [synth.hamiltonian_dense(rng, 1, n, -4, 4, 0.3)[0] for n in nbs]
        P = [(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(n) for n in nbs]
        pole = synth.sigma_two_pole(rng, m, 3.0)
        systems.append(synth.System(H, P, pole, pole.sample(8.0 + 4 * sidx, 40), 8.0 + 4 * sidx, 1.0))
    return systems


CASES = {
    "d_toy": (lambda: [synth.d_toy().systems[0]], [0.3]),
    "ce_like_small": (lambda: [synth.ce_like(nk=5, n_iw=48).systems[0]], [0.1]),
    "window_13": (lambda: [synth.random_system(5, 4, 13, 3, 32, 10.0)], [0.05]),
    "window_29": (lambda: [synth.random_system(6, 3, 29, 5, 24, 10.0)], [0.15]),
    "window_35_split_rows": (lambda: [synth.random_system(8, 3, 35, 4, 24, 10.0)], [-0.1]),
    "window_40_two_orbitals": (lambda: [synth.random_system(9, 3, 40, 2, 20, 12.0)], [-0.3]),
    "ragged_three_systems": (ragged_systems, [0.2, -0.4, 1.1]),
    # two or three warps per matrix (windows of 41 to 96 bands)
    "nio_like_small": (lambda: [synth.nio_like(nk=3, n_iw=40).systems[0]], [0.2]),
    "window_57": (lambda: [synth.random_system(4, 3, 57, 6, 24, 15.0)], [-0.2]),
    "window_64": (lambda: [synth.random_system(3, 3, 64, 10, 24, 15.0)], [0.1]),
    "window_96": (lambda: [synth.random_system(5, 2, 96, 12, 24, 20.0)], [0.3]),
    "ragged_41_to_96": (ragged_wide_systems, [0.2, -0.4, 1.1]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_occupation_matches_oracle(w32_kernel, name):
    make, mus = CASES[name]
    systems = make()
    g = make_gf(systems, precision="mixed")
    n, dn = g.occupation(mus)
    g.close()
    o = oracle.get()
    for i, s in enumerate(systems):
        r = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mus[i], weights=s.weights, want_rho=False)
        assert abs(n[i] - r["N"]) <= TOL_N * max(1.0, abs(r["N"])), (i, n[i], r["N"])
        assert abs(dn[i] - r["dN_dmu"]) <= TOL_DN * abs(r["dN_dmu"]), (i, dn[i], r["dN_dmu"])


def test_find_mu_on_the_warp_kernel(w32_kernel):
    s = synth.ce_like(nk=4, n_iw=64).systems[0]
    g = make_gf([s], precision="mixed")
    mu, it = g.find_mu([s.n_target], 0.0, tol=1e-8 * s.n_target, max_iter=60)
    g.close()
    r = oracle.get().density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, float(mu[0]), weights=s.weights,
                             want_rho=False)
    assert abs(r["N"] - s.n_target) <= 1e-7 * s.n_target


def test_repeated_calls_are_bitwise_identical(w32_kernel):
    s = synth.ce_like(nk=3, n_iw=40).systems[0]
    g = make_gf([s], precision="mixed")
    a = g.occupation([0.2])
    b = g.occupation([0.2])
    g.close()
    assert a[0][0] == b[0][0] and a[1][0] == b[1][0]
