"""N(mu) passes on the tcgen05 tensor-core kernel (GF_KERNEL=tc) against the oracle.

The kernel inverts A = (i w_n + mu) I - H_k - P_k^+ Sigma P_k by blocked Gauss-Jordan
elimination with the matrix in tensor memory: panels of 16 pivots on the CUDA cores,
trailing updates as TF32 tensor-core GEMMs with hi + lo split operands (three products),
FP32 accumulation.  Its inverse is about as accurate as a single-word FP32 one, with
the tensor cores' accumulation a few times coarser, so the contract tolerances of
the mixed path hold: N within 1e-7 relative of the FP64 oracle (it reaches 5e-10 to
8e-8 on these cases), dN/dmu within 1e-5.

Cases: windows from 1 to 128 bands (padding to a multiple of 8, short last blocks,
one to four matrices per CTA), several systems in one launch, the d-shell toy, and
small Ce-like and NiO-like cases.  The kernel's bounded wait is tested by a run
that issues no MMA: the wait runs out, the call returns GF_ETIMEOUT, and the same
context computes correctly afterwards.
"""
import numpy as np
import pytest

import oracle
from paper_1111_2157_gb300 import gf, synth
from tests.parity import make_gf

pytestmark = pytest.mark.gpu
TOL_N, TOL_DN = 1e-7, 1e-5


@pytest.fixture
def tc_kernel(monkeypatch):
    monkeypatch.setenv("GF_KERNEL", "tc")


def ragged_systems():
    rng = synth.rng_for(4242)
    systems = []
    for sidx, (m, nbs) in enumerate([(3, [1, 2, 7, 33, 5]), (5, [6, 17, 40]), (2, [64, 3, 100, 128])]):
        H = [synth.hamiltonian_dense(rng, 1, n, -4, 4, 0.3)[0] for n in nbs]
        P = [(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(n) for n in nbs]
        pole = synth.sigma_two_pole(rng, m, 3.0)
        systems.append(synth.System(H, P, pole, pole.sample(8.0 + 4 * sidx, 40), 8.0 + 4 * sidx, 1.0))
    return systems


CASES = {
    "d_toy": (lambda: [synth.d_toy().systems[0]], [0.3]),
    "ce_like_small": (lambda: [synth.ce_like(nk=5, n_iw=48).systems[0]], [0.1]),
    "nio_like_small": (lambda: [synth.nio_like(nk=3, n_iw=40).systems[0]], [0.2]),
    "window_128": (lambda: [synth.random_system(21, 2, 128, 12, 24, 20.0)], [0.1]),
    "window_13": (lambda: [synth.random_system(5, 4, 13, 3, 32, 10.0)], [0.05]),
    "ragged_three_systems": (ragged_systems, [0.2, -0.4, 1.1]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_occupation_matches_oracle(tc_kernel, name):
    make, mus = CASES[name]
    systems = make()
    g = make_gf(systems, precision="mixed")
    n, dn = g.occupation(mus)
    log = g.tuning_log()
    g.close()
    assert "tensor cores" in log or log == "", log
    o = oracle.get()
    for i, s in enumerate(systems):
        r = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mus[i], weights=s.weights, want_rho=False)
        assert abs(n[i] - r["N"]) <= TOL_N * max(1.0, abs(r["N"])), (i, n[i], r["N"])
        assert abs(dn[i] - r["dN_dmu"]) <= TOL_DN * abs(r["dN_dmu"]), (i, dn[i], r["dN_dmu"])


def test_only_tensor_core_launches(tc_kernel):
    """With GF_KERNEL=tc the N(mu) pass runs on the tensor-core kernel alone."""
    s = synth.random_system(5, 4, 13, 3, 32, 10.0)
    g = make_gf([s], precision="mixed")
    g.occupation([0.05])
    log = g.tuning_log()
    g.close()
    assert "tensor cores" in log and "FP32 register" not in log, log


def test_repeated_calls_are_bitwise_identical(tc_kernel):
    s = synth.nio_like(nk=3, n_iw=40).systems[0]
    g = make_gf([s], precision="mixed")
    a = g.occupation([0.2])
    b = g.occupation([0.2])
    g.close()
    assert a[0][0] == b[0][0] and a[1][0] == b[1][0]


def test_bounded_wait_reports_timeout(tc_kernel, monkeypatch):
    """No MMA is issued, so every group's bounded wait runs out: GF_ETIMEOUT, and the
    context stays usable (the next call, with the MMAs, matches the oracle)."""
    monkeypatch.setenv("GF_AUTOTUNE", "0")
    s = synth.random_system(5, 2, 13, 3, 8, 10.0)
    g = make_gf([s], precision="mixed")
    monkeypatch.setenv("GF_TC_TEST_SKIP_MMA", "1")
    with pytest.raises(gf.GFError) as err:
        g.occupation([0.05])
    assert err.value.status == gf.GF_ETIMEOUT
    monkeypatch.delenv("GF_TC_TEST_SKIP_MMA")
    n, _ = g.occupation([0.05])
    g.close()
    r = oracle.get().density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, 0.05, weights=s.weights, want_rho=False)
    assert abs(n[0] - r["N"]) <= TOL_N * max(1.0, abs(r["N"]))
