"""Batched path: several systems with ragged band windows in one persistent launch, graph replay."""
import numpy as np
import pytest

import oracle
from paper_1111_2157_gb300 import synth
from tests.parity import make_gf, pack, rel

pytestmark = pytest.mark.gpu


def _batched_small():
    # the batched workload's generators (8 systems, N_b(k) in [48, 128], m in [10, 14]),
    # with 0.2 % of its k-points and 24 frequencies
    return synth.batched(n_iw=24, nk_scale=0.002).systems


@pytest.mark.parametrize("precision", ["fp64", "mixed", "pair"])
def test_one_launch_for_all_systems_matches_oracle(precision):
    systems = _batched_small()
    g = make_gf(systems, precision=precision)
    mus = [0.1 * i for i in range(len(systems))]
    n, dn = g.occupation(mus)
    g.local(mus)  # the first call of a mode may also run the autotuner's sample launches
    gl = g.local(mus).cpu().numpy()
    st = g.stats()
    off = 0
    # mixed: N at the contract (1e-7), G_loc from refined projections (1e-8), dN/dmu from
    # unrefined FP32 inverses (1e-5)
    tol_n, tol_dn, tol_g = (1e-10, 1e-10, 1e-10) if precision == "fp64" else (1e-7, 1e-5, 1e-8)
    for i, s in enumerate(systems):
        r = oracle.get().density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mus[i], want_rho=False)
        assert abs(n[i] - r["N"]) < tol_n * r["N"]
        assert abs(dn[i] - r["dN_dmu"]) < tol_dn * r["dN_dmu"]
        size = s.n_iw * s.m * s.m
        if i < 2:
            glo = oracle.get().local(s.H, s.P, s.sigma, s.beta, mus[i])
            assert rel(gl[off:off + size], glo.reshape(-1)) < tol_g
        off += size
    # G_loc of all systems comes from one point-kernel launch per band-window bucket
    # (N_b <= 64, <= 96, > 96) plus one k-reduction
    assert st["launches"] <= 4


def test_batched_equals_one_context_per_system():
    systems = _batched_small()[:4]
    mus = [0.2, -0.1, 0.4, 0.0]
    g = make_gf(systems)
    n_all, _ = g.occupation(mus)
    for i, s in enumerate(systems):
        gi = make_gf([s])
        n_i, _ = gi.occupation([mus[i]])
        assert abs(n_i[0] - n_all[i]) < 1e-12 * abs(n_all[i])
        gi.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "pair"])
def test_graph_replay_is_bitwise_identical(precision):
    systems = _batched_small()[:3]
    g0 = make_gf(systems, precision=precision)
    g1 = make_gf(systems, precision=precision, graph=True)
    # the FP64 kernels round alike whatever the tiles; the FP32 and FP32-pair kernels round
    # differently per autotuned tile shape, and two contexts may pick different shapes, so
    # across contexts they are compared to their precision, and bitwise within a context
    # (the first evaluation launches normally, the third replays the captured graph)
    tol = 0.0 if precision == "fp64" else (1e-12 if precision == "pair" else 1e-7)
    first = None
    for mus in ([0.0, 0.1, 0.2], [0.3, -0.2, 0.05], [0.0, 0.1, 0.2], [1.0, 1.0, -1.0]):
        a = g0.occupation(mus)
        b = g1.occupation(mus)
        assert np.all(np.abs(a[0] - b[0]) <= tol * np.abs(a[0]))
        assert np.all(np.abs(a[1] - b[1]) <= 100 * tol * np.abs(a[1]))
        if first is None:
            first = b
        elif mus == [0.0, 0.1, 0.2]:
            assert np.array_equal(first[0], b[0]) and np.array_equal(first[1], b[1])
    # the replayed evaluations still drive the mu search (the mixed path's N carries FP32
    # rounding of about 1e-9 relative, so its search stops at 1e-8 relative)
    targets = [s.n_target for s in systems]
    mu_tol = 1e-8 * min(targets) if precision == "mixed" else 1e-10
    m0, _ = g0.find_mu(targets, 0.0, tol=mu_tol)
    m1, _ = g1.find_mu(targets, 0.0, tol=mu_tol)
    if precision == "fp64":
        assert np.array_equal(m0, m1)
    n1, _ = g1.occupation(m1)
    assert np.all(np.abs(n1 - np.asarray(targets)) <= mu_tol)
    # inputs changed after capture: the graph reads the new inputs
    s2 = [synth.System(s.H, s.P, s.pole, s.sigma * 0.5, s.beta, s.n_target) for s in systems]
    sig = pack([t.sigma for t in s2])
    g0.set_sigma(sig, pack([t.sigma_inf for t in s2]))
    g1.set_sigma(sig, pack([t.sigma_inf for t in s2]))
    a, b = g0.occupation([0.1, 0.1, 0.1])[0], g1.occupation([0.1, 0.1, 0.1])[0]
    assert np.all(np.abs(a - b) <= tol * np.abs(a))


def _rounded(s):
    """The system as its complex64 inputs carry it (what the library receives for a c64 system)."""
    if s.dtype != "c64":
        return s
    r = lambda a: np.asarray(a).astype(np.complex64).astype(np.complex128)  # noqa: E731
    H = [r(h) for h in s.H] if isinstance(s.H, list) else r(s.H)
    P = [r(p) for p in s.P] if isinstance(s.P, list) else r(s.P)
    pole = synth.PoleSigma(r(s.pole.sigma_inf), s.pole.p, s.pole.V)
    return synth.System(H, P, pole, r(s.sigma), s.beta, s.n_target, dtype="c64")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_complex128_and_complex64_systems_in_one_context(precision):
    """Half the batched systems are complex64: one context takes every system in its own dtype
    (one launch per window bucket), matches the oracle on the complex64-rounded inputs, and, in
    FP64, equals bit for bit a context given the same rounded values in complex128."""
    from paper_1111_2157_gb300.gf import GreensFunction
    systems = _batched_small()[:4]
    assert {s.dtype for s in systems} == {"c128", "c64"}
    g = GreensFunction.for_systems(systems, precision=precision, input_dtype="per_system")
    g.set_hamiltonian(pack([pack(s.H) for s in systems]))
    g.set_projectors(pack([pack(s.P) for s in systems]))
    g.set_sigma(pack([s.sigma for s in systems]), pack([s.sigma_inf for s in systems]))
    mus = [0.1, -0.2, 0.3, 0.0]
    n, dn = g.occupation(mus)
    gl = g.local(mus).cpu().numpy()
    ref = [_rounded(s) for s in systems]
    tol_n, tol_g = (1e-10, 1e-10) if precision == "fp64" else (1e-7, 1e-8)
    off = 0
    for i, s in enumerate(ref):
        r = oracle.get().density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mus[i], want_rho=False)
        assert abs(n[i] - r["N"]) < tol_n * r["N"]
        size = s.n_iw * s.m * s.m
        if i < 2:
            glo = oracle.get().local(s.H, s.P, s.sigma, s.beta, mus[i])
            assert rel(gl[off:off + size], glo.reshape(-1)) < tol_g
        off += size
    if precision == "fp64":
        g2 = make_gf(ref)
        n2, dn2 = g2.occupation(mus)
        assert np.array_equal(n, n2) and np.array_equal(dn, dn2)
