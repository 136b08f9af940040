"""Projector orthonormalisation and the DMFT step on the GPU against oracle/dmft.py."""
import numpy as np
import pytest

import oracle
from oracle import dmft
from paper_1111_2157_gb300 import gf as gfm
from paper_1111_2157_gb300 import synth
from tests.parity import make_gf, pack, rel

pytestmark = pytest.mark.gpu


def test_lowdin_projectors_match_oracle_and_feed_the_path():
    s = synth.ce_like(nk=6, n_iw=24).systems[0]
    rng = np.random.default_rng(81)
    W = [np.diag(rng.uniform(0.5, 1.5, s.m)) @ s.P[k] + 0.05 * (
        rng.standard_normal(s.P[k].shape) + 1j * rng.standard_normal(s.P[k].shape)) for k in range(s.nk)]
    g = make_gf([s])
    P = g.set_projectors_lowdin(pack(W)).cpu().numpy()
    ref = dmft.lowdin(W)
    assert rel(P, pack(ref)) < 1e-12
    # the context now uses the orthonormal projectors
    mu = 0.2
    gl = g.local(mu).cpu().numpy()
    glo = oracle.get().local(s.H, np.array(ref), s.sigma, s.beta, mu)
    assert rel(gl, glo.reshape(-1)) < 1e-10


def test_lowdin_rejects_dependent_projections():
    s = synth.random_system(82, 2, 6, 3, 8, 10.0)
    W = [p.copy() for p in s.P]
    W[1][2] = W[1][0]  # two equal rows
    g = make_gf([s])
    with pytest.raises(gfm.GFError, match="ESINGULAR"):
        g.set_projectors_lowdin(pack(W))


def test_impurity_levels_and_hybridization():
    systems = [synth.ce_like(nk=5, n_iw=32).systems[0], synth.random_system(83, 4, 9, 3, 32, 20.0)]
    g = make_gf(systems)
    vdc = [2.5, 0.4]
    mus = [0.3, -0.2]
    E = g.impurity_levels(vdc).cpu().numpy()
    gl = g.local(mus)
    D = g.hybridization(mus, gl, vdc).cpu().numpy()
    glh = gl.cpu().numpy()
    oe, og = 0, 0
    for i, s in enumerate(systems):
        Er = dmft.impurity_levels(s.H, s.P, v_dc=vdc[i])
        assert rel(E[oe:oe + s.m * s.m], Er.reshape(-1)) < 1e-12
        oe += s.m * s.m
        size = s.n_iw * s.m * s.m
        Dr = dmft.hybridization(glh[og:og + size].reshape(s.n_iw, s.m, s.m), s.sigma, Er, s.beta, mus[i])
        assert rel(D[og:og + size], Dr.reshape(-1)) < 1e-11
        og += size

