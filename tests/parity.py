"""Helpers for GPU-vs-oracle parity tests (the oracle is the reference)."""
from __future__ import annotations

import numpy as np

import oracle


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def pack(blocks):
    return np.concatenate([np.asarray(b).reshape(-1) for b in blocks])


def make_gf(systems, precision="fp64", tail_order=2, input_dtype="c128", graph=False, lowrank=False):
    from paper_1111_2157_gb300.gf import GreensFunction
    g = GreensFunction.for_systems(systems, precision=precision, tail_order=tail_order,
                                   input_dtype=input_dtype, graph=graph, lowrank=lowrank)
    g.set_hamiltonian(pack([pack(s.H) for s in systems]))
    g.set_projectors(pack([pack(s.P) for s in systems]))
    g.set_sigma(pack([s.sigma for s in systems]), pack([s.sigma_inf for s in systems]))
    return g


def split_sys(flat, systems, per):
    out, off = [], 0
    for s in systems:
        n = per(s)
        out.append(np.asarray(flat[off:off + n]))
        off += n
    return out


def oracle_all(s, mu, tail_order=2, gloc=True):
    o = oracle.get()
    r = o.density(s.H, s.P, s.sigma, s.sigma_inf, s.beta, mu, weights=s.weights, tail_order=tail_order)
    gl = o.local(s.H, s.P, s.sigma, s.beta, mu, weights=s.weights) if gloc else None
    return r, gl


def check_system_set(systems, mus, tol, precision="fp64", tail_order=2, input_dtype="c128",
                     report=None, lowrank=False):
    """Every output of the CUDA path (G_loc, N, dN/dmu, n_corr, rho) against the oracle."""
    g = make_gf(systems, precision=precision, tail_order=tail_order, input_dtype=input_dtype,
                lowrank=lowrank)
    gl = g.local(mus).cpu().numpy()
    n, dn = g.occupation(mus)
    rho, nc = g.density_matrix(mus)
    rho = rho.cpu().numpy()
    g.close()
    gls = split_sys(gl, systems, lambda s: s.n_iw * s.m * s.m)
    rhos = split_sys(rho, systems, lambda s: int(np.sum(s.nb.astype(np.int64) ** 2)))
    for i, s in enumerate(systems):
        r, glo = oracle_all(s, mus[i], tail_order=tail_order)
        errs = {"G_loc": rel(gls[i], glo.reshape(-1)),
                "N": abs(n[i] - r["N"]) / max(1.0, abs(r["N"])),
                "dN_dmu": abs(dn[i] - r["dN_dmu"]) / abs(r["dN_dmu"]),
                "n_corr": abs(nc[i] - r["n_corr"]) / max(1.0, abs(r["n_corr"])),
                "rho": rel(rhos[i], pack(r["rho"]))}
        if report is not None:
            report.append(errs)
        for name, err in errs.items():
            t = tol[name] if isinstance(tol, dict) else tol
            assert err < t, f"{name} system {i}: {err:.3e} >= {t:.1e}"
