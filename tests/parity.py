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


def make_gf(systems, precision="fp64", tail_order=2, input_dtype="c128"):
    from paper_1111_2157_gb300.gf import GreensFunction
    g = GreensFunction.for_systems(systems, precision=precision, tail_order=tail_order,
                                   input_dtype=input_dtype)
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
