"""The arithmetic of the mixed path's refined projections, modelled in numpy on the CPU.

The mixed kernels invert A = (i w_n + mu) I - H_k - P_k^+ Sigma P_k in single-word FP32 and
refine only the columns the projections consume: Y0 = X P^+ (FP32), R = P^+ - A Y0 with a
residual exact to about 2^-44 (FP32 pairs on the GPU; FP64 here), rounded to FP32,
dY = X R (FP32), Y = Y0 + dY, and P G P^+ = P Y.  This model shows what the GPU tests'
bounds rest on: the unrefined FP32 projection is off by about kappa 2^-24 (1e-7 to 1e-6),
outside the 1e-8 bound that the tests hold G_loc to, and one refinement step brings it to
about (kappa 2^-24)^2, far inside.  It also shows that Tr X (the N(mu) sum, unrefined) has
an FP32-level error per frequency that averages down over many frequencies.
"""
import numpy as np
import pytest


def point_matrix(rng, nb, m, w, mu):
    h = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
    h = 0.3 * (h + h.conj().T) + np.diag(rng.uniform(-8, 8, nb))
    q, _ = np.linalg.qr(rng.standard_normal((nb, m)) + 1j * rng.standard_normal((nb, m)))
    p = q.conj().T                                   # m x nb, orthonormal rows
    s = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    sigma = 0.5 * (s + s.conj().T) - 1j * np.eye(m)  # causal: negative imaginary part
    a = (1j * w + mu) * np.eye(nb) - h - p.conj().T @ sigma @ p
    return a, p


def refined_projection(a, p):
    a32 = a.astype(np.complex64)
    x = np.linalg.inv(a32)                           # single-word FP32 inverse
    pd32 = p.conj().T.astype(np.complex64)
    y0 = x @ pd32                                    # FP32
    r = (p.conj().T - a @ y0.astype(np.complex128)).astype(np.complex64)
    dy = x @ r                                       # FP32
    y = y0.astype(np.complex128) + dy.astype(np.complex128)
    return p @ (y0.astype(np.complex128)), p @ y, x


@pytest.mark.parametrize("seed,nb,m,w", [(1, 40, 14, 0.0314), (2, 40, 14, 1.0), (3, 96, 20, 0.0785)])
def test_one_refinement_step_meets_the_bound(seed, nb, m, w):
    rng = np.random.default_rng(seed)
    a, p = point_matrix(rng, nb, m, w, mu=0.2)
    exact = p @ np.linalg.solve(a, p.conj().T)
    unrefined, refined, _ = refined_projection(a, p)
    scale = np.max(np.abs(exact))
    err0 = np.max(np.abs(unrefined - exact)) / scale
    err1 = np.max(np.abs(refined - exact)) / scale
    assert err0 > 1e-8          # the unrefined FP32 projection fails the G_loc bound
    assert err1 < 1e-10         # one step with an exact residual meets it with room
    assert err1 < 1e-3 * err0


def test_trace_error_averages_over_frequencies():
    """Tr X per frequency carries an FP32-level error; its sum over many frequencies (the
    N(mu) sum) has a much smaller relative error, which is why N takes Tr X unrefined."""
    rng = np.random.default_rng(9)
    nb, m, beta = 40, 14, 100.0
    h = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
    h = 0.3 * (h + h.conj().T) + np.diag(rng.uniform(-8, 8, nb))
    q, _ = np.linalg.qr(rng.standard_normal((nb, m)) + 1j * rng.standard_normal((nb, m)))
    p = q.conj().T
    errs, tr64, tr32 = [], 0.0, 0.0
    for n in range(256):
        w = (2 * n + 1) * np.pi / beta
        a = (1j * w + 0.1) * np.eye(nb) - h - p.conj().T @ (-0.5j * np.eye(m)) @ p
        t64 = np.trace(np.linalg.inv(a)).real
        t32 = float(np.trace(np.linalg.inv(a.astype(np.complex64))).real)
        errs.append(abs(t32 - t64) / max(abs(t64), 1e-30))
        tr64 += t64
        tr32 += t32
    assert max(errs) > 1e-8                      # single frequencies: FP32-level error
    assert abs(tr32 - tr64) / abs(tr64) < 1e-6   # the sum: errors of both signs average
