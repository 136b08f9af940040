"""The blocked exchange (sweep) form of Gauss-Jordan elimination that the tensor-core
kernel (k_point_tc) computes, written out in numpy and checked against a direct inverse.

Per block of b pivot columns Q: the b sweeps run on the panel M[:, Q] alone (pivot =
the unused row of largest max(|Re|, |Im|)); the other columns J take one rank-b update
M'[:, J] = M[:, J] + L M[P, J]_old with L = M'[:, Q] minus 1 at (p_t, q_t), as a real GEMM
[Re L | Im L] [[Re R, -Im R], [Im R, Re R]]^T with R the old pivot rows (zero in the
panel's columns).  Windows are padded to a multiple of 8 with an identity block; the
last block may hold 8 pivots.  After all blocks X[i][c] = M[p_i][q_c].
"""
import numpy as np
import pytest


def blocked_sweep_inverse(A, block=16):
    N = A.shape[0]
    Np = (N + 7) & ~7
    M = np.eye(Np, dtype=complex)
    M[:N, :N] = A
    used = np.zeros(Np, bool)
    piv = np.zeros(Np, int)
    for j0 in range(0, Np, block):
        b = min(block, Np - j0)
        V = M[:, j0:j0 + b].copy()
        old = M.copy()
        pivot_step = -np.ones(Np, int)
        for t in range(b):
            key = np.where(~used, np.maximum(abs(V[:, t].real), abs(V[:, t].imag)), -1.0)
            p = int(np.argmax(key))
            piv[j0 + t] = p
            r = 1.0 / V[p, t]
            w = V[p] * r
            w[t] = r
            for i in range(Np):
                if i == p:
                    l = -1.0
                    V[i] = 0.0
                else:
                    l = V[i, t]
                    V[i, t] = 0.0
                V[i] = V[i] - l * w
            used[p] = True
            pivot_step[p] = t
        L = V.copy()
        rows = np.nonzero(pivot_step >= 0)[0]
        L[rows, pivot_step[rows]] -= 1.0
        # GEMM operands in their real form (K = 2 x 16, unused depth zero)
        a_op = np.zeros((128, 32))
        a_op[:Np, :b] = L.real
        a_op[:Np, 16:16 + b] = L.imag
        b_op = np.zeros((2 * Np, 32))
        for t in range(b):
            row = old[piv[j0 + t]].copy()
            row[j0:j0 + b] = 0.0
            b_op[:Np, t] = row.real
            b_op[Np:, 16 + t] = row.real
            b_op[:Np, 16 + t] = -row.imag
            b_op[Np:, t] = row.imag
        d = np.zeros((128, 2 * Np))
        d[:Np, :Np] = M.real
        d[:Np, Np:] = M.imag
        d[:Np, j0:j0 + b] = V.real
        d[:Np, Np + j0:Np + j0 + b] = V.imag
        d += a_op @ b_op.T
        M = d[:Np, :Np] + 1j * d[:Np, Np:]
    q = np.argsort(piv)
    return M[np.ix_(piv[:N], q[:N])]


@pytest.mark.parametrize("n", [1, 8, 13, 40, 96, 100, 128])
def test_blocked_sweep_equals_the_inverse(n):
    rng = np.random.default_rng(1000 + n)
    # a Green's-function-like matrix: (i w + mu) I - H with a dense Hermitian H
    h = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    h = 0.5 * (h + h.conj().T)
    a = (0.7 + 0.05j) * np.eye(n) - h
    x = blocked_sweep_inverse(a)
    ref = np.linalg.inv(a)
    assert np.max(np.abs(x - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_needs_pivoting():
    """A zero leading diagonal: partial pivoting is what makes the sweep succeed."""
    a = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [2.0, 3.0, 0.0]], dtype=complex)
    assert np.allclose(blocked_sweep_inverse(a), np.linalg.inv(a), atol=1e-14)


def test_block_width_does_not_change_the_result():
    rng = np.random.default_rng(7)
    a = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40)) + 4j * np.eye(40)
    assert np.allclose(blocked_sweep_inverse(a, block=16), blocked_sweep_inverse(a, block=8), atol=1e-12)
