"""The one-warp Gauss-Jordan elimination of the mixed warp kernels (warp_invert), emulated
lane by lane in numpy and checked against a direct inverse.

What the kernel does per pivot step j (exchange form, partial pivoting, no row swaps):
  * lane l holds row l in registers rotated left by j columns, so the pivot column is
    register 0; rows 32 to 39 (windows of 33 to 40 bands) are split over groups of four
    lanes, lane l holding register columns 10 (l mod 4) .. 10 (l mod 4) + 9 of row
    32 + l / 4;
  * the pivot is the unused row with the largest max(|Re|, |Im|) in register 0 (a split
    row's entry lives on the first lane of its group), ties to the lowest row;
  * the pivot row goes to a buffer; r = 1 / u_0; every other row: l = a_0 r,
    a_c -= l u_c (c != 0), a_0 = -l; the pivot row keeps its values, a_0 = 1, and its
    lazy scale becomes r (its stored entries are the true ones divided by r);
  * every row rotates left by one (a split row passes its first entry to the previous
    lane of its group, the first lane's wraps to the last).
After N steps register x holds original column (x + N) mod 40; the true inverse is
X[i][c] = s_p B[p_i][q_c] with p the pivot rows, q = p^{-1}.
"""
import numpy as np
import pytest

NMAX, SEG = 40, 10


def pivot_key(v):
    return max(abs(v.real), abs(v.imag))


def warp_invert(A):
    N = A.shape[0]
    assert N <= NMAX
    a0 = np.zeros((32, NMAX), complex)   # whole rows
    a1 = np.zeros((32, SEG), complex)    # split-row segments
    for lane in range(32):
        if lane < N:
            a0[lane, :N] = A[lane]
        g, r1 = lane & 3, 32 + (lane >> 2)
        for y in range(SEG):
            c = SEG * g + y
            if r1 < N and c < N:
                a1[lane, y] = A[r1, c]
    used0 = np.zeros(32, bool)
    used1 = np.zeros(32, bool)
    sc0 = np.ones(32, complex)
    sc1 = np.ones(32, complex)
    piv = []
    for _ in range(N):
        best, prow = -1.0, -1
        for lane in range(32):
            cand = []
            if lane < N and not used0[lane]:
                cand.append((pivot_key(a0[lane, 0]), lane))
            g, r1 = lane & 3, 32 + (lane >> 2)
            if g == 0 and r1 < N and not used1[lane]:
                cand.append((pivot_key(a1[lane, 0]), r1))
            for k, row in cand:
                if k > best or (k == best and row < prow):
                    best, prow = k, row
        assert best > 0.0
        buf = np.zeros(NMAX, complex)
        if prow < 32:
            buf[:] = a0[prow]
        else:
            for lane in range(32):
                if 32 + (lane >> 2) == prow:
                    g = lane & 3
                    buf[SEG * g:SEG * g + SEG] = a1[lane]
        r = 1.0 / buf[0]
        lead_vals = np.array([a1[lane & ~3, 0] for lane in range(32)])
        for lane in range(32):
            isp = lane == prow
            lq = 0.0 if isp else a0[lane, 0] * r
            a0[lane, 1:] -= lq * buf[1:]
            col = 1.0 if isp else -lq
            a0[lane] = np.roll(a0[lane], -1)
            a0[lane, -1] = col
            if isp:
                used0[lane], sc0[lane] = True, r
        upd = a1.copy()
        for lane in range(32):
            g, r1 = lane & 3, 32 + (lane >> 2)
            isp = r1 == prow
            lq = 0.0 if isp else lead_vals[lane] * r
            upd[lane] -= lq * buf[SEG * g:SEG * g + SEG]
            if g == 0:
                upd[lane, 0] = 1.0 if isp else -lq
            if isp:
                used1[lane], sc1[lane] = True, r
        for lane in range(32):
            nxt = (lane & ~3) | ((lane + 1) & 3)
            a1[lane, :-1] = upd[lane, 1:]
            a1[lane, -1] = upd[nxt, 0]
        piv.append(prow)
    B = np.zeros((N, N), complex)
    for lane in range(32):
        if lane < N:
            for x in range(NMAX):
                c = (x + N) % NMAX
                if c < N:
                    B[lane, c] = sc0[lane] * a0[lane, x]
        g, r1 = lane & 3, 32 + (lane >> 2)
        if r1 < N:
            for y in range(SEG):
                c = (SEG * g + y + N) % NMAX
                if c < N:
                    B[r1, c] = sc1[lane] * a1[lane, y]
    q = np.argsort(piv)
    return B[np.ix_(piv, q)]


@pytest.mark.parametrize("n", [1, 2, 13, 32, 33, 36, 39, 40])
def test_warp_elimination_equals_the_inverse(n):
    rng = np.random.default_rng(500 + n)
    h = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    h = 0.5 * (h + h.conj().T)
    a = (0.4 + 0.1j) * np.eye(n) - h
    x = warp_invert(a)
    ref = np.linalg.inv(a)
    assert np.max(np.abs(x - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_pivot_on_a_split_row():
    """A matrix whose largest pivot candidates sit in rows 32 to 39 (split rows)."""
    n = 40
    rng = np.random.default_rng(3)
    a = 0.01 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    perm = np.roll(np.arange(n), 8)       # row i carries its large entry in column (i + 8) mod 40
    a[np.arange(n), perm] += 5.0 + np.arange(n)
    x = warp_invert(a)
    assert np.allclose(x, np.linalg.inv(a), atol=1e-12)


def test_needs_pivoting():
    a = np.zeros((34, 34), complex)
    a[np.arange(34), (np.arange(34) + 1) % 34] = 1.0 + 0.5j   # zero diagonal
    a += 0.01 * np.eye(34)
    assert np.allclose(warp_invert(a), np.linalg.inv(a), atol=1e-10)
