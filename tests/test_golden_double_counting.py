"""Pins of the double-counting oracle (Sec. 3.2.3) that do not retype its formulas.

Eq. U_eff gives U_bar in closed form, Eq. E_DC the double-counting energy and Eq. V_DC its
derivative. All three follow from the local interaction of Eq. H_U, which these tests build
spin-orbital by spin-orbital and then enumerate:

* U_bar is the mean of the pair interaction of Eq. H_U over all M(2M - 1) pairs of the 2M
  spin-orbitals;
* E_DC(n) is the mean of <H_U> over every way of placing n electrons in the 2M spin-orbitals,
  found by listing the configurations;
* V_DC(n) is the central difference [E(n + 1) - E(n - 1)] / 2 of those brute-force means,
  which is exact because E is quadratic in n.

Eq. H_U is read with its second sum over all spin pairs (sigma, sigma') of two different
orbitals, and its third over equal spins only. Two electrons in one orbital interact with U,
in different orbitals with opposite spins with U - 2J, and with equal spins with U - 3J.

The parameter sets are the ones the paper prints for its benchmarks (Sec. 4), stored with
their citations in tests/golden/interaction_parameters.txt. A grid with J != 0 in every
shell l = 0..3 adds synthetic cases.
"""
import itertools
import os
from fractions import Fraction

from oracle import dmft

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "interaction_parameters.txt")
GRID = [(U, J, l) for (U, J) in [(8.0, 1.0), (6.0, 0.75), (4.5, 0.5)] for l in range(4)]


def load_parameters():
    """Rows (name, U, J, l, n) of the golden file; the source column is kept as text."""
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, U, J, l, n = line.split()[:5]
            rows.append((name, float(U), float(J), int(l), int(n)))
    return rows


def _pair_kinds(l):
    """For each unordered pair of the 2M spin-orbitals (orbital b, spin s): 0 for the same
    orbital (U), 1 for different orbitals and opposite spins (U - 2J), 2 for different
    orbitals and equal spins (U - 3J)."""
    so = [(b, s) for b in range(2 * l + 1) for s in (0, 1)]
    kinds = {}
    for i, j in itertools.combinations(range(len(so)), 2):
        (bi, si), (bj, sj) = so[i], so[j]
        kinds[(i, j)] = 0 if bi == bj else (2 if si == sj else 1)
    return len(so), kinds


def _interaction(U, J):
    U, J = Fraction(U), Fraction(J)
    return (U, U - 2 * J, U - 3 * J)


def brute_u_bar(U, J, l):
    _, kinds = _pair_kinds(l)
    v = _interaction(U, J)
    return sum(v[k] for k in kinds.values()) / len(kinds)


def brute_mean_energy(U, J, l, n):
    """Mean of <H_U> over all n-electron configurations (exact, by listing them)."""
    n_so, kinds = _pair_kinds(l)
    if n < 2:
        return Fraction(0)
    counts = [0, 0, 0]
    n_conf = 0
    for occ in itertools.combinations(range(n_so), n):
        n_conf += 1
        for pair in itertools.combinations(occ, 2):
            counts[kinds[pair]] += 1
    v = _interaction(U, J)
    return sum(c * vk for c, vk in zip(counts, v)) / n_conf


def _close(got, want, tol=1e-14):
    want = float(want)
    return abs(got - want) <= tol * max(1.0, abs(want))


def test_golden_file_holds_the_printed_benchmarks():
    names = [r[0] for r in load_parameters()]
    assert names == ["gamma-Ce", "Am", "NiO"]


def test_u_bar_is_the_pair_average_of_h_u():
    for _, U, J, l, n in load_parameters():
        assert _close(dmft.double_counting(U, J, l, n)[0], brute_u_bar(U, J, l))
    for U, J, l in GRID:
        assert _close(dmft.double_counting(U, J, l, 1.0)[0], brute_u_bar(U, J, l))


def test_e_dc_is_the_mean_configuration_energy():
    for _, U, J, l, n in load_parameters():
        assert _close(dmft.double_counting(U, J, l, n)[2], brute_mean_energy(U, J, l, n))
    for U, J, l in GRID:
        for n in sorted({2, 2 * l + 1, 4 * l + 1}):
            assert _close(dmft.double_counting(U, J, l, n)[2], brute_mean_energy(U, J, l, n))


def test_v_dc_is_the_central_difference_of_the_mean_energy():
    for _, U, J, l, n in load_parameters():
        want = (brute_mean_energy(U, J, l, n + 1) - brute_mean_energy(U, J, l, n - 1)) / 2
        assert _close(dmft.double_counting(U, J, l, n)[1], want)
    for U, J, l in GRID:
        for n in sorted({1, 2 * l + 1, 4 * l + 1}):
            want = (brute_mean_energy(U, J, l, n + 1) - brute_mean_energy(U, J, l, n - 1)) / 2
            assert _close(dmft.double_counting(U, J, l, n)[1], want)


def test_nio_values_by_hand():
    """NiO (U = 8, J = 1, d shell, n = 8): U_bar = 52/9 from the pair count of Eq. H_U
    (5 pairs at U, 20 at U - 2J, 20 at U - 3J over 45 pairs)."""
    assert brute_u_bar(8.0, 1.0, 2) == Fraction(5 * 8 + 20 * 6 + 20 * 5, 45) == Fraction(52, 9)
