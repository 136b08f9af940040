"""Plant plausible mistakes in a copy of the oracle's C source; some pin must catch each.

The mutated copies are compiled with gcc into a temporary folder and run on
the CPU only.  The shipped oracle is untouched.
"""
import pytest

import oracle
from tests import oracle_pins

MUTATIONS = {
    "embed_missing_conj": ("s += conj(P[a * nb + i]) * T[a * nb + j];", "s += P[a * nb + i] * T[a * nb + j];"),
    "mu_sign": ("((i == j) ? (mu + I * wn) : 0.0)", "((i == j) ? (-mu + I * wn) : 0.0)"),
    "dropped_half": ("if (i == j) v += 0.5;", ""),
    "tail_m2_transposed": ("tail += M2[i * n + j] / (iw * iw);", "tail += M2[j * n + i] / (iw * iw);"),
    "dropped_beta_quarter": ("if (tail_order >= 2) v -= 0.25 * beta * M2[i * n + j];", ""),
    "projection_transposed": ("s += X[i * nb + j] * conj(P[b * nb + j]);", "s += X[j * nb + i] * conj(P[b * nb + j]);"),
    "m2_missing_sigma_inf": ("M2[i * n + j] = Hk[i * n + j] + w.E[i * n + j] - ((i == j) ? mu : 0.0);",
                             "M2[i * n + j] = Hk[i * n + j] - ((i == j) ? mu : 0.0);"),
    "dndmu_sign": ("trG2 += creal(-tr);", "trG2 += creal(tr);"),
    "bosonic_grid": ("return (2.0 * n + 1.0) * M_PI / beta;", "return (2.0 * n + 2.0) * M_PI / beta;"),
    "backward_missing_conj": ("acc[a * m + b] += wk[k] * n_bar * (2.0 / beta) * conj(Bk[b * m + a]);",
                              "acc[a * m + b] += wk[k] * n_bar * (2.0 / beta) * Bk[b * m + a];"),
    "backward_a_not_adjoint": ("for (int c = 0; c < m; c++) s += conj(Ak[c * m + a]) * Mt[c * m + b];",
                               "for (int c = 0; c < m; c++) s += Ak[a * m + c] * Mt[c * m + b];"),
    "lu_update_sign": ("for (int c = j + 1; c < n; c++) a[i * n + c] -= l * a[j * n + c];",
                       "for (int c = j + 1; c < n; c++) a[i * n + c] += l * a[j * n + c];"),
    "matsubara_factor_halved": ("cplx v = (acc[i * n + j] + conj(acc[j * n + i])) / beta;",
                                "cplx v = (acc[i * n + j] + conj(acc[j * n + i])) / (2.0 * beta);"),
    "rho_not_hermitian_part": ("cplx v = (acc[i * n + j] + conj(acc[j * n + i])) / beta;",
                               "cplx v = (acc[i * n + j] + conj(acc[i * n + j])) / beta;"),
    "second_tail_sign": ("if (tail_order >= 2) tail += M2[i * n + j] / (iw * iw);",
                         "if (tail_order >= 2) tail -= M2[i * n + j] / (iw * iw);"),
    "dndmu_missing_closed_tail": ("if (tail_order >= 2) dn += 0.25 * beta * n;", ""),
    "gloc_unweighted": ("for (size_t q = 0; q < mm; q++) acc[q] += wk[k] * Q[q];",
                        "for (size_t q = 0; q < mm; q++) acc[q] += Q[q];"),
    "occupation_unweighted": ("partN[3 * t + 0] += wk[k] * tr;", "partN[3 * t + 0] += tr;"),
    # the tail_order = 1 branch: the second moment subtracted anyway, or its exact sum added back
    # without it being subtracted
    "tail1_keeps_second_moment": ("if (tail_order >= 2) tail += M2[i * n + j] / (iw * iw);",
                                  "if (tail_order >= 1) tail += M2[i * n + j] / (iw * iw);"),
    "tail1_adds_second_sum": ("if (tail_order >= 2) v -= 0.25 * beta * M2[i * n + j];",
                              "if (tail_order >= 1) v -= 0.25 * beta * M2[i * n + j];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.SOURCE.read_text()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant = oracle.variant(src.replace(old, new), tmp_path)
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            err, tol = pin(mutant)
            if not err <= tol:
                caught.append(pin.__name__)
        except Exception as exc:  # a failed call also counts as caught
            caught.append(f"{pin.__name__} ({type(exc).__name__})")
        if caught:
            break
    assert caught, f"no pin catches the planted mistake {name}"
