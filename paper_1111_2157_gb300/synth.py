"""Seeded synthetic inputs shaped like the paper's Ce, Am and NiO workloads.

This module is the one thing the CUDA path and the CPU oracle share: it draws
H_k, P_k and a pole-form self-energy and holds none of the method's arithmetic
(no Green's function, projection, Matsubara sum or mu search).  All draws use
``numpy.random.Generator(PCG64(seed))``.

Recipes (energies in eV, beta in 1/eV):

* ``H_k``  -- band-window Hamiltonian.  ``diag``: diagonal, eigenvalues uniform in
  [lo, hi].  ``dense``: Hermitian, diagonal uniform in [lo, hi], off-diagonal
  complex Gaussian with E|h_ij|^2 = s^2 (real and imaginary parts N(0, s^2/2)).
* ``P_k``  -- m x N_b projector <alpha_k|phi_nk> with orthonormal rows: the
  conjugate transpose of Q from the QR of an N_b x m complex Gaussian (the
  rows of P are unit vectors, as Eq. S_norm asks of the full Bloch set).
* ``Sigma`` -- pole form Sigma(i w) = Sigma_inf + sum_i V_i^+ V_i / (i w - p_i)
  (Sec. 3.2.4, Eq. se_pole) with V_i a 1 x m row; causal (Im Sigma <= 0 for
  w > 0) because every weight |V_i|^2 is positive.  ``hubbard_diag``: U/2 +
  (U^2/4)/(i w - Delta) on every orbital.  ``two_pole``: two poles per orbital at
  +-U/2 + N(0, 0.1) with weight U^2/8 each, rotated by a seeded unitary (dense
  m x m).  ``afm``: the two-pole form per (atom, spin) block of 5 d orbitals,
  poles shifted by -delta / +delta for spin up / down on atom A and the
  opposite on atom B.  Sigma_inf = U/2 I.

The Matsubara grid on which Sigma is sampled is the fermionic w_n = (2n+1) pi/beta,
n = 0..N_w-1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1111_2157


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def hamiltonian_diag(rng, nk, nb, lo, hi):
    H = np.zeros((nk, nb, nb), np.complex128)
    e = rng.uniform(lo, hi, size=(nk, nb))
    idx = np.arange(nb)
    H[:, idx, idx] = e
    return H


def hamiltonian_dense(rng, nk, nb, lo, hi, s):
    d = rng.uniform(lo, hi, size=(nk, nb))
    X = (rng.standard_normal((nk, nb, nb)) + 1j * rng.standard_normal((nk, nb, nb))) * (s / np.sqrt(2.0))
    U = np.triu(X, 1)
    H = U + np.conj(np.swapaxes(U, 1, 2))
    idx = np.arange(nb)
    H[:, idx, idx] = d
    return np.ascontiguousarray(H)


def projectors(rng, nk, nb, m):
    Z = rng.standard_normal((nk, nb, m)) + 1j * rng.standard_normal((nk, nb, m))
    Q, _ = np.linalg.qr(Z)
    return np.ascontiguousarray(np.conj(np.swapaxes(Q, 1, 2)))


def unitary(rng, m):
    Z = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    Q, R = np.linalg.qr(Z)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


@dataclass
class PoleSigma:
    """Sigma(i w) = sigma_inf + sum_i V[i]^+ V[i] / (i w - p[i]); V is [np, m]."""
    sigma_inf: np.ndarray
    p: np.ndarray
    V: np.ndarray

    def sample(self, beta: float, n_iw: int) -> np.ndarray:
        wn = (2.0 * np.arange(n_iw) + 1.0) * np.pi / beta
        f = 1.0 / (1j * wn[:, None] - self.p[None, :])
        sig = np.einsum("ia,ni,ib->nab", np.conj(self.V), f, self.V)
        return np.ascontiguousarray(sig + self.sigma_inf[None])


def sigma_hubbard_diag(m, U, delta):
    sigma_inf = (U / 2.0) * np.eye(m, dtype=np.complex128)
    p = np.full(m, delta)
    V = (U / 2.0) * np.eye(m, dtype=np.complex128)
    return PoleSigma(sigma_inf, p, V)


def sigma_two_pole(rng, m, U, spread=0.1, shifts=None, rotation=True):
    """Two poles per orbital at +-U/2 (+ shift[alpha]) + N(0, spread), weights U^2/8."""
    shifts = np.zeros(m) if shifts is None else np.asarray(shifts, float)
    R = unitary(rng, m) if rotation else np.eye(m, dtype=np.complex128)
    p, V = [], []
    amp = np.sqrt(U * U / 8.0)
    for a in range(m):
        for sgn in (+1.0, -1.0):
            p.append(sgn * U / 2.0 + shifts[a] + spread * rng.standard_normal())
            V.append(amp * np.conj(R[:, a]))
    return PoleSigma((U / 2.0) * np.eye(m, dtype=np.complex128), np.array(p), np.array(V))


def sigma_afm(rng, U, delta=1.0, n_atoms=2, n_orb=5, spread=0.1):
    """Block-diagonal AFM self-energy over (atom, spin) blocks of n_orb orbitals."""
    m = n_atoms * 2 * n_orb
    p, V = [], []
    amp = np.sqrt(U * U / 8.0)
    for atom in range(n_atoms):
        for spin in range(2):
            sgn_shift = (-1.0 if spin == 0 else 1.0) * (1.0 if atom % 2 == 0 else -1.0)
            R = unitary(rng, n_orb)
            base = (atom * 2 + spin) * n_orb
            for a in range(n_orb):
                for sgn in (+1.0, -1.0):
                    p.append(sgn * U / 2.0 + sgn_shift * delta + spread * rng.standard_normal())
                    v = np.zeros(m, np.complex128)
                    v[base:base + n_orb] = amp * np.conj(R[:, a])
                    V.append(v)
    return PoleSigma((U / 2.0) * np.eye(m, dtype=np.complex128), np.array(p), np.array(V))


@dataclass
class System:
    """One lattice problem: H [nk, nb, nb] (or a list of ragged blocks), P [nk, m, nb]."""
    H: object
    P: object
    pole: PoleSigma
    sigma: np.ndarray
    beta: float
    n_target: float
    dtype: str = "c128"
    weights: np.ndarray | None = None
    h_diagonal: bool = False

    @property
    def nk(self):
        return len(self.H)

    @property
    def m(self):
        return self.P[0].shape[0]

    @property
    def n_iw(self):
        return self.sigma.shape[0]

    @property
    def sigma_inf(self):
        return self.pole.sigma_inf

    @property
    def nb(self):
        if isinstance(self.H, np.ndarray):
            return np.full(self.nk, self.H.shape[1], np.int32)
        return np.array([h.shape[0] for h in self.H], np.int32)


@dataclass
class Workload:
    name: str
    systems: list = field(default_factory=list)
    precision: str = "fp64"


def d_toy(nk=64, n_iw=256, seed=SEED_BASE + 1):
    """Plain FP64 d-shell toy: N_b=8, m=5, beta=40, H diagonal in [-5, 5], U=4, Delta=0.1."""
    rng = rng_for(seed)
    H = hamiltonian_diag(rng, nk, 8, -5.0, 5.0)
    P = projectors(rng, nk, 8, 5)
    pole = sigma_hubbard_diag(5, 4.0, 0.1)
    beta = 40.0
    return Workload("d_toy", [System(H, P, pole, pole.sample(beta, n_iw), beta, 5.0, h_diagonal=True)])


def ce_like(nk=1000, n_iw=1024, nb=40, m=14, beta=100.0, U=6.0, seed=SEED_BASE + 2, name="ce_like"):
    """Ce-like f-system: dense Hermitian H (diag [-8, 8], off-diag s=0.3), two-pole Sigma, U=6."""
    rng = rng_for(seed)
    H = hamiltonian_dense(rng, nk, nb, -8.0, 8.0, 0.3)
    P = projectors(rng, nk, nb, m)
    pole = sigma_two_pole(rng, m, U)
    return Workload(name, [System(H, P, pole, pole.sample(beta, n_iw), beta, nb / 2.0)])


def nio_like(nk=4096, n_iw=2048, nb=96, beta=40.0, U=8.0, seed=SEED_BASE + 3):
    """NiO-like AFM cell: 2 atoms x 5 d x 2 spin (m=20), N_b=96, beta=40, U=8."""
    rng = rng_for(seed)
    H = hamiltonian_dense(rng, nk, nb, -8.0, 8.0, 0.3)
    P = projectors(rng, nk, nb, 20)
    pole = sigma_afm(rng, U)
    return Workload("nio_like", [System(H, P, pole, pole.sample(beta, n_iw), beta, nb / 2.0)],
                    precision="mixed")


def batched(n_systems=8, n_iw=1024, nk_choices=(512, 1000, 2048, 4096), nb_range=(48, 128),
            m_range=(10, 14), beta=40.0, U=6.0, seed=SEED_BASE + 4, nk_scale=1.0):
    """Several systems with ragged band windows N_b(k) uniform in nb_range; half c128, half c64."""
    rng = rng_for(seed)
    systems = []
    for s in range(n_systems):
        nk = max(1, int(round(int(rng.choice(nk_choices)) * nk_scale)))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        nbs = rng.integers(max(nb_range[0], m), nb_range[1] + 1, size=nk)
        H, P = [], []
        for nb in nbs:
            H.append(hamiltonian_dense(rng, 1, int(nb), -8.0, 8.0, 0.3)[0])
            P.append(projectors(rng, 1, int(nb), m)[0])
        pole = sigma_two_pole(rng, m, U)
        n_target = float(np.mean(nbs)) / 2.0
        systems.append(System(H, P, pole, pole.sample(beta, n_iw), beta, n_target,
                              dtype="c128" if s % 2 == 0 else "c64"))
    return Workload("batched", systems)


def adjoint_case(nk=2048, n_iw=1024, seed=SEED_BASE + 5):
    """Differentiation workload: N_b=64, m=14, beta=100, Ce-like generators."""
    return ce_like(nk=nk, n_iw=n_iw, nb=64, m=14, beta=100.0, seed=seed, name="adjoint")


def random_system(seed, nk, nb, m, n_iw, beta, U=4.0, dense=True, n_target=None):
    """Small generic system for tests (dense H in [-4, 4], two-pole rotated Sigma)."""
    rng = rng_for(seed)
    if dense:
        H = hamiltonian_dense(rng, nk, nb, -4.0, 4.0, 0.3)
    else:
        H = hamiltonian_diag(rng, nk, nb, -4.0, 4.0)
    P = projectors(rng, nk, nb, m)
    pole = sigma_two_pole(rng, m, U)
    return System(H, P, pole, pole.sample(beta, n_iw), beta,
                  nb / 2.0 if n_target is None else n_target, h_diagonal=not dense)
