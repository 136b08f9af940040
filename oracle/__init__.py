"""Plain FP64 CPU oracle for the lattice Green's function path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``gf_oracle.c`` (compiled with
gcc into ``liboracle.so`` beside it) with ctypes.  Nothing here shares code with
the CUDA library.

Every function follows the definitions of arXiv:1111.2157:

* ``green``    -- one G(k, i w_n) = [(i w_n + mu) I - H_k - P_k^+ Sigma P_k]^{-1}
                  (Sec. 3.2.2, Eq. dmftloop1)
* ``local``    -- G_loc(i w_n) = sum_k w_k P_k G P_k^+ (the k-sum inside Eq. dmftloop2)
* ``density``  -- rho_k, N = sum_k w_k Tr rho_k, n_corr and dN/dmu
                  (Sec. 3.3 Eq. rho_LDA+DMFT and Eq. fix_mu; Sec. 3.4 Eq. nf_LDA+DMFT)
* ``find_mu``  -- N(mu) = N_target by Brent's method (Sec. 3.3, Eq. fix_mu)
* ``backward`` -- vector-Jacobian product of (G_loc, N) w.r.t. (Sigma(i w_n), mu)
                  (not in the paper; derived from the same definitions)

The Matsubara tail (1/(i w) and 1/(i w)^2 moments) is this implementation's
reading of Eq. rho_LDA+DMFT, which the paper writes without one; the header of
``gf_oracle.c`` gives the formulas.

Pins (``tests/test_oracle_pins.py``): the Sigma = 0 closed forms from the band
eigenvalues, the pseudo-Hamiltonian closed form of Sec. 3.3 for pole-form Sigma,
the 2 x 2 inverse written out, the high-frequency moment of G, the symmetry
G(-i w) = G(i w)^+, non-negative spectral weight, and central finite
differences for ``backward``.  ``tests/test_oracle_mutations.py`` plants
mistakes in a copy of the C source and checks that a pin catches each one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
SOURCE = _HERE / "gf_oracle.c"
_LIB = _HERE / "liboracle.so"

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def compile_source(src: Path, out: Path) -> Path:
    """gcc -O2 -fopenmp -shared; written to a temporary name, then renamed."""
    tmp = out.with_name(out.name + f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
           str(src), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> Path:
    """Compile gf_oracle.c into liboracle.so (when missing or older than the source)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < SOURCE.stat().st_mtime:
        compile_source(SOURCE, _LIB)
    return _LIB


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _pack(H, P):
    """Accept uniform ([nk, nb, nb], [nk, m, nb]) arrays or ragged lists of per-k blocks."""
    if isinstance(H, np.ndarray) and H.ndim == 3:
        nk, nb = H.shape[0], H.shape[1]
        nbs = np.full(nk, nb, dtype=np.int32)
        Hp, Pp = _c128(H).reshape(-1), _c128(P).reshape(-1)
        m = P.shape[1]
    else:
        nbs = np.array([h.shape[0] for h in H], dtype=np.int32)
        m = P[0].shape[0]
        Hp = _c128(np.concatenate([np.asarray(h).reshape(-1) for h in H]))
        Pp = _c128(np.concatenate([np.asarray(p).reshape(-1) for p in P]))
    return nbs, m, Hp, Pp


def _weights(nk, w):
    if w is None:
        return np.full(nk, 1.0 / nk)
    return np.ascontiguousarray(w, dtype=np.float64)


class Oracle:
    """ctypes binding of one compiled copy of gf_oracle.c."""

    def __init__(self, lib_path: Path):
        lib = ctypes.CDLL(str(lib_path))
        lib.gfo_matsubara.restype = ctypes.c_double
        lib.gfo_matsubara.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.gfo_set_threads.argtypes = [ctypes.c_int]
        lib.gfo_get_threads.restype = ctypes.c_int
        lib.gfo_green.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double,
                                  ctypes.c_double, _dp]
        lib.gfo_local.argtypes = [ctypes.c_int, _ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, _ip,
                                  _dp, ctypes.c_double, ctypes.c_double, _dp]
        lib.gfo_density.argtypes = [ctypes.c_int, _ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int,
                                    _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp]
        lib.gfo_find_mu.argtypes = [ctypes.c_int, _ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int,
                                    _dp, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    _dp, _dp, _ip]
        lib.gfo_backward.argtypes = [ctypes.c_int, _ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int,
                                     _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp,
                                     ctypes.c_double, _dp, _dp]
        self.lib = lib

    def set_threads(self, n: int) -> None:
        self.lib.gfo_set_threads(int(n))

    def get_threads(self) -> int:
        return int(self.lib.gfo_get_threads())

    def matsubara(self, n: int, beta: float) -> float:
        """w_n = (2n+1) pi / beta."""
        return float(self.lib.gfo_matsubara(int(n), float(beta)))

    def green(self, H_k, P_k, sigma_n, wn, mu):
        """One G(k, i w_n) (Eq. dmftloop1), nb x nb complex128."""
        H_k, P_k, sigma_n = _c128(H_k), _c128(P_k), _c128(sigma_n)
        nb, m = H_k.shape[0], P_k.shape[0]
        G = np.empty((nb, nb), np.complex128)
        rc = self.lib.gfo_green(nb, m, _ptr(H_k), _ptr(P_k), _ptr(sigma_n), float(wn), float(mu),
                                _ptr(G))
        if rc:
            raise RuntimeError(f"oracle green failed ({rc})")
        return G

    def local(self, H, P, sigma, beta, mu, n_idx=None, weights=None):
        """G_loc(i w_n) at frequency indices ``n_idx`` (default: all of sigma's), [n, m, m]."""
        nbs, m, Hp, Pp = _pack(H, P)
        nk = len(nbs)
        sigma = _c128(sigma)
        if n_idx is None:
            n_idx = np.arange(sigma.shape[0])
            sig_sel = sigma
        else:
            n_idx = np.asarray(n_idx)
            sig_sel = _c128(sigma[n_idx])
        idx = np.ascontiguousarray(n_idx, dtype=np.int32)
        w = _weights(nk, weights)
        out = np.zeros((len(idx), m, m), np.complex128)
        rc = self.lib.gfo_local(nk, nbs.ctypes.data_as(_ip), m, _ptr(Hp), _ptr(Pp), _ptr(w),
                                len(idx), idx.ctypes.data_as(_ip), _ptr(sig_sel), float(beta),
                                float(mu), _ptr(out))
        if rc:
            raise RuntimeError(f"oracle local failed ({rc})")
        return out

    def density(self, H, P, sigma, sigma_inf, beta, mu, weights=None, tail_order=2, want_rho=True):
        """Matsubara sum: dict(N, n_corr, dN_dmu, rho) (rho per k, or None)."""
        nbs, m, Hp, Pp = _pack(H, P)
        nk = len(nbs)
        sigma, sigma_inf = _c128(sigma), _c128(sigma_inf)
        w = _weights(nk, weights)
        tot = int(np.sum(nbs.astype(np.int64) ** 2))
        rho = np.zeros(tot, np.complex128) if want_rho else None
        o = np.zeros(3)
        rc = self.lib.gfo_density(nk, nbs.ctypes.data_as(_ip), m, _ptr(Hp), _ptr(Pp), _ptr(w),
                                  sigma.shape[0], _ptr(sigma), _ptr(sigma_inf), float(beta),
                                  float(mu), int(tail_order), _ptr(rho) if want_rho else None,
                                  _ptr(o))
        if rc:
            raise RuntimeError(f"oracle density failed ({rc})")
        if want_rho:
            if np.all(nbs == nbs[0]):
                rho = rho.reshape(nk, nbs[0], nbs[0])
            else:
                out, off = [], 0
                for n in nbs:
                    out.append(rho[off:off + n * n].reshape(n, n))
                    off += n * n
                rho = out
        return {"N": o[0], "n_corr": o[1], "dN_dmu": o[2], "rho": rho}

    def find_mu(self, H, P, sigma, sigma_inf, beta, n_target, mu_lo, mu_hi, weights=None,
                tail_order=2, tol=1e-12, max_iter=200):
        """mu with N(mu) = n_target (Eq. fix_mu); returns (mu, N, evaluations)."""
        nbs, m, Hp, Pp = _pack(H, P)
        nk = len(nbs)
        sigma, sigma_inf = _c128(sigma), _c128(sigma_inf)
        w = _weights(nk, weights)
        mu, nn, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        rc = self.lib.gfo_find_mu(nk, nbs.ctypes.data_as(_ip), m, _ptr(Hp), _ptr(Pp), _ptr(w),
                                  sigma.shape[0], _ptr(sigma), _ptr(sigma_inf), float(beta),
                                  int(tail_order), float(n_target), float(mu_lo), float(mu_hi),
                                  float(tol), int(max_iter), ctypes.byref(mu), ctypes.byref(nn),
                                  ctypes.byref(it))
        if rc:
            raise RuntimeError(f"oracle find_mu failed ({rc})")
        return mu.value, nn.value, it.value

    def backward(self, H, P, sigma, sigma_inf, beta, mu, gloc_bar=None, n_bar=0.0, weights=None,
                 tail_order=2):
        """(Sigma_bar [n_w, m, m], mu_bar) for L with dL = Re<gloc_bar, dG_loc> + n_bar dN."""
        nbs, m, Hp, Pp = _pack(H, P)
        nk = len(nbs)
        sigma, sigma_inf = _c128(sigma), _c128(sigma_inf)
        w = _weights(nk, weights)
        gb = None if gloc_bar is None else _c128(gloc_bar)
        sbar = np.zeros_like(sigma)
        mub = ctypes.c_double()
        rc = self.lib.gfo_backward(nk, nbs.ctypes.data_as(_ip), m, _ptr(Hp), _ptr(Pp), _ptr(w),
                                   sigma.shape[0], _ptr(sigma), _ptr(sigma_inf), float(beta),
                                   float(mu), int(tail_order), None if gb is None else _ptr(gb),
                                   float(n_bar), _ptr(sbar), ctypes.byref(mub))
        if rc:
            raise RuntimeError(f"oracle backward failed ({rc})")
        return sbar, mub.value


_default: Oracle | None = None


def get() -> Oracle:
    """The oracle built from gf_oracle.c (compiled on first use)."""
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def variant(src_text: str, workdir: Path) -> Oracle:
    """Compile an edited copy of the oracle source (used to plant mistakes in tests)."""
    workdir = Path(workdir)
    src = workdir / "gf_oracle_variant.c"
    src.write_text(src_text)
    out = workdir / f"liboracle_variant_{abs(hash(src_text)) % 10**12}.so"
    return Oracle(compile_source(src, out))
