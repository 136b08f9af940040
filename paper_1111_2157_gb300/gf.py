"""Thin ctypes binding of libgf (include/gf.h).

Argument marshalling only: every step of the path runs in the CUDA library.
Arrays may be numpy arrays or torch tensors, on the host or on the context's
device; outputs are torch tensors on the device unless an ``out`` is given.
The library is loaded on first use; if it is missing the call fails loudly.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libgf.so"
_lib = None

GF_OK, GF_EINVAL, GF_ENOMEM, GF_ECUDA, GF_ESINGULAR, GF_ENOTCONV, GF_ETIMEOUT, GF_ESTATE = range(8)
STATUS_NAMES = {0: "GF_OK", 1: "GF_EINVAL", 2: "GF_ENOMEM", 3: "GF_ECUDA", 4: "GF_ESINGULAR",
                5: "GF_ENOTCONV", 6: "GF_ETIMEOUT", 7: "GF_ESTATE"}
PRECISION = {"fp64": 0, "mixed": 1, "pair": 2}
DTYPE = {"c128": 0, "c64": 1}

EXPORTS = ["gf_create", "gf_destroy", "gf_set_hamiltonian", "gf_set_projectors", "gf_set_sigma",
           "gf_local", "gf_occupation", "gf_find_mu", "gf_density_matrix", "gf_backward",
           "gf_evaluate", "gf_occupation_static", "gf_last_error", "gf_last_stats",
           "gf_tuning_log", "gf_set_sigma_poles", "gf_pole_occupation", "gf_pole_find_mu",
           "gf_pole_density_matrix", "gf_pole_local", "gf_heev_batched",
           "gf_set_projectors_lowdin", "gf_impurity_levels", "gf_hybridization",
           "gf_double_counting", "gf_pole_spectral", "gf_pole_energy"]


class GFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GFDesc(ctypes.Structure):
    _fields_ = [("n_systems", ctypes.c_int32), ("n_k", ctypes.c_int32),
                ("nb", ctypes.POINTER(ctypes.c_int32)), ("nb_uniform", ctypes.c_int32),
                ("k_system", ctypes.POINTER(ctypes.c_int32)),
                ("m_system", ctypes.POINTER(ctypes.c_int32)), ("n_iw", ctypes.c_int32),
                ("beta", ctypes.POINTER(ctypes.c_double)), ("k_weight", ctypes.POINTER(ctypes.c_double)),
                ("precision", ctypes.c_int32), ("input_dtype", ctypes.c_int32),
                ("tail_order", ctypes.c_int32), ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("flags", ctypes.c_int32), ("system_dtype", ctypes.POINTER(ctypes.c_int32))]
GF_FLAG_GRAPH = 1
GF_FLAG_LOWRANK = 2


def load():
    """Load libgf.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH.name} is not built: run `python -m paper_1111_2157_gb300.build` "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(str(LIB_PATH))
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    lib.gf_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(GFDesc)]
    lib.gf_destroy.argtypes = [vp]
    lib.gf_set_hamiltonian.argtypes = [vp, vp, ctypes.c_int32]
    lib.gf_set_projectors.argtypes = [vp, vp]
    lib.gf_set_sigma.argtypes = [vp, vp, vp]
    lib.gf_local.argtypes = [vp, dp, vp]
    lib.gf_occupation.argtypes = [vp, dp, dp, dp]
    lib.gf_find_mu.argtypes = [vp, dp, ctypes.c_double, ctypes.c_int32, dp, ip]
    lib.gf_density_matrix.argtypes = [vp, dp, vp, dp]
    lib.gf_backward.argtypes = [vp, dp, vp, dp, vp, dp]
    lib.gf_evaluate.argtypes = [vp, dp, vp, vp, dp, dp, dp]
    lib.gf_occupation_static.argtypes = [vp, vp, vp, vp, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int32, vp, dp, dp]
    lib.gf_set_sigma_poles.argtypes = [vp, ip, vp, vp, vp]
    lib.gf_pole_occupation.argtypes = [vp, dp, dp, dp]
    lib.gf_pole_find_mu.argtypes = [vp, dp, ctypes.c_double, ctypes.c_int32, dp, ip]
    lib.gf_pole_density_matrix.argtypes = [vp, dp, vp, dp]
    lib.gf_pole_local.argtypes = [vp, dp, vp]
    lib.gf_heev_batched.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, vp, vp]
    lib.gf_pole_spectral.argtypes = [vp, dp, ctypes.c_int32, dp, ctypes.c_double, dp, dp]
    lib.gf_pole_energy.argtypes = [vp, dp, dp, dp]
    lib.gf_set_projectors_lowdin.argtypes = [vp, vp, vp]
    lib.gf_impurity_levels.argtypes = [vp, dp, vp]
    lib.gf_hybridization.argtypes = [vp, dp, vp, dp, vp]
    lib.gf_double_counting.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                       ctypes.c_double, dp, dp, dp]
    lib.gf_last_error.argtypes = [vp]
    lib.gf_last_error.restype = ctypes.c_char_p
    lib.gf_tuning_log.argtypes = [vp]
    lib.gf_tuning_log.restype = ctypes.c_char_p
    lib.gf_last_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                  dp, dp]
    for name in EXPORTS:
        if name not in ("gf_last_error", "gf_tuning_log"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _is_tensor(x):
    import torch
    return isinstance(x, torch.Tensor)


def heev_batched(A, max_sweeps=40, stream=None):
    """Eigen-decomposition of a batch of Hermitian matrices A [n_mat, n, n]
    (complex128 CUDA tensor) by the library's Jacobi kernel: (w ascending, V)."""
    import torch
    lib = load()
    A = A.to(torch.complex128).contiguous()
    n_mat, n = A.shape[0], A.shape[-1]
    w = torch.empty((n_mat, n), dtype=torch.float64, device=A.device)
    V = torch.empty((n_mat, n, n), dtype=torch.complex128, device=A.device)
    if stream is None:
        stream = torch.cuda.current_stream(A.device).cuda_stream
    st = lib.gf_heev_batched(ctypes.c_void_p(A.data_ptr()), n_mat, n, int(max_sweeps),
                             ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                             ctypes.c_void_p(int(stream)))
    if st != GF_OK:
        raise GFError(st, lib.gf_last_error(None).decode())
    return w, V


def double_counting(U, J, l, n):
    """(U_bar, V_DC, E_DC) of the double-counting formulas (host arithmetic in libgf)."""
    lib = load()
    ub, vdc, edc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = lib.gf_double_counting(float(U), float(J), int(l), float(n), ctypes.byref(ub),
                                ctypes.byref(vdc), ctypes.byref(edc))
    if st != GF_OK:
        raise GFError(st, lib.gf_last_error(None).decode())
    return ub.value, vdc.value, edc.value


def _doubles(values, n):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(values, dtype=np.float64), (n,)))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class _Arg:
    """Pointer to array data (numpy or torch; host or device) kept alive for a call."""

    def __init__(self, x, complex_dtype=None):
        import torch
        if isinstance(x, (list, tuple)):
            x = np.concatenate([np.asarray(b).reshape(-1) for b in x])
        if isinstance(x, torch.Tensor):
            if complex_dtype is not None:
                x = x.to(dtype=getattr(torch, complex_dtype))
            self.obj = x.contiguous()
            self.ptr = self.obj.data_ptr()
        else:
            arr = np.asarray(x)
            if complex_dtype is not None:
                arr = arr.astype(np.dtype(complex_dtype), copy=False)
            self.obj = np.ascontiguousarray(arr)
            self.ptr = self.obj.ctypes.data


def _flat(x):
    import torch
    if isinstance(x, torch.Tensor):
        return x.reshape(-1)
    return np.asarray(x).reshape(-1)


class _SysArg:
    """Packed per-system input with a dtype per system: system s's block (counts[s] complex
    numbers) converted to dtypes[s] ("c128"/"c64"), the blocks concatenated as raw bytes.
    x is one packed array of sum(counts) numbers or a list of per-system arrays."""

    def __init__(self, x, counts, dtypes):
        import torch
        if isinstance(x, (list, tuple)):
            parts = [_flat(p) for p in x]
        else:
            flat, parts, off = _flat(x), [], 0
            for n in counts:
                parts.append(flat[off:off + n])
                off += n
        if any(len(p) != n for p, n in zip(parts, counts)) or len(parts) != len(counts):
            raise ValueError("per-system input sizes do not match the context")
        cd = {"c128": "complex128", "c64": "complex64"}
        if any(isinstance(p, torch.Tensor) for p in parts):
            dev = next(p.device for p in parts if isinstance(p, torch.Tensor))
            bufs = []
            for p, d in zip(parts, dtypes):
                t = p if isinstance(p, torch.Tensor) else torch.from_numpy(np.asarray(p))
                t = t.to(device=dev, dtype=getattr(torch, cd[d])).contiguous()
                bufs.append(torch.view_as_real(t).reshape(-1).view(torch.uint8))
            self.obj = torch.cat(bufs)
            self.ptr = self.obj.data_ptr()
        else:
            self.obj = np.concatenate([np.ascontiguousarray(p, dtype=cd[d]).view(np.uint8)
                                       for p, d in zip(parts, dtypes)])
            self.ptr = self.obj.ctypes.data


class GreensFunction:
    """One libgf context: inputs live on the device, every call runs the CUDA path.

    nb: int (uniform) or per-k sequence; m and beta: per system (scalars for one
    system); k_system: per-k system index (non-decreasing) for several systems;
    input_dtype: "c128", "c64", or a list with one of them per system (the inputs of the
    gf_set_* calls are then packed with each system's block in its own dtype).
    """

    def __init__(self, nb, m, n_iw, beta, k_system=None, n_k=None, k_weight=None, precision="fp64",
                 input_dtype="c128", tail_order=2, device=0, stream=None, graph=False, lowrank=False):
        import torch
        self.lib = load()
        self.device = int(device)
        self.sys_dtypes = None
        if isinstance(input_dtype, (list, tuple)):
            self.sys_dtypes = [str(t) for t in input_dtype]
            input_dtype = self.sys_dtypes[0]
        self.input_dtype = input_dtype
        m = np.atleast_1d(np.asarray(m, dtype=np.int32))
        beta = np.atleast_1d(np.asarray(beta, dtype=np.float64))
        n_sys = len(m)
        if np.ndim(nb) == 0:
            if n_k is None:
                raise ValueError("n_k is required with a uniform nb")
            nb_arr = None
            self.nb = np.full(int(n_k), int(nb), np.int32)
        else:
            nb_arr = np.ascontiguousarray(nb, dtype=np.int32)
            self.nb = nb_arr
        n_k = len(self.nb)
        ks = None if k_system is None else np.ascontiguousarray(k_system, dtype=np.int32)
        self.k_system = np.zeros(n_k, np.int32) if ks is None else ks
        self.m, self.beta, self.n_iw, self.n_sys, self.n_k = m, beta, int(n_iw), n_sys, n_k
        kw = None if k_weight is None else np.ascontiguousarray(k_weight, dtype=np.float64)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream if torch.cuda.is_available() else 0
        sd = (np.ascontiguousarray([DTYPE[t] for t in self.sys_dtypes], dtype=np.int32)
              if self.sys_dtypes is not None else None)
        if sd is not None and len(sd) != n_sys:
            raise ValueError("input_dtype list must have one entry per system")
        self._keep = [nb_arr, ks, m, beta, kw, sd]
        d = GFDesc()
        d.n_systems, d.n_k = n_sys, n_k
        d.nb = nb_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if nb_arr is not None else None
        d.nb_uniform = int(self.nb[0])
        d.k_system = ks.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if ks is not None else None
        d.m_system = m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.n_iw = self.n_iw
        d.beta = beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.k_weight = kw.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if kw is not None else None
        d.precision = PRECISION[precision]
        d.input_dtype = DTYPE[input_dtype]
        d.tail_order = int(tail_order)
        d.device = self.device
        d.stream = int(stream)
        d.flags = (GF_FLAG_GRAPH if graph else 0) | (GF_FLAG_LOWRANK if lowrank else 0)
        d.system_dtype = sd.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if sd is not None else None
        h = ctypes.c_void_p()
        st = self.lib.gf_create(ctypes.byref(h), ctypes.byref(d))
        if st != GF_OK:
            raise GFError(st, self.lib.gf_last_error(None).decode())
        self.h = h
        msys = self.m[self.k_system]
        self.tot_h = int(np.sum(self.nb.astype(np.int64) ** 2))
        self.tot_p = int(np.sum(msys.astype(np.int64) * self.nb))
        self.tot_sig = int(np.sum(self.n_iw * self.m.astype(np.int64) ** 2))
        self.tot_sinf = int(np.sum(self.m.astype(np.int64) ** 2))
        nb64 = self.nb.astype(np.int64)
        self._cnt = {
            "H": [int(np.sum(nb64[self.k_system == s] ** 2)) for s in range(n_sys)],
            "Hd": [int(np.sum(nb64[self.k_system == s])) for s in range(n_sys)],
            "P": [int(self.m[s]) * int(np.sum(nb64[self.k_system == s])) for s in range(n_sys)],
            "Sig": [self.n_iw * int(self.m[s]) ** 2 for s in range(n_sys)],
            "Sinf": [int(self.m[s]) ** 2 for s in range(n_sys)]}

    @classmethod
    def for_systems(cls, systems, precision="fp64", input_dtype="c128", tail_order=2, device=0,
                    graph=False, lowrank=False):
        """Context for a list of ``synth.System`` (one or several, ragged or not);
        input_dtype="per_system" takes each system's own ``dtype``."""
        if input_dtype == "per_system":
            input_dtype = [s.dtype for s in systems]
        nb = np.concatenate([s.nb for s in systems])
        ks = np.concatenate([np.full(s.nk, i, np.int32) for i, s in enumerate(systems)])
        n_iw = systems[0].n_iw
        return cls(nb, [s.m for s in systems], n_iw, [s.beta for s in systems],
                   k_system=ks if len(systems) > 1 else None, precision=precision,
                   input_dtype=input_dtype, tail_order=tail_order, device=device, graph=graph,
                   lowrank=lowrank)

    def _check(self, st):
        if st != GF_OK:
            raise GFError(st, self.lib.gf_last_error(self.h).decode())

    def _cdt(self):
        return "complex128" if self.input_dtype == "c128" else "complex64"

    def _in(self, x, kind):
        """Marshal an input array of the given kind (H, Hd, P, Sig, Sinf)."""
        if self.sys_dtypes is not None:
            return _SysArg(x, self._cnt[kind], self.sys_dtypes)
        return _Arg(x, self._cdt())

    def close(self):
        if getattr(self, "h", None):
            self.lib.gf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, n, out):
        import torch
        if out is None:
            out = torch.empty(n, dtype=torch.complex128, device=f"cuda:{self.device}")
        return out

    # ---------------------------------------------------------------- inputs
    def set_hamiltonian(self, H, diagonal=False):
        a = self._in(H, "Hd" if diagonal else "H")
        self._check(self.lib.gf_set_hamiltonian(self.h, a.ptr, 1 if diagonal else 0))

    def set_projectors(self, P):
        a = self._in(P, "P")
        self._check(self.lib.gf_set_projectors(self.h, a.ptr))

    def set_sigma(self, sigma, sigma_inf):
        a, b = self._in(sigma, "Sig"), self._in(sigma_inf, "Sinf")
        self._check(self.lib.gf_set_sigma(self.h, a.ptr, b.ptr))

    # --------------------------------------------------------------- compute
    def local(self, mu, out=None):
        """G_loc packed per system [n_iw][m][m], complex128."""
        _, mp = _doubles(mu, self.n_sys)
        out = self._out(self.tot_sig, out)
        o = _Arg(out)
        self._check(self.lib.gf_local(self.h, mp, ctypes.c_void_p(o.ptr)))
        return out

    def occupation(self, mu):
        """(N, dN/dmu) per system."""
        keep, mp = _doubles(mu, self.n_sys)
        n, d = np.zeros(self.n_sys), np.zeros(self.n_sys)
        self._check(self.lib.gf_occupation(self.h, mp, n.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return n, d

    def find_mu(self, n_target, mu0=0.0, tol=1e-10, max_iter=60):
        """mu per system with |N - n_target| <= tol; returns (mu, evaluations)."""
        _, tp = _doubles(n_target, self.n_sys)
        mu = np.ascontiguousarray(np.broadcast_to(np.asarray(mu0, np.float64), (self.n_sys,))).copy()
        it = ctypes.c_int32()
        self._check(self.lib.gf_find_mu(self.h, tp, float(tol), int(max_iter),
                                        mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        ctypes.byref(it)))
        return mu, it.value

    def density_matrix(self, mu, out=None, want_rho=True):
        """(rho packed per k [N_b][N_b] complex128 or None, n_corr per system)."""
        _, mp = _doubles(mu, self.n_sys)
        nc = np.zeros(self.n_sys)
        o = _Arg(self._out(self.tot_h, out)) if want_rho else None
        self._check(self.lib.gf_density_matrix(self.h, mp, ctypes.c_void_p(o.ptr if o else 0),
                                               nc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return (o.obj if o else None), nc

    def evaluate(self, mu, gloc=True, rho=True, occupation=True, n_corr=True, gloc_out=None,
                 rho_out=None):
        """One fused pass: dict(gloc, rho, N, dN_dmu, n_corr) for the requested outputs."""
        _, mp = _doubles(mu, self.n_sys)
        go = _Arg(self._out(self.tot_sig, gloc_out)) if gloc else None
        ro = _Arg(self._out(self.tot_h, rho_out)) if rho else None
        n, d, nc = np.zeros(self.n_sys), np.zeros(self.n_sys), np.zeros(self.n_sys)
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        self._check(self.lib.gf_evaluate(
            self.h, mp, ctypes.c_void_p(go.ptr if go else 0), ctypes.c_void_p(ro.ptr if ro else 0),
            dptr(n) if occupation else None, dptr(d) if occupation else None,
            dptr(nc) if n_corr else None))
        return {"gloc": go.obj if go else None, "rho": ro.obj if ro else None,
                "N": n if occupation else None, "dN_dmu": d if occupation else None,
                "n_corr": nc if n_corr else None}

    def backward(self, mu, gloc_bar=None, n_bar=None, out=None):
        """(Sigma_bar packed like Sigma, complex128; mu_bar per system)."""
        _, mp = _doubles(mu, self.n_sys)
        gb = _Arg(gloc_bar, "complex128") if gloc_bar is not None else None
        nb_keep = None
        nbp = None
        if n_bar is not None:
            nb_keep, nbp = _doubles(n_bar, self.n_sys)
        out = self._out(self.tot_sig, out)
        o = _Arg(out)
        mub = np.zeros(self.n_sys)
        self._check(self.lib.gf_backward(self.h, mp, ctypes.c_void_p(gb.ptr if gb else 0), nbp,
                                         ctypes.c_void_p(o.ptr),
                                         mub.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out, mub

    # ------------------------------------- projectors and the DMFT step
    def set_projectors_lowdin(self, W, out=None):
        """Make P_k = (W_k W_k^+)^{-1/2} W_k the projectors; returns P (complex128)."""
        a = self._in(W, "P")
        out = self._out(self.tot_p, out)
        o = _Arg(out)
        self._check(self.lib.gf_set_projectors_lowdin(self.h, a.ptr, ctypes.c_void_p(o.ptr)))
        return out

    def impurity_levels(self, v_dc=None, out=None):
        """E_imp = sum_k w_k P H P^+ - V_DC, packed [sum m_s^2] complex128."""
        keep, vp_ = (None, None) if v_dc is None else _doubles(v_dc, self.n_sys)
        out = self._out(self.tot_sinf, out)
        o = _Arg(out)
        self._check(self.lib.gf_impurity_levels(self.h, vp_, ctypes.c_void_p(o.ptr)))
        return out

    def hybridization(self, mu, gloc, v_dc=None, out=None):
        """Delta(i w_n) = (i w_n + mu) - E_imp - Sigma - G_loc^{-1}, packed like Sigma."""
        _, mp = _doubles(mu, self.n_sys)
        keep, vp_ = (None, None) if v_dc is None else _doubles(v_dc, self.n_sys)
        g = _Arg(gloc, "complex128")
        out = self._out(self.tot_sig, out)
        o = _Arg(out)
        self._check(self.lib.gf_hybridization(self.h, mp, g.ptr, vp_, ctypes.c_void_p(o.ptr)))
        return out

    # ------------------------------------------------ pole (pseudo-H) path
    def set_sigma_poles(self, n_poles, poles, V, sigma_inf):
        """Pole form of Sigma per system: n_poles [n_sys], poles [sum n_p] real,
        V [sum n_p * m_s] complex (row i = V_i), sigma_inf packed [sum m_s^2]."""
        npl = np.ascontiguousarray(np.atleast_1d(n_poles), dtype=np.int32)
        pa = _Arg(np.asarray(poles, dtype=np.float64).reshape(-1) if not _is_tensor(poles) else
                  poles.double().reshape(-1))
        if self.sys_dtypes is not None:
            cnt_v = [int(n) * int(m) for n, m in zip(npl, self.m)]
            va, sa = _SysArg(V, cnt_v, self.sys_dtypes), self._in(sigma_inf, "Sinf")
        else:
            va, sa = _Arg(V, self._cdt()), _Arg(sigma_inf, self._cdt())
        self._check(self.lib.gf_set_sigma_poles(self.h, npl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                pa.ptr, va.ptr, sa.ptr))

    def pole_occupation(self, mu):
        """(N, dN/dmu) per system from the pseudo-Hamiltonian eigenpairs."""
        _, mp = _doubles(mu, self.n_sys)
        n, d = np.zeros(self.n_sys), np.zeros(self.n_sys)
        self._check(self.lib.gf_pole_occupation(self.h, mp, n.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return n, d

    def pole_find_mu(self, n_target, mu0=0.0, tol=1e-10, max_iter=60):
        _, tp = _doubles(n_target, self.n_sys)
        mu = np.ascontiguousarray(np.broadcast_to(np.asarray(mu0, np.float64), (self.n_sys,))).copy()
        it = ctypes.c_int32()
        self._check(self.lib.gf_pole_find_mu(self.h, tp, float(tol), int(max_iter),
                                             mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             ctypes.byref(it)))
        return mu, it.value

    def pole_density_matrix(self, mu, out=None, want_rho=True):
        _, mp = _doubles(mu, self.n_sys)
        nc = np.zeros(self.n_sys)
        o = _Arg(self._out(self.tot_h, out)) if want_rho else None
        self._check(self.lib.gf_pole_density_matrix(self.h, mp, ctypes.c_void_p(o.ptr if o else 0),
                                                    nc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return (o.obj if o else None), nc

    def pole_local(self, mu, out=None):
        _, mp = _doubles(mu, self.n_sys)
        out = self._out(self.tot_sig, out)
        o = _Arg(out)
        self._check(self.lib.gf_pole_local(self.h, mp, ctypes.c_void_p(o.ptr)))
        return out

    def pole_spectral(self, mu, eps, eta, pdos=True):
        """(DOS [n_sys, n_eps], PDOS per system [n_eps, m_s] or None) on the real axis."""
        _, mp = _doubles(mu, self.n_sys)
        e = np.ascontiguousarray(eps, dtype=np.float64)
        dos = np.zeros((self.n_sys, len(e)))
        pd = np.zeros(len(e) * int(np.sum(self.m))) if pdos else None
        dp_ = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.gf_pole_spectral(self.h, mp, len(e), e.ctypes.data_as(dp_), float(eta),
                                              dos.ctypes.data_as(dp_),
                                              pd.ctypes.data_as(dp_) if pdos else None))
        if not pdos:
            return dos, None
        out, off = [], 0
        for m in self.m:
            out.append(pd[off:off + len(e) * m].reshape(len(e), m))
            off += len(e) * m
        return dos, out

    def pole_energy(self, mu):
        """(h_ks, e_ps) per system: Tr(H rho) and sum_l (E_l - mu)|Psi_b,l|^2 n_F."""
        _, mp = _doubles(mu, self.n_sys)
        a, b = np.zeros(self.n_sys), np.zeros(self.n_sys)
        dp_ = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.gf_pole_energy(self.h, mp, a.ctypes.data_as(dp_), b.ctypes.data_as(dp_)))
        return a, b

    def tuning_log(self):
        """Kernel configuration chosen for this context (autotuner report)."""
        return self.lib.gf_tuning_log(self.h).decode()

    def stats(self):
        """dict(launches, points, kernel_ms, flops) of the last compute call."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        ms, fl = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.gf_last_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms),
                                           ctypes.byref(fl)))
        return {"launches": a.value, "points": b.value, "kernel_ms": ms.value, "flops": fl.value}
