"""The C-ABI library loads and exports every entry point include/gf.h declares (no GPU needed)."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

from paper_1111_2157_gb300 import build as gfbuild
from paper_1111_2157_gb300 import gf

ROOT = Path(__file__).resolve().parent.parent


def declared_symbols():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        names |= set(re.findall(r"^\s*(?:gf_status|const char \*)\s*(gf_\w+)\s*\(", text, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    gfbuild.build()
    return gf.load()


def test_header_declares_the_boundary():
    want = {"gf_create", "gf_destroy", "gf_set_hamiltonian", "gf_set_projectors", "gf_set_sigma",
            "gf_local", "gf_occupation", "gf_find_mu", "gf_density_matrix", "gf_backward",
            "gf_last_error"}
    assert want <= declared_symbols()


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(declared_symbols()):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_python_binding_names_match_header():
    assert set(gf.EXPORTS) == declared_symbols()


def _desc(**kw):
    m = (ctypes.c_int32 * 1)(5)
    beta = (ctypes.c_double * 1)(40.0)
    d = gf.GFDesc()
    d.n_systems, d.n_k, d.nb, d.nb_uniform = 1, 4, None, 8
    d.k_system, d.m_system, d.n_iw, d.beta, d.k_weight = None, m, 16, beta, None
    d.precision, d.input_dtype, d.tail_order, d.device, d.stream, d.flags = 0, 0, 2, 0, None, 0
    for k, v in kw.items():
        setattr(d, k, v)
    return d, (m, beta)


@pytest.mark.parametrize("field,value", [("n_systems", 0), ("n_k", 0), ("n_iw", 0),
                                         ("nb_uniform", 0), ("tail_order", 3), ("precision", 7),
                                         ("input_dtype", 5)])
def test_create_rejects_invalid_descriptor(lib, field, value):
    d, keep = _desc(**{field: value})
    h = ctypes.c_void_p()
    st = lib.gf_create(ctypes.byref(h), ctypes.byref(d))
    assert st == gf.GF_EINVAL
    assert not h.value
    assert lib.gf_last_error(None).decode()


def test_create_rejects_invalid_system_dtype(lib):
    sd = (ctypes.c_int32 * 1)(7)
    d, keep = _desc(system_dtype=sd)
    h = ctypes.c_void_p()
    assert lib.gf_create(ctypes.byref(h), ctypes.byref(d)) == gf.GF_EINVAL
    assert not h.value
    assert "system_dtype" in lib.gf_last_error(None).decode()


def test_per_system_packing_of_inputs():
    """The binding packs each system's block in its own dtype, blocks one after the other."""
    a = np.arange(6) + 1j * np.arange(6)
    x = gf._SysArg(a, [2, 4], ["c128", "c64"])
    assert x.obj.nbytes == 2 * 16 + 4 * 8
    assert np.array_equal(x.obj[:32].view(np.complex128), a[:2])
    assert np.array_equal(x.obj[32:].view(np.complex64), a[2:].astype(np.complex64))


def test_create_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.gf_create(ctypes.byref(h), None) == gf.GF_EINVAL
    assert lib.gf_create(None, None) == gf.GF_EINVAL
    assert lib.gf_destroy(None) == gf.GF_OK


def test_no_cpu_fallback_without_device(lib):
    """Without a usable GPU the library refuses to create a context (no CPU path exists)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    d, keep = _desc()
    h = ctypes.c_void_p()
    assert lib.gf_create(ctypes.byref(h), ctypes.byref(d)) == gf.GF_ECUDA
    assert not h.value


def _arr(ctype, vals):
    return (ctype * len(vals))(*vals)


@pytest.mark.parametrize("case,message", [
    ("nb_zero", "N_b(k)"), ("k_system_range", "k_system out of range"),
    ("k_system_order", "non-decreasing"), ("m_zero", "every m"), ("beta_zero", "beta"),
    ("empty_system", "no k-points"), ("weight_nan", "k_weight")])
def test_create_rejects_inconsistent_tables(lib, case, message):
    """Per-k and per-system tables are checked before any CUDA call; the half-built context is
    freed and *out stays NULL."""
    keep = []
    if case == "nb_zero":
        kw = dict(nb=_arr(ctypes.c_int32, [8, 8, 0, 8]))
    elif case == "k_system_range":
        kw = dict(k_system=_arr(ctypes.c_int32, [0, 0, 1, 1]))
    elif case == "k_system_order":
        kw = dict(n_systems=2, k_system=_arr(ctypes.c_int32, [0, 1, 0, 1]),
                  m_system=_arr(ctypes.c_int32, [5, 5]), beta=_arr(ctypes.c_double, [40.0, 40.0]))
    elif case == "m_zero":
        kw = dict(m_system=_arr(ctypes.c_int32, [0]))
    elif case == "beta_zero":
        kw = dict(beta=_arr(ctypes.c_double, [0.0]))
    elif case == "empty_system":
        kw = dict(n_systems=2, k_system=_arr(ctypes.c_int32, [0, 0, 0, 0]),
                  m_system=_arr(ctypes.c_int32, [5, 5]), beta=_arr(ctypes.c_double, [40.0, 40.0]))
    else:
        kw = dict(k_weight=_arr(ctypes.c_double, [0.25, float("nan"), 0.25, 0.25]))
    keep.append(kw)
    d, _ = _desc(**kw)
    h = ctypes.c_void_p()
    assert lib.gf_create(ctypes.byref(h), ctypes.byref(d)) == gf.GF_EINVAL
    assert not h.value
    assert message in lib.gf_last_error(None).decode()


def declared_prototypes():
    """{name: (return type, [parameter types])} of every prototype in include/*.h."""
    protos = {}
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", " ", h.read_text(), flags=re.S)
        for ret, name, params in re.findall(
                r"^\s*(gf_status|const char \*)\s*(gf_\w+)\s*\(([^;]*?)\)\s*;", text, re.M):
            types = []
            for p in " ".join(params.split()).split(","):
                p = p.strip()
                if p in ("", "void"):
                    continue
                types.append(re.sub(r"\s*\b\w+$", "", p) if not p.endswith("*") else p)
            protos[name] = (ret, types)
    return protos


def _kind_of_c(t):
    if "*" in t:
        return "pointer"
    return {"int32_t": "int32", "int": "int32", "double": "double"}[t.replace("const ", "").strip()]


def _kind_of_ctypes(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "pointer"
    if t is ctypes.c_int32:
        return "int32"
    if t is ctypes.c_double:
        return "double"
    return repr(t)


def test_binding_signatures_match_the_header():
    """Every ctypes argtypes/restype of the binding has the header's arity and the same kind
    (pointer, int32, double) at each position, so no pointer is truncated to an int."""
    lib = gf.load()
    protos = declared_prototypes()
    assert set(protos) == set(gf.EXPORTS)
    for name, (ret, params) in sorted(protos.items()):
        fn = getattr(lib, name)
        got = [_kind_of_ctypes(t) for t in fn.argtypes]
        want = [_kind_of_c(t) for t in params]
        assert got == want, f"{name}: binding {got}, header {want}"
        assert fn.restype is (ctypes.c_char_p if ret.startswith("const char") else ctypes.c_int), name
