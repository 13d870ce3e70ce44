"""The C ABI library loads and exports every symbol that include/sib.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1612_02208_gb300 import build, sib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "sib.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sib_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert header_symbols() == sorted(sib.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in header_symbols():
        assert hasattr(lib, name), name


def test_binding_signatures_and_defaults():
    lib = sib.load()
    o = sib.SibOpts()
    lib.sib_default_opts(ctypes.byref(o))
    assert (o.smoother, o.nu1, o.nu2, o.cheb_iters, o.max_it, o.restart, o.add_SKXn) == (0, 2, 2, 2, 100, 100, 1)
    assert o.rtol == 1e-8 and o.vcycle_fp32 == 1 and o.omega < 0
    assert lib.sib_last_error(None) == b"null context"
    assert lib.sib_num_levels(None) == sib.SIB_ERR_ARG


def test_create_rejects_bad_sizes_without_touching_the_device():
    lib = sib.load()
    c = ctypes.c_void_p()
    for N, nmin in ((48, 8), (8, 3), (4, 8), (16384, 8), (64, 32)):
        assert lib.sib_create(ctypes.byref(c), N, nmin) == sib.SIB_ERR_ARG
        assert not c.value


def test_create_fails_loudly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = sib.load()
    c = ctypes.c_void_p()
    rc = lib.sib_create(ctypes.byref(c), 32, 8)
    assert rc in (sib.SIB_ERR_CUDA, sib.SIB_ERR_ALLOC) and not c.value


def header_struct_fields(name):
    """(member, type) pairs of `typedef struct { ... } name;` in include/sib.h, in declaration order."""
    text = open(os.path.join(ROOT, "include", "sib.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct\s*\{(.*?)\}\s*" + name + r"\s*;", text, flags=re.S).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(int|double)\s+(.*)", decl)
        assert m, decl
        for member in m.group(2).split(","):
            out.append((member.strip(), m.group(1)))
    return out


def test_options_struct_layout_matches_the_header():
    """The ctypes mirror of sib_opts has the header's members in the same order with the same types
    (a shorter or reordered mirror would let sib_default_opts write past it or scramble options)."""
    ctype = {"int": ctypes.c_int, "double": ctypes.c_double}
    want = [(n, ctype[t]) for n, t in header_struct_fields("sib_opts")]
    assert [(n, t) for n, t in sib.SibOpts._fields_] == want
    lib = sib.load()
    o = sib.SibOpts()
    lib.sib_default_opts(ctypes.byref(o))
    assert (o.fuse_small, o.smooth_krylov, o.sc_relax, o.box, o.box_overlap) == (1, 0, sib.RELAX_JACOBI, 4, 1)
