"""CPU checks of the C-ABI boundary: libsaa builds, loads, exports every
entry point that include/saa.h declares, and fails cleanly without a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2404_11631_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "saa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(saa_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libsaa():
    return C.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("saa_eval", "saa_grad", "saa_solve", "saa_generate", "saa_ctx_create"):
        assert required in names


def test_every_declared_symbol_is_exported(libsaa):
    for name in _declared():
        assert hasattr(libsaa, name), name


def test_binding_uses_the_declared_names():
    from paper_2404_11631_gb300 import saa
    assert set(saa.EXPORTED) <= set(_declared())
    for public in ("saa_eval", "saa_grad", "saa_solve", "saa_generate"):
        assert callable(getattr(saa, public))


def test_status_strings_and_limits(libsaa):
    libsaa.saa_status_string.restype = C.c_char_p
    for code in range(7):
        assert libsaa.saa_status_string(code).startswith(b"SAA_")
    libsaa.saa_max_dim.restype = C.c_int32
    assert libsaa.saa_max_dim(0) >= 1024 and libsaa.saa_max_dim(1) >= 1024


def test_context_creation_fails_cleanly_without_a_device(libsaa):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    libsaa.saa_last_error.restype = C.c_char_p
    rc = libsaa.saa_ctx_create(C.byref(ctx), 0)
    assert rc == 1 and not ctx.value
    assert b"device" in libsaa.saa_last_error()


def _header_params():
    src = open(os.path.join(ROOT, "include", "saa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(saa_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = [p.strip() for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        out[m.group(1)] = ["ptr" if "*" in p else "int" for p in params]
    return out


def test_binding_argtypes_match_the_header():
    # argument count and pointer / integer kind of every bound entry point
    import ctypes
    from paper_2404_11631_gb300 import saa
    L = saa.lib()
    params = _header_params()
    checked = 0
    for name, kinds in params.items():
        fn = getattr(L, name)
        if fn.argtypes is None:
            continue
        assert len(fn.argtypes) == len(kinds), name
        for t, kind in zip(fn.argtypes, kinds):
            is_ptr = t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "contents") or t.__name__.startswith("LP_")
            assert is_ptr == (kind == "ptr"), (name, t, kind)
        checked += 1
    assert checked >= 12


def _c_layout(struct, fields):
    # sizeof and offsetof of a header struct, from a C compiler
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    body = "".join(f'printf("%zu ", offsetof({struct}, {f}));' for f in fields)
    src = (f'#include <stdio.h>\n#include <stddef.h>\n#include "saa.h"\n'
           f'int main(void) {{ printf("%zu ", sizeof({struct})); {body} return 0; }}\n')
    with tempfile.TemporaryDirectory() as td:
        c, exe = os.path.join(td, "l.c"), os.path.join(td, "l")
        with open(c, "w") as fh:
            fh.write(src)
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("struct,mirror", [("saa_problem", "_CProblem"), ("saa_newsvendor", "_CNewsvendor"),
                                           ("saa_logistic", "_CLogistic")])
def test_binding_structs_match_the_header_layout(struct, mirror):
    # the ctypes mirrors of the header's host structs: same size, same field offsets
    from paper_2404_11631_gb300 import saa
    cls = getattr(saa, mirror)
    names = [f[0] for f in cls._fields_]
    cnames = ["lambda" if n == "lam" else n for n in names]
    size, offs = _c_layout(struct, cnames)
    assert C.sizeof(cls) == size
    assert [getattr(cls, n).offset for n in names] == offs


def test_problem_validation_on_the_host():
    # argument checks of the binding that run before any device call
    import torch
    from paper_2404_11631_gb300 import saa
    mu = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError):
        saa.Problem(mu=mu, chol=None, N=10).c_struct()     # neither chol nor sd, and CPU tensors
    with pytest.raises(ValueError):
        saa.Problem(mu=mu, chol=torch.eye(4, dtype=torch.float64), N=10).c_struct()   # not on a GPU
