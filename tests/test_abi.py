"""The C-ABI library builds, loads without a GPU, exports every entry point
declared in include/lbm.h, and rejects bad parameters on the host."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_1510_03560_gb300 import build as B
from paper_1510_03560_gb300 import lbm as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)) - {"lbm_alloc_fn", "lbm_free_fn"})


def test_header_declares_the_api():
    names = declared_functions()
    for required in ("lbm_create", "lbm_set_geometry", "lbm_step", "lbm_get_macro",
                     "lbm_active_blocks", "lbm_destroy", "lbm_mass", "lbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(L.EXPORTS) == sorted(declared_functions())


def test_struct_layout_matches_header(lib, tmp_path):
    """The ctypes mirrors have the C compiler's size and field offsets."""
    fields = {"lbm_params": L.Params, "lbm_stats": L.Stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm.h"', "int main(void){"]
    for cname, py in fields.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        cname, fname, val = line.split()
        py = fields[cname]
        expect = C.sizeof(py) if fname == "sizeof" else getattr(py, fname).offset
        assert int(val) == expect, line


def _params(**over):
    p = L.Params()
    p.nx = p.ny = p.nz = 16
    p.ncomp = 2
    p.tau = 1.0
    p.beta = 1.16
    p.pr_a, p.pr_b, p.pr_R, p.pr_omega, p.T_over_Tc = 2 / 49, 2 / 21, 1.0, 0.344, 0.85
    p.g_self = -1.0
    for k, v in over.items():
        if k == "block":
            for a in range(3):
                p.block[a] = v[a]
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("over,frag", [
    (dict(nx=12), "multiple of the 8x8x8 block"),
    (dict(block=(4, 4, 4)), "unsupported block shape"),
    (dict(block=(8, 8, 4)), "unsupported block shape"),
    (dict(block=(32, 4, 4)), "multiple of the 32x4x4 block"),
    (dict(block=(16, 8, 4), storage=1), "need the FP32 storage form"),
    (dict(ncomp=3), "ncomp"),
    (dict(tau=0.5), "tau"),
    (dict(S=-1.0), "S must be"),
    (dict(max_blocks=-2), "max_blocks"),
    (dict(storage=3), "storage form"),
    (dict(storage=-1), "storage form"),
    (dict(streaming=2), "streaming pattern"),
    (dict(streaming=1, storage=1), "A-A streaming needs"),
    (dict(streaming=1, ncomp=1), "A-A streaming needs"),
])
def test_create_rejects_bad_parameters_without_cuda(lib, over, frag):
    h = C.c_void_p()
    rc = lib.lbm_create(C.byref(_params(**over)), C.byref(h))
    assert rc == L.EINVAL
    assert not h.value
    assert frag in lib.lbm_last_error(None).decode()


def test_null_arguments_are_rejected(lib):
    assert lib.lbm_create(None, None) == L.EINVAL
    assert lib.lbm_destroy(None) == L.OK
    assert lib.lbm_step(None, 1) == L.EINVAL
    assert lib.lbm_velocities(None) == L.EINVAL


def test_velocity_set_is_d3q19_with_opposites(lib):
    e = L.velocities()
    eo, _, _ = O.lattice()
    assert sorted(map(tuple, e)) == sorted(map(tuple, eo))
    assert tuple(e[0]) == (0, 0, 0)
