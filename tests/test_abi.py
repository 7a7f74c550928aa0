"""CPU checks of the C-ABI boundary: the library loads, exports every symbol
include/rt_m1.h declares, rejects bad arguments before touching the GPU, and
its host-side group table agrees with the oracle's independent quadrature."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import binding as B
from paper_1508_07888_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^RT_API\s+[^(]*?\b(\w+)\s*\(", txt, flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    L = B.lib()
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert set(names) >= set(B.EXPORTS)


@pytest.mark.parametrize("edges,T", [(I.GROUPS_1, 1e5), (I.GROUPS_3, 5e4), (I.GROUPS_2, 5e4)])
def test_group_table_matches_oracle(edges, T):
    a = B.rt_group_table(edges, T)
    b = O.group_table(edges, T)
    for k in a:
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12)
        assert np.array_equal(I.f32(a[k]), I.f32(b[k])), k


def test_timestep_matches_paper_reading():
    t = {"sigN": [1.0], "sigE": [1.0], "Eavg": [1.0], "frac": [1.0]}
    p = B.make_params(1, t, 3e9, cfl=0.9)
    assert B.rt_timestep(p, 6e20) == pytest.approx(0.9 * 6e20 / (3 * 3e9), rel=1e-15, abs=0)
    p.cfl = 0.0
    assert B.rt_timestep(p, 6e20) < 0


def _bad(**kw):
    t = {"sigN": [1e-18], "sigE": [1e-18], "Eavg": [3e-11], "frac": [1.0]}
    base = dict(cfl=0.9)
    base.update(kw)
    G = base.pop("G", 1)
    p = B.make_params(1, t, base.pop("c_red", 3e9), **base)
    p.ngroups = G
    h = C.c_void_p()
    box = B.rt_box()
    return B.lib().rt_create(C.byref(h), C.byref(p), C.byref(box), 1, None)


@pytest.mark.parametrize("kw", [dict(G=0), dict(G=5), dict(cfl=1.5), dict(cfl=0.0),
                                dict(c_red=-1.0), dict(nsub=-1), dict(precision=7),
                                dict(bc=(0, 1, 0, 0, 0, 0)), dict(bc=(3, 3, 0, 0, 0, 0)),
                                dict(rates_const=True, isothermal=False),
                                dict(max_halvings=-1), dict(chem_tune=-1), dict(chem_tune=8)])
def test_create_rejects_bad_params(kw):
    assert _bad(**kw) == B.RT_ERR_ARG
    assert B.rt_last_error(None)


def test_create_rejects_bad_boxes_and_null_handle():
    t = {"sigN": [1e-18], "sigE": [1e-18], "Eavg": [3e-11], "frac": [1.0]}
    p = B.make_params(1, t, 3e9)
    h = C.c_void_p()
    box = B.rt_box()
    box.nx = box.ny = box.nz = 0
    assert B.lib().rt_create(C.byref(h), C.byref(p), C.byref(box), 1, None) == B.RT_ERR_ARG
    assert B.lib().rt_create(None, C.byref(p), C.byref(box), 1, None) == B.RT_ERR_ARG
    assert B.lib().rt_create(C.byref(h), C.byref(p), None, 0, None) == B.RT_ERR_ARG
    assert B.lib().rt_step(None, 1, None) == B.RT_ERR_STATE
    assert B.lib().rt_query(None, None) == B.RT_ERR_STATE
    B.lib().rt_destroy(None)


def test_group_table_rejects_bad_edges():
    with pytest.raises(B.RTError):
        B.rt_group_table([10.0, 20.0], 5e4)
    with pytest.raises(B.RTError):
        B.rt_group_table([13.6, 13.0], 5e4)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of rt_params, rt_box and rt_stats have the sizes and
    field offsets a C compiler gives the declarations in include/rt_m1.h."""
    import ctypes as C
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    structs = {"rt_params": B.rt_params, "rt_box": B.rt_box, "rt_stats": B.rt_stats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "rt_m1.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, v = ln.split()
            got[(a, b)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


@pytest.mark.parametrize("side", [256, 1 << 20, (1 << 31) - 1])
def test_static_transport_size_check_cannot_overflow(side):
    """rt_transport_static checks the box against its fixed scratch before any
    CUDA call, one factor at a time: a box whose byte count overflows 64 bits
    (2^20 or 2^31 - 1 cells per axis) is rejected, not wrapped under the limit.
    U is a dummy aligned address that is never dereferenced."""
    f = B.lib().rt_transport_static
    f.restype = C.c_int
    f.argtypes = [C.POINTER(B.rt_params), C.POINTER(B.rt_box), C.c_int, C.c_void_p]
    t = {"sigN": [0.0], "sigE": [0.0], "Eavg": [0.0], "frac": [1.0]}
    p = B.make_params(1, t, 3e9, isothermal=True, rates_const=True)
    box = B.rt_box()
    box.nx = box.ny = box.nz = side
    box.dx, box.nunit = 3e20, 1.0
    box.U = 1 << 20
    assert f(C.byref(p), C.byref(box), 1, None) == B.RT_ERR_TOO_LARGE
    assert "does not fit" in B.rt_last_error(None)
    box.nx = box.ny = box.nz = 0
    assert f(C.byref(p), C.byref(box), 1, None) == B.RT_ERR_ARG
    assert "positive" in B.rt_last_error(None)
