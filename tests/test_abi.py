"""Host-side checks of the C-ABI library: it loads, exports every entry point include/gsph.h declares,
its structs match the header's layout, and invalid configurations are rejected before any device
work (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2310_03596_gb300 import build as gbuild
from paper_2310_03596_gb300 import gsph, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gsph.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "gsph.h")).read()
    return sorted(set(re.findall(r"\b(gsph_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 17
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(gsph.EXPORTS) == names


def _c_layout(tmp_path, struct, fields):
    src = tmp_path / "probe.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gsph.h"', 'int main(void) {',
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ['  return 0;', '}']
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    return [int(v) for v in subprocess.check_output([str(exe)]).split()]


@pytest.mark.parametrize("py,cname", [(gsph.Material, "gsph_material"), (gsph.Wall, "gsph_wall"),
                                      (gsph.Config, "gsph_config"), (gsph.ExchangeStats, "gsph_exchange_stats"),
                                      (gsph.Timings, "gsph_timings"), (gsph.AdjConfig, "gsph_adj_cfg")])
def test_struct_layout_matches_header(tmp_path, py, cname):
    fields = [f for f, _ in py._fields_]
    got = _c_layout(tmp_path, cname, fields)
    assert got[0] == C.sizeof(py)
    assert got[1:] == [getattr(py, f).offset for f in fields]


def test_status_strings(lib):
    for code, text in gsph.STATUS.items():
        assert lib.gsph_status_str(code).decode() == text


def _cfg(**kw):
    c = gsph.config_from_scene(scenes.cube_impact(n_side=4))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("bad", [dict(h=0.0), dict(cfl=-1.0), dict(K=0), dict(K=17), dict(n_materials=0),
                                 dict(n_materials=5), dict(n_walls=7), dict(precision=3), dict(swap_period=-1),
                                 dict(alpha=1.5), dict(overlap=2), dict(integrator=2),
                                 dict(integrator=1, overlap=1), dict(reconstruction=2),
                                 dict(reconstruction=1, integrator=1), dict(reconstruction=1, overlap=1),
                                 dict(variable_h=2), dict(variable_h=1, overlap=1)])
def test_invalid_config_rejected_on_host(lib, bad):
    h = C.c_void_p()
    assert lib.gsph_create(C.byref(_cfg(**bad)), C.byref(h)) == gsph.INVALID_ARG
    assert not h.value


def test_invalid_grid_rejected_on_host(lib):
    c = _cfg()
    c.grid_dims[0] = 1 << 14
    c.grid_dims[1] = 1 << 14
    h = C.c_void_p()
    assert lib.gsph_create(C.byref(c), C.byref(h)) == gsph.INVALID_ARG
    c = _cfg()
    c.walls[0].axis = 3
    assert lib.gsph_create(C.byref(c), C.byref(h)) == gsph.INVALID_ARG


def test_null_arguments_rejected(lib):
    assert lib.gsph_create(None, None) == gsph.INVALID_ARG
    assert lib.gsph_step(None, 1, None) == gsph.INVALID_ARG
    assert lib.gsph_sync(None, None) == gsph.INVALID_ARG
    assert lib.gsph_radix_sort_pairs(None, None, 10, 8, None, 0, None) == gsph.INVALID_ARG
    assert lib.gsph_radix_sort_pairs(None, None, 0, 8, None, 0, None) == gsph.OK
    assert lib.gsph_radix_sort_pairs(None, None, 10, 33, None, 0, None) == gsph.INVALID_ARG
    assert lib.gsph_set_timing(None, 1) == gsph.INVALID_ARG
    assert lib.gsph_set_timing_ex(None, 1, 1) == gsph.INVALID_ARG
    assert lib.gsph_get_timings(None, None) == gsph.INVALID_ARG


def test_sort_workspace_grows_with_n(lib):
    a = lib.gsph_radix_sort_workspace(1000, 20)
    b = lib.gsph_radix_sort_workspace(1 << 20, 20)
    assert b >= 8 * (1 << 20) > a > 0
