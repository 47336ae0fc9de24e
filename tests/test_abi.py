"""The C-ABI library loads and exports every symbol include/axpic.h declares,
and the ctypes structures match the C layout (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2604_24627_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "axpic.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(axpic_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2604_24627_gb300 import build
        build.build()
    return _lib.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 17
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (axpic_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)
        assert n in _lib.EXPORTS, "binding lacks " + n


def test_host_only_calls(lib):
    assert _lib.axpic_version().startswith("axpic")
    p = _lib.default_params()
    assert p.tally_nbins == 160 and abs(p.brems_gamma_shape - 1.70) < 1e-15 and p.brems_ee == 1
    assert lib.axpic_last_error(None) == b"no context"
    # NULL arguments are rejected before any CUDA call
    assert lib.axpic_init_plasma(None, None, None, None) == _lib.AXPIC_E_INVALID
    assert lib.axpic_step(None, 0, 7) == _lib.AXPIC_E_INVALID
    assert lib.axpic_sync(None) == _lib.AXPIC_E_INVALID


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "axpic.h"
#define P(T, f) printf(#T "." #f " %zu\\n", offsetof(T, f));
int main(void) {
  printf("axpic_species %zu\\n", sizeof(axpic_species));
  printf("axpic_plasma_desc %zu\\n", sizeof(axpic_plasma_desc));
  printf("axpic_params %zu\\n", sizeof(axpic_params));
  P(axpic_plasma_desc, electrons) P(axpic_plasma_desc, axions) P(axpic_plasma_desc, cell_volume_cm3)
  P(axpic_params, kappa_fixed_keV) P(axpic_params, seed) P(axpic_params, tally_Emax_keV)
  P(axpic_params, threads_per_block) P(axpic_params, decide_chunk) P(axpic_params, T_mode)
  P(axpic_params, rate_model) P(axpic_params, sr_table_nne) P(axpic_params, step_branches)
  P(axpic_params, brems_gamma_shape)
  P(axpic_species, wp) P(axpic_species, xyz) P(axpic_species, count)
  P(axpic_species, capacity)
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True,
                                                              text=True).stdout.strip().splitlines())
    assert int(out["axpic_species"]) == ctypes.sizeof(_lib.Species)
    assert int(out["axpic_plasma_desc"]) == ctypes.sizeof(_lib.PlasmaDesc)
    assert int(out["axpic_params"]) == ctypes.sizeof(_lib.Params)
    for key, val in out.items():
        if "." in key:
            T, f = key.split(".")
            cls = {"axpic_plasma_desc": _lib.PlasmaDesc, "axpic_params": _lib.Params,
                   "axpic_species": _lib.Species}[T]
            assert getattr(cls, f).offset == int(val), key
