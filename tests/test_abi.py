"""Host-side checks of the C-ABI library (no GPU): it builds, loads, exports
every entry point include/snk.h declares, and rejects bad input before any
device work."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "snk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(snk_[a-zA-Z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("snk_create", "snk_set_density", "snk_build_K", "snk_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2303_14280_gb300 as snk
    L = snk.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(snk.SYMBOLS) == _declared()


def test_options_defaults():
    import paper_2303_14280_gb300 as snk
    o = snk.options()
    assert o.batch_max == 4096 and o.eps_E == 1e-12 and o.screen == 1 and o.precision == 0
    # the plain FP64 form unless a form is asked for
    assert o.gemm == 0 and o.ds_integrals == 0 and o.graph == 0 and o.distance_bound == 1
    assert o.tc_slices_hi == 5 and o.tc_slices_lo == 4
    assert o.learned_skip == -11.0 and o.learned_fp32 == -99.0 and o.fp32_bound == 1e-6
    assert snk.options(gemm="split").gemm == 2 and snk.options(precision="mixed").precision == 1
    with pytest.raises(ValueError):
        snk.options(gemmm="split")            # a misspelled option is an error, not a no-op


def test_generated_os_code_is_current():
    gen = os.path.join(ROOT, "paper_2303_14280_gb300", "csrc", "gen_os.py")
    out = subprocess.run([sys.executable, gen], capture_output=True, text=True, check=True).stdout
    cur = open(os.path.join(ROOT, "paper_2303_14280_gb300", "csrc", "os_generated.cuh")).read()
    assert out == cur


def test_create_rejects_bad_input_on_the_host():
    """Validation happens before any CUDA call, so it is testable without a GPU."""
    import synth
    from paper_2303_14280_gb300 import Engine, SnkError
    p = synth.chain4()
    b = p.basis
    bad = synth.Basis(l=np.where(np.arange(b.n_shells) == 3, 3, b.l).astype(np.int32), nprim=b.nprim,
                      atom=b.atom, center=b.center, exps=b.exps, coefs=b.coefs)
    with pytest.raises(SnkError) as e:
        Engine(bad, p.grid)
    assert e.value.status == -2
    nanb = synth.Basis(l=b.l, nprim=b.nprim, atom=b.atom, center=b.center,
                       exps=np.where(np.arange(b.exps.shape[0]) == 0, np.nan, b.exps), coefs=b.coefs)
    with pytest.raises(SnkError) as e:
        Engine(nanb, p.grid)
    assert e.value.status == -2
    negw = synth.Grid(xyz=p.grid.xyz, w=p.grid.w, atom=np.full_like(p.grid.atom, -1))
    with pytest.raises(SnkError) as e:
        Engine(p.basis, negw)
    assert e.value.status == -1
    with pytest.raises(SnkError) as e:
        Engine(p.basis, p.grid, batch_max=0)
    assert e.value.status == -1


def test_null_handle_calls_fail_cleanly():
    import paper_2303_14280_gb300 as snk
    L = snk.lib()
    assert L.snk_set_density(None, None) == -1
    assert L.snk_build_K(None, None) == -1
    assert L.snk_last_error(None) == b"NULL handle"
    L.snk_destroy(None)


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a C program built with gcc."""
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "snk.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("cname,pyname", [("snk_options", "SnkOptions"), ("snk_stats", "SnkStats"),
                                          ("snk_basis", "SnkBasis"), ("snk_grid", "SnkGrid")])
def test_binding_structs_match_the_header_layout(cname, pyname, tmp_path):
    """The ctypes mirrors of the header structs have the C compiler's size and
    every field at the C compiler's offset."""
    import paper_2303_14280_gb300 as snk
    cls = getattr(snk, pyname)
    fields = [f[0] for f in cls._fields_]
    size, offs = _c_layout(cname, fields, tmp_path)
    assert ctypes.sizeof(cls) == size
    for f, off in zip(fields, offs):
        assert getattr(cls, f).offset == off, f
