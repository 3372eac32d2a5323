"""The C-ABI library builds, loads and exports every symbol its header declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "strtr.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return")))


@pytest.fixture(scope="module")
def built_lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import __graft_entry__ as g
    g.build()
    import paper_2307_00719_gb300 as p
    return p


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("str_init", "str_init_cores", "str_update", "rstr_update", "str_update_batch",
                     "tr_reconstruct", "tr_fit_error", "str_get_core", "str_get_samples", "str_save",
                     "str_load", "str_get_stats", "str_status_string", "str_destroy",
                     "tr_masked_loss_fwd", "tr_masked_loss_bwd"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    L = ctypes.CDLL(built_lib.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib.LIB_PATH], capture_output=True, text=True)
    exported = set(line.split()[-1] for line in out.stdout.splitlines() if " T " in line)
    assert set(_declared_functions()) <= exported


def test_binding_covers_every_declared_symbol(built_lib):
    bound = {name for name, _, _ in built_lib._SIGS}
    assert set(_declared_functions()) == bound


def test_struct_layouts_match_c(built_lib, tmp_path):
    """sizeof/offsetof of the ABI structs, printed by a C program compiled with
    gcc against the header, equal the ctypes mirrors used by the binding."""
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "strtr.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(str_options), offsetof(str_options, t_capacity),
         offsetof(str_options, init_tol), offsetof(str_options, m), offsetof(str_options, stream_id),
         offsetof(str_options, graphs));
  printf("%zu %zu %zu\n", sizeof(str_tensor), offsetof(str_tensor, dims), offsetof(str_tensor, on_host));
  printf("%zu %zu %zu\n", sizeof(str_stats), offsetof(str_stats, min_pivot_ratio), offsetof(str_stats, class_ms));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [list(map(int, line.split())) for line in subprocess.run([str(exe)], capture_output=True,
                                                                      text=True).stdout.splitlines()]
    O, T, S = built_lib.StrOptions, built_lib.StrTensor, built_lib.StrStats
    assert vals[0] == [ctypes.sizeof(O), O.t_capacity.offset, O.init_tol.offset, O.m.offset,
                       O.stream_id.offset, O.graphs.offset]
    assert vals[1] == [ctypes.sizeof(T), T.dims.offset, T.on_host.offset]
    assert vals[2] == [ctypes.sizeof(S), S.min_pivot_ratio.offset, S.class_ms.offset]


def test_host_only_calls(built_lib):
    o = built_lib.default_options()
    assert o.compute == built_lib.STR_F64 and o.sweeps == 1 and o.rescale == 1
    assert o.sketch == built_lib.SKETCH_NONE and o.init_max_it == 100 and abs(o.init_tol - 1e-8) < 1e-20
    assert built_lib.lib().str_status_string(4) == b"normal-equation matrix not positive definite"
    assert built_lib.lib().str_default_options(None) == 1
