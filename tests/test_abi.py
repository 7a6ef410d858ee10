"""The C ABI library loads without a GPU, exports every function that
include/mpmc.h declares, and the binding's struct layouts match the header
(sizes and offsets printed by a gcc-compiled probe of the header)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "mpmc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2504_14063_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def declared_functions():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mpmc_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mpmc_init_state", "mpmc_rhs", "mpmc_rk_step", "mpmc_step_n", "mpmc_rhs_adjoint"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_header(tmp_path):
    from paper_2504_14063_gb300 import binding as b
    probe = tmp_path / "probe.c"
    probe.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HDR}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu\\n", sizeof(mpmc_grid), sizeof(mpmc_eos), sizeof(mpmc_model),
         sizeof(mpmc_stage), sizeof(mpmc_stats));
  printf("%zu %zu %zu %zu %zu\\n", offsetof(mpmc_grid, inflow), offsetof(mpmc_eos, Sc),
         offsetof(mpmc_model, precision), offsetof(mpmc_model, lambda_liquid), offsetof(mpmc_stage, Gamma));
  return 0;
}}
""")
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-o", str(exe), str(probe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    sizes = [int(x) for x in out[:5]]
    offs = [int(x) for x in out[5:]]
    assert sizes == [ctypes.sizeof(t) for t in (b.Grid, b.Eos, b.ModelC, b.StageC, b.StatsC)]
    assert offs == [b.Grid.inflow.offset, b.Eos.Sc.offset, b.ModelC.precision.offset,
                    b.ModelC.lambda_liquid.offset, b.StageC.Gamma.offset]


def test_flag_and_status_constants_match_header():
    """The binding's tape-bit, status, precision and interpolation constants
    are the header's #define values (MPMC_F_*, MPMC_*)."""
    from paper_2504_14063_gb300 import binding as b
    txt = open(HDR).read()
    defs = {}
    for name, val in re.findall(r"#define\s+MPMC_([A-Z0-9_]+)\s+\(?([0-9]+u?(?:\s*<<\s*[0-9]+)?)\)?", txt):
        defs[name] = eval(val.replace("u", ""))
    flags = {k[2:]: v for k, v in defs.items() if k.startswith("F_")}
    assert flags["DIFF_DROPPED"] == 256
    for k, v in flags.items():
        assert getattr(b, "F_" + k) == v, k
    for k in ("OK", "INVALID_ARG", "CUDA_ERROR", "INADMISSIBLE", "EOS_NO_CONVERGE", "OUT_OF_MEMORY", "FP64", "MIXED"):
        assert getattr(b, k) == defs[k], k
    assert [s for s, _ in b.StatsC._fields_][-1] == "diff_dropped"


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    """Host-side validation happens before any CUDA call."""
    from paper_2504_14063_gb300 import binding as b
    from paper_2504_14063_gb300 import workloads as W
    p = W.interface_advection_1d(n=16)
    g, e, m = b.structs_from_problem(p)
    h = ctypes.c_void_p()
    e.n_species = 9
    assert b.lib.mpmc_create(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), None, ctypes.byref(h)) == b.INVALID_ARG
    e.n_species = 2
    g.n[0] = 2
    assert b.lib.mpmc_create(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), None, ctypes.byref(h)) == b.INVALID_ARG
    assert h.value is None
    # 2^31 - 1 cells or faces: beyond the kernels' 32-bit indexing
    g.n[0] = 2 ** 31 - 1
    assert b.lib.mpmc_create(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), None, ctypes.byref(h)) == b.INVALID_ARG
    g.n[0] = 2 ** 31 - 2     # 2^31 - 2 cells + the inflow slot, 2^31 - 1 faces
    assert b.lib.mpmc_create(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), None, ctypes.byref(h)) == b.INVALID_ARG
    assert h.value is None
    # an unknown interpolation
    g.n[0] = 16
    m.recon = 4
    assert b.lib.mpmc_create(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), None, ctypes.byref(h)) == b.INVALID_ARG
    # viscosity with a non-positive Prandtl number
    m.recon, m.viscous, m.precision, m.prandtl = 0, 1, b.FP64, 0.0
    assert b.lib.mpmc_create(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), None, ctypes.byref(h)) == b.INVALID_ARG
    assert h.value is None


def test_null_context_queries_without_a_gpu(lib):
    """The size queries answer 0 for a null context; the recording and
    reverse steps reject it before any CUDA call."""
    from paper_2504_14063_gb300 import binding as b
    assert b.lib.mpmc_cache_doubles(None) == 0
    assert b.lib.mpmc_ncells(None) == 0
    assert b.lib.mpmc_rk_step_record(None, None, 0.0, None, None, None) == b.INVALID_ARG
    assert b.lib.mpmc_rk_step_adjoint(None, None, None, None, 0.0, None, None, None) == b.INVALID_ARG


def test_characteristic_boundaries_are_validated_without_a_gpu(lib):
    """MPMC_BC_CHAR (the header's value) is accepted along x only; the
    allocation-free entry refuses it before any CUDA call."""
    from paper_2504_14063_gb300 import binding as b
    from paper_2504_14063_gb300 import workloads as W
    txt = open(HDR).read()
    assert re.search(r"#define\s+MPMC_BC_CHAR\s+4\b", txt) and W.BC_CHAR == 4
    p = W.acoustic_tube(n=16, ny=4)
    g, e, m = b.structs_from_problem(p)
    h = ctypes.c_void_p()
    g.bc_lo[1] = g.bc_hi[1] = W.BC_CHAR
    assert b.lib.mpmc_create(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), None, ctypes.byref(h)) == b.INVALID_ARG
    assert h.value is None
    g.bc_lo[1] = g.bc_hi[1] = W.BC_PERIODIC
    g.bc_hi[0] = 5
    assert b.lib.mpmc_create(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), None, ctypes.byref(h)) == b.INVALID_ARG
    g.bc_hi[0] = W.BC_CHAR
    f = b.lib.mpmc_rhs_noalloc
    f.restype = ctypes.c_int
    need = ctypes.c_size_t(0)
    assert f(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), None, None, None, None, ctypes.byref(need)) == \
        b.INVALID_ARG
