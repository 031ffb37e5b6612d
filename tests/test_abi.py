"""The C-ABI library builds, loads, and exports every entry point that
include/ibm_schur.h declares; the ctypes structures match the C layout.  No
compute call (no GPU needed)."""
import ctypes as C
import re
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "ibm_schur.h"


def header_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ibm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(built_lib):
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(built_lib, n), n


def test_binding_declares_every_symbol():
    from paper_2501_15314_gb300 import _lib
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == header_functions()


def test_struct_layout_matches_c(tmp_path):
    from paper_2501_15314_gb300 import _lib
    src = tmp_path / "sz.c"
    src.write_text('#include "ibm_schur.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(ibm_grid_desc),'
                   ' sizeof(ibm_solve_opts), sizeof(ibm_solve_stats),'
                   ' offsetof(ibm_solve_stats, helm_iters), offsetof(ibm_solve_opts, helm_rtol));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out == [C.sizeof(_lib.ibm_grid_desc), C.sizeof(_lib.ibm_solve_opts),
                   C.sizeof(_lib.ibm_solve_stats), _lib.ibm_solve_stats.helm_iters.offset,
                   _lib.ibm_solve_opts.helm_rtol.offset]


def test_default_opts_and_null_arguments(built_lib):
    from paper_2501_15314_gb300 import _lib
    o = _lib.default_opts()
    assert o.precond_prec == _lib.IBM_PREC_FP32 and o.rtol == 1e-8 and o.restart == 40
    # argument validation happens before any CUDA call
    out = C.c_void_p()
    assert built_lib.ibm_create(None, None, C.byref(out)) == _lib.IBM_ERR_ARG
    g = _lib.ibm_grid_desc(2, 8, 8, 0.1, 100.0, 0.01)
    assert built_lib.ibm_create(C.byref(g), None, C.byref(out)) == _lib.IBM_ERR_ARG
    assert built_lib.ibm_set_markers(None, 0, None) == _lib.IBM_ERR_ARG
    assert built_lib.ibm_last_error(None) == b"null context"
    built_lib.ibm_destroy(None)


def test_product_path_does_not_import_oracle():
    pkg = ROOT / "paper_2501_15314_gb300"
    for f in pkg.glob("*.py"):
        text = f.read_text()
        assert "import oracle" not in text and "from oracle" not in text, f
    for f in (pkg / "csrc").glob("*"):
        assert "oracle" not in f.read_text(), f
    bench = ROOT / "bench.py"
    if bench.exists():
        # only the CPU-baseline / reference leg (inside a function) uses it
        for line in bench.read_text().splitlines():
            if "import oracle" in line or "from oracle" in line:
                assert line.startswith("    "), line


def test_missing_library_fails_loudly(tmp_path):
    # with the shared library absent, the first call into the package raises;
    # nothing falls back to a CPU implementation
    code = ("import sys; from pathlib import Path\n"
            f"sys.path.insert(0, {str(ROOT)!r})\n"
            "from paper_2501_15314_gb300 import _lib\n"
            f"_lib.LIB_PATH = Path({str(tmp_path / 'libibmschur.so')!r})\n"
            "from paper_2501_15314_gb300.api import IBMSolver\n"
            "try:\n"
            "    IBMSolver(16)\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(3)\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "is not built" in r.stdout


@pytest.mark.parametrize("compiler,std,ext", [("gcc", "-std=c99", "c"), ("g++", "-std=c++11", "cpp")])
def test_header_is_strict_c_and_cpp(tmp_path, compiler, std, ext):
    # the boundary is plain C: the header compiles warning-free as ISO C99 and C++11
    src = tmp_path / f"h.{ext}"
    src.write_text('#include "ibm_schur.h"\nint main(void) { ibm_solve_opts o; '
                   'ibm_default_opts(&o); return o.restart > 0 ? 0 : 1; }\n')
    subprocess.run([compiler, std, "-pedantic", "-Wall", "-Wextra", "-Werror",
                    f"-I{ROOT / 'include'}", "-c", str(src), "-o", str(tmp_path / "h.o")],
                   check=True)


def test_noalloc_argument_checks_need_no_gpu(built_lib):
    # the checks that precede any CUDA call: body count, cell width, missing
    # outputs; zero markers give zero sums without touching a device
    from paper_2501_15314_gb300 import _lib
    fn = built_lib.ibm_body_forces_noalloc
    centers = (C.c_double * (3 * 1025))()
    out = (C.c_double * (6 * 1025))(*([7.0] * (6 * 1025)))
    assert fn(None, None, None, 0, 0, centers, 0.1, None, out) == _lib.IBM_ERR_ARG
    assert fn(None, None, None, 0, 1025, centers, 0.1, None, out) == _lib.IBM_ERR_ARG
    assert fn(None, None, None, 0, 2, centers, 0.0, None, out) == _lib.IBM_ERR_ARG
    assert fn(None, None, None, 0, 2, None, 0.1, None, out) == _lib.IBM_ERR_ARG
    assert fn(None, None, None, 0, 2, centers, 0.1, None, None) == _lib.IBM_ERR_ARG
    assert fn(None, None, None, -1, 2, centers, 0.1, None, out) == _lib.IBM_ERR_ARG
    assert fn(None, None, None, 5, 2, centers, 0.1, None, out) == _lib.IBM_ERR_ARG  # no F, X
    assert fn(None, None, None, 0, 3, centers, 0.1, None, out) == _lib.IBM_OK
    assert list(out[:18]) == [0.0] * 18 and out[18] == 7.0


def test_noalloc_refuses_misaligned_and_host_pointers_before_any_launch(built_lib):
    # F, X must be 8-byte aligned, body_id 4-byte aligned, and all three
    # device memory of the current device; otherwise IBM_ERR_ARG comes back
    # before anything is launched (here without a GPU: the pointer checks
    # themselves need no device)
    from paper_2501_15314_gb300 import _lib
    fn = built_lib.ibm_body_forces_noalloc
    centers = (C.c_double * 3)()
    out = (C.c_double * 6)()
    host = (C.c_double * 64)()
    a = C.addressof(host)
    assert a % 8 == 0
    launches = built_lib.ibm_kernel_launches()
    for F, X, bid in ((a + 4, a, a), (a, a + 2, a), (a, a, a + 2), (a, a, a)):
        assert fn(F, X, bid, 5, 1, centers, 0.1, None, out) == _lib.IBM_ERR_ARG
    assert built_lib.ibm_kernel_launches() == launches


def test_every_context_call_rejects_a_null_context(built_lib):
    # every entry point taking an ibm_ctx returns IBM_ERR_ARG for NULL before
    # any CUDA call (all other arguments zero or NULL)
    from paper_2501_15314_gb300 import _lib
    no_ctx = {"ibm_create", "ibm_destroy", "ibm_last_error", "ibm_num_cells", "ibm_num_faces",
              "ibm_default_opts", "ibm_default_fsi_opts", "ibm_kernel_launches",
              "ibm_body_forces_noalloc"}
    checked = 0
    for name, _, args in _lib.SIGNATURES:
        if name in no_ctx:
            continue
        vals = [0 if a in (C.c_int, C.c_int32, C.c_int64) else 0.0 if a is C.c_double else None
                for a in args]
        assert getattr(built_lib, name)(*vals) == _lib.IBM_ERR_ARG, name
        checked += 1
    assert checked >= 19
    assert built_lib.ibm_num_cells(None) == 0 and built_lib.ibm_num_faces(None) == 0


def test_binding_rejects_host_tensors():
    # the binding passes device pointers only: a CPU tensor (or a wrong dtype,
    # a strided view, a wrong size) is refused before any library call, so no
    # call can silently run on host memory
    import torch
    from paper_2501_15314_gb300.api import RigidSpheres, _ptr
    with pytest.raises(ValueError, match="CUDA"):
        _ptr(torch.zeros(8, dtype=torch.float64), name="u")
    with pytest.raises(TypeError):
        _ptr([0.0] * 8, name="u")
    # host state of the two-way spheres is a plain ctypes array
    rs = RigidSpheres([0.1, 0.2], 2.0, [[0.3, 0.3, 0.3], [0.7, 0.6, 0.5]],
                      velocities=[[1, 2, 3], [4, 5, 6]])
    assert rs.n == 2 and rs.get("radius").tolist() == [0.1, 0.2]
    assert rs.get("us").tolist() == [[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]]
    assert rs.get("rot").tolist() == [[1, 0, 0, 0, 1, 0, 0, 0, 1]] * 2
