"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/laplace.h declares; host-only calls (defaults, error strings, size queries and their
refusals) work on the CPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "laplace.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lap_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_02427_gb300 import build
    try:
        path = build.build()
    except RuntimeError as exc:
        pytest.skip(f"no CUDA toolkit to build the library: {exc}")
    return C.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("lap_create", "lap_destroy", "lap_solve", "lap_residual", "lap_workspace_bytes",
                 "lap_strerror", "lap_smooth", "lap_restrict", "lap_prolong_add",
                 "lap_coarse_solve", "lap_line_sweep", "lap_jacobi_sweep"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    from paper_2208_02427_gb300 import binding
    p = binding.Params()
    lib.lap_default_params(C.byref(p))
    assert p.method == binding.METHODS["sor"] and p.tol == 1e-10 and p.nu1 == 2 and p.nu2 == 2
    assert p.coarsest_min == 5 and p.smoother_w == 1.0 and p.check_every == 1
    lib.lap_strerror.restype = C.c_char_p
    assert lib.lap_strerror(0) == b"ok"
    assert b"invalid" in lib.lap_strerror(-1)


def test_struct_layouts_match_header(tmp_path):
    """Every field offset and struct size of the ctypes mirrors equals the C compiler's."""
    import shutil
    import subprocess
    from paper_2208_02427_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"lap_grid": binding.Grid, "lap_params": binding.Params, "lap_result": binding.Result}
    lines = []
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "laplace.h"\nint main(void){'
                    + "".join(lines) + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    seen = {}
    for row in subprocess.check_output([str(exe)], text=True).split("\n"):
        if row:
            cname, key, val = row.split()
            seen[(cname, key)] = int(val)
    for cname, py in structs.items():
        assert seen[(cname, "size")] == C.sizeof(py)
        for fname, _ in py._fields_:
            assert seen[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_grid_limits_match_header(tmp_path):
    """The binding's grid limits are the header's macros."""
    import shutil
    import subprocess
    from paper_2208_02427_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    prog = tmp_path / "limits.c"
    prog.write_text('#include <stdio.h>\n#include "laplace.h"\nint main(void){'
                    'printf("%ld %ld\\n", (long)LAP_GRID_MAX_M, (long)LAP_GRID_MAX_N); return 0;}\n')
    exe = tmp_path / "limits"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    m, n = (int(v) for v in subprocess.check_output([str(exe)], text=True).split())
    assert (m, n) == (binding.GRID_MAX_M, binding.GRID_MAX_N)


def test_size_query_refuses_what_the_solve_refuses(lib):
    """lap_workspace_bytes is host arithmetic: it gives lap_solve's refusals from the shape
    alone, with nothing allocated. Refused (LAP_EUNSUPPORTED): one column more than
    LAP_GRID_MAX_M, one row more than LAP_GRID_MAX_N, the diagonal summation order past its
    32-bit walk numbering (2^28 x 97: 16 strips of 2^27 + 2 walks, 2^31 + 32 in all; 2^28 x 91
    has 15 strips and is taken, and the printed order takes both), the diagonal order with
    dx != dy, ADI lines past 16383 unknowns, lexicographic sweeps past 28672 points and a
    coarsest multigrid level past 1024 unknowns."""
    from paper_2208_02427_gb300 import binding as b
    M, N = b.GRID_MAX_M, b.GRID_MAX_N

    def query(shape, dx=1.0, dy=1.0, **kw):
        g = b.Grid(shape[0], shape[1], dx, dy, shape[0])
        out = C.c_size_t(0)
        return lib.lap_workspace_bytes(C.byref(g), C.byref(b.params(**kw)), C.byref(out))

    EUNSUPPORTED = -4
    assert query((M, 5), method="jacobi") == 0
    assert query((5, N), method="jacobi") == 0
    assert query((M + 1, 5), method="jacobi") == EUNSUPPORTED
    assert query((5, N + 1), method="jacobi") == EUNSUPPORTED
    assert query((M, 91), method="sor", w=1.5, sum_order="diagonal") == 0
    assert query((M, 97), method="sor", w=1.5, sum_order="diagonal") == EUNSUPPORTED
    assert query((M, 97), method="sor", w=1.5) == 0
    assert query((65, 65), 1.0, 0.5, method="sor", w=1.5, sum_order="diagonal") == EUNSUPPORTED
    assert query((16385, 5), method="adi", w=1.3) == 0
    assert query((16386, 5), method="adi", w=1.3) == EUNSUPPORTED
    assert query((224, 128), method="sor_lex", w=1.5) == 0
    assert query((225, 128), method="sor_lex", w=1.5) == EUNSUPPORTED
    assert query((34, 34), method="mg", max_levels=1) == 0
    assert query((35, 34), method="mg", max_levels=1) == EUNSUPPORTED
