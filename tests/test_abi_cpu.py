"""CPU-only checks of the C ABI: the library loads, exports every function
include/cpaa.h declares, and its host-side stopping rule agrees with the
oracle's.  No GPU call is made."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2112_01743_gb300 import build
    build.build()
    import paper_2112_01743_gb300 as pkg
    return pkg


def _declared():
    src = open(os.path.join(ROOT, "include", "cpaa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cpaa_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_names(L):
    assert _declared() == sorted(L.EXPORTED_SYMBOLS)


def test_header_constants_match_the_binding(L):
    """The flag and limit macros of include/cpaa.h have the binding's values."""
    src = open(os.path.join(ROOT, "include", "cpaa.h")).read()
    names = ("CPAA_GRAPH_DEVICE_INPUT", "CPAA_GRAPH_VALIDATE", "CPAA_GRAPH_TRUSTED", "CPAA_DEVICE_IO",
             "CPAA_TIME_ROUNDS", "CPAA_SERVER_FUSED", "CPAA_NOALLOC_MAX_N", "CPAA_SERVER_MAX_SEEDS",
             "CPAA_GRAPH_AUTOTUNE", "CPAA_SPARSE_FRONTIER", "CPAA_INTERVAL", "CPAA_CERTIFY_INTERVAL")
    for name in names:
        m = re.search(r"#define\s+%s\s+(\d+)u?\b" % name, src)
        assert m, name
        assert int(m.group(1)) == getattr(L, name), name


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings(L):
    assert L.cpaa_status_string(L.CPAA_OK) == "CPAA_OK"
    assert L.cpaa_status_string(L.CPAA_ENOTCONV) == "CPAA_ENOTCONV"
    assert L.cpaa_status_string(99) == "CPAA_UNKNOWN"


def test_options_defaults(L):
    o = L.cpaa_options_init()
    assert (o.precision, o.normalize, o.fixed_rounds, o.max_rounds, o.flags) == (0, 0, 0, 2000, 0)


@pytest.mark.parametrize("c", [0.5, 0.85, 0.95, 0.99])
@pytest.mark.parametrize("kappa", [1.0, 1.44, 74.0, 1.6e4])
@pytest.mark.parametrize("norm", [0, 1])
def test_stopping_rule_matches_oracle(L, c, kappa, norm):
    from oracle import oracle as O
    for tol in (1e-3, 1e-6, 1e-10, 1e-12):
        assert L.cpaa_rounds_needed(c, tol, kappa, norm) == O.rounds_needed(c, tol, kappa, norm)
        for M in (1, 7, 30):
            a, b = L.cpaa_l1_bound(c, M, kappa, norm), O.l1_bound(c, M, kappa, norm)
            assert abs(a - b) <= 1e-14 * abs(b)


@pytest.mark.parametrize("c", [0.5, 0.85, 0.95])
@pytest.mark.parametrize("lo", [-1.0, -0.9, -0.6, 0.0, 0.5])
@pytest.mark.parametrize("norm", [0, 1])
def test_interval_stopping_rule_matches_oracle(L, c, lo, norm):
    """The library's own bound and rounds for the series on [lambda_lo, 1]
    equal the oracle's (written separately from it); lambda_lo = -1 gives the
    plain rule."""
    from oracle import oracle as O
    for kappa in (1.0, 74.0, 1.6e4):
        for tol in (1e-3, 1e-6, 1e-10):
            assert L.cpaa_rounds_needed_interval(c, lo, tol, kappa, norm) == \
                O.rounds_needed_interval(c, lo, tol, kappa, norm)
            if lo == -1.0:
                assert L.cpaa_rounds_needed_interval(c, lo, tol, kappa, norm) == L.cpaa_rounds_needed(c, tol, kappa, norm)
        for M in (1, 7, 30):
            a, b = L.cpaa_l1_bound_interval(c, lo, M, kappa, norm), O.l1_bound_interval(c, lo, M, kappa, norm)
            assert abs(a - b) <= 1e-13 * abs(b)
    assert L.cpaa_rounds_needed_interval(c, 1.0, 1e-6, 1.0) == -1
    assert L.cpaa_rounds_needed_interval(c, -1.5, 1e-6, 1.0) == -1
    assert math.isnan(L.cpaa_l1_bound_interval(c, 1.0, 3, 1.0))


def test_stopping_rule_rejects_bad_args(L):
    assert L.cpaa_rounds_needed(0.0, 1e-6, 1.0) == -1
    assert L.cpaa_rounds_needed(1.0, 1e-6, 1.0) == -1
    assert L.cpaa_rounds_needed(0.85, 0.0, 1.0) == -1
    assert L.cpaa_rounds_needed(0.85, 1e-300, 1.0, 0, 50) == -1


def test_config1_rounds_from_eq41():
    """The 10k-vertex configuration stops on ERR_M < 1e-10 (Eq. 41 alone): 39
    rounds at c = 0.85."""
    from oracle import oracle as O
    M = next(m for m in range(1, 200) if O.err_bound(0.85, m) < 1e-10)
    assert M == 39


def test_struct_layouts_match_the_header(L, tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets (compiled with the host C compiler against include/cpaa.h)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"cpaa_options": L.CpaaOptions, "cpaa_info": L.CpaaInfo,
               "cpaa_server_stats": L.CpaaServerStats, "cpaa_layout": L.CpaaLayout,
               "cpaa_layout_params": L.CpaaLayoutParams}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "cpaa.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def test_plain_c_program_links_and_calls_host_entry_points(L, tmp_path):
    """A C program with no Python in it compiles against include/cpaa.h,
    links libcpaa.so and gets the same answers from the host-side entry points
    (options defaults, the stopping rule, status names) as the binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "use_abi.c"
    src.write_text(r'''
#include <stdio.h>
#include "cpaa.h"
int main(void) {
    cpaa_options o;
    cpaa_options_init(&o);
    printf("%d %d %d %d %u %d %d\n", (int)o.precision, o.normalize, o.fixed_rounds, o.max_rounds,
           o.flags, o.batch_width, (int)o.stop_rule);
    printf("%d %d %d\n", cpaa_rounds_needed(0.85, 1e-6, 74.0, 0, 2000),
           cpaa_rounds_needed(0.99, 1e-12, 1.6e4, 1, 2000), cpaa_rounds_needed(0.5, 1e-300, 1.0, 0, 10));
    printf("%.17g %.17g\n", cpaa_l1_bound(0.85, 30, 74.0, 0), cpaa_l1_bound(0.95, 7, 1.44, 1));
    printf("%s %s\n", cpaa_status_string(CPAA_OK), cpaa_status_string(CPAA_ENOTCONV));
    printf("[%s]\n", cpaa_last_error());
    return 0;
}
''')
    exe = tmp_path / "use_abi"
    libdir = os.path.dirname(L.library_path)
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lcpaa", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    o = L.cpaa_options_init()
    assert out[0].split() == [str(v) for v in (o.precision, o.normalize, o.fixed_rounds, o.max_rounds,
                                               o.flags, o.batch_width, o.stop_rule)]
    assert [int(v) for v in out[1].split()] == [L.cpaa_rounds_needed(0.85, 1e-6, 74.0, 0, 2000),
                                                L.cpaa_rounds_needed(0.99, 1e-12, 1.6e4, 1, 2000), -1]
    b = [float(v) for v in out[2].split()]
    assert b == [L.cpaa_l1_bound(0.85, 30, 74.0, 0), L.cpaa_l1_bound(0.95, 7, 1.44, 1)]
    assert out[3].split() == ["CPAA_OK", "CPAA_ENOTCONV"]
    assert out[4] == "[]"


def test_graph_create_rejects_bad_csr_before_any_device_work(L):
    """cpaa_graph_create checks a host CSR's sizes and row pointers on the host
    before its first CUDA call: empty or oversized graphs, a bad row_ptr and a
    degree-0 vertex (Sec. 2.1 needs d_i > 0) are EINVAL, with the reason."""
    i32 = lambda v: np.asarray(v, dtype=np.int32)
    ok_rp, ok_cx = i32([0, 1, 2]), i32([1, 0])
    cases = [
        (0, 2, ok_rp, ok_cx, "n out of range"),
        (2, 0, ok_rp, ok_cx, "nnz out of range"),
        (2, 1 << 31, ok_rp, ok_cx, "nnz out of range"),
        (2, 2, None, ok_cx, "NULL"),
        (2, 2, ok_rp, None, "NULL"),
        (2, 2, i32([1, 1, 2]), ok_cx, "row_ptr[0]"),
        (2, 3, ok_rp, i32([1, 0, 0]), "row_ptr[n] != nnz"),
        (3, 3, i32([0, 2, 1, 3]), i32([1, 2, 0]), "decreases at row 1"),
        (3, 2, i32([0, 1, 1, 2]), i32([2, 0]), "vertex 1 has degree 0"),
    ]
    for n, nnz, rp, cx, why in cases:
        with pytest.raises(L.CpaaError) as e:
            L.cpaa_graph_create(n, nnz, rp, cx)
        assert e.value.status == L.CPAA_EINVAL, why
        assert why in str(e.value), (why, str(e.value))


def test_layout_params_checked_before_any_device_work(L):
    """cpaa_graph_create_ex rejects out-of-range layout parameters (and an
    unknown tuning precision) on the host, before its first CUDA call."""
    rp, cx = np.asarray([0, 1, 2], dtype=np.int32), np.asarray([1, 0], dtype=np.int32)
    bad = [({"hub_degree": 31}, "hub_degree"), ({"hub_degree": -1}, "hub_degree"),
           ({"hub_tile": 100}, "hub_tile"), ({"hub_tile": 1026}, "hub_tile"), ({"hub_tile": 1 << 21}, "hub_tile"),
           ({"long_chunk": -3}, "long_chunk"), ({"sort_window": 48}, "sort_window"),
           ({"sort_window": 1 << 21}, "sort_window"), ({"tune_precision": 9}, "tune_precision")]
    for params, why in bad:
        with pytest.raises(L.CpaaError) as e:
            L.cpaa_graph_create_ex(2, 2, rp, cx, 0, params)
        assert e.value.status == L.CPAA_EINVAL, why
        assert why in str(e.value), (why, str(e.value))


def test_server_rejects_the_interval_flags(L):
    """The server runs the series on [-1, 1] only: either interval flag is
    EINVAL at creation, before any device work."""
    import ctypes
    for flag in (L.CPAA_INTERVAL, L.CPAA_CERTIFY_INTERVAL):
        o = L.cpaa_options_init()
        o.flags = flag
        h = ctypes.c_void_p()
        st = L.lib().cpaa_server_create(1 << 20, ctypes.byref(o), ctypes.byref(h))
        assert st == L.CPAA_EINVAL and not h.value
        assert "[-1, 1]" in L.cpaa_last_error()


def test_host_side_argument_checks(L):
    """Checks made before any device work: NULL handles, and the server's
    options (precision, normalisation, stopping rule)."""
    def einval(fn, why):
        with pytest.raises(L.CpaaError) as e:
            fn()
        assert e.value.status == L.CPAA_EINVAL, why
        assert why in str(e.value), (why, str(e.value))

    p, pi = np.full(2, 0.5), np.empty(2)
    einval(lambda: L.cpaa_solve(None, p, 0.85, 1e-6, pi), "graph is NULL")
    einval(lambda: L.cpaa_power_solve(None, p, 0.85, 1e-6, pi), "graph is NULL")
    einval(lambda: L.cpaa_graph_info(None), "graph is NULL")
    einval(lambda: L.cpaa_graph_layout(None), "NULL")
    einval(lambda: L.Server(1 << 30, precision=7), "unknown precision")
    einval(lambda: L.Server(1 << 30, normalize=2), "normalize must be 0 or 1")
    einval(lambda: L.Server(1 << 30, stop_rule=5), "unknown stop_rule")
    einval(lambda: L.cpaa_server_submit(None, 0, np.array([1], dtype=np.int32), None, 0.85, 1e-6), "NULL")
    einval(lambda: L.cpaa_server_get_stats(None), "NULL")


def _fresh_python(code):
    import subprocess
    import sys
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)


def test_missing_library_fails_loudly(L):
    """With no built library the binding raises on first use; there is no
    other implementation to fall back to."""
    r = _fresh_python(
        "import paper_2112_01743_gb300.cpaa as m\n"
        "m.library_path = '/nonexistent/libcpaa.so'\n"
        "try:\n"
        "    m.cpaa_options_init()\n"
        "except ImportError as e:\n"
        "    print('raised:', e)\n"
        "else:\n"
        "    print('no error')\n")
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("raised:") and "not built" in r.stdout, r.stdout


def test_product_never_loads_the_oracle(L):
    """The library and its binding import nothing from oracle/ (only the tests,
    the smoke check and the benchmark's CPU leg may)."""
    r = _fresh_python(
        "import sys, paper_2112_01743_gb300 as pkg\n"
        "pkg.cpaa_options_init(); pkg.cpaa_rounds_needed(0.85, 1e-6, 10.0)\n"
        "print(sorted(m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')))\n")
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "[]", r.stdout
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2112_01743_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", src, re.M), f
                assert "cpaa_oracle" not in src and "liboracle" not in src, f
