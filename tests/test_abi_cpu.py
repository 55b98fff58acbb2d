"""C ABI checks that need no GPU: the library builds and loads, exports every function
that include/submat.h declares, and rejects bad patterns on the host before any CUDA call."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_1710_10899_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        if shutil.which("nvcc") is None:
            pytest.skip("libsubmat.so not built and nvcc not available")
        from paper_1710_10899_gb300 import build
        build.build()
    return pkg.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "submat.h")).read()
    return sorted(set(re.findall(r"SUBMAT_API\s+[\w\s\*]+?\b(submat_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    import paper_1710_10899_gb300 as pkg
    assert sorted(pkg.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_defaults(lib):
    import paper_1710_10899_gb300 as pkg
    for code in pkg.STATUS:
        assert lib.submat_status_string(code)
    o = pkg.Opts()
    lib.submat_default_opts(ctypes.byref(o))
    assert o.precision == pkg.PREC_MIXED_F16 and o.k_max == 40 and o.use_graph == 1
    assert o.root_sign == -1 and o.kappa_max == 100.0
    assert o.grad_deterministic == 0 and o.grad_wave_mib == 0


def _plan_status(lib, rowptr, colind, p=2):
    import paper_1710_10899_gb300 as pkg
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    csr = pkg.CSR(len(rp) - 1, len(ci), rp.ctypes.data, ci.ctypes.data if len(ci) else None, 0)
    h = ctypes.c_void_p()
    st = lib.submat_plan(ctypes.byref(csr), p, None, ctypes.byref(h))
    return pkg.STATUS[st]


def test_host_side_validation(lib):
    import paper_1710_10899_gb300 as pkg
    # these are rejected before the library touches the GPU
    assert _plan_status(lib, [0, 1], [0], p=0) == "SUBMAT_EINVAL"
    assert _plan_status(lib, [1, 1], [0]) == "SUBMAT_EINVAL"            # rowptr[0] != 0
    assert _plan_status(lib, [0, 2, 1], [0, 1]) == "SUBMAT_EINVAL"      # decreasing rowptr
    assert _plan_status(lib, [0, 1, 1], [0]) == "SUBMAT_ENODIAG"        # empty row
    assert _plan_status(lib, [0, 1, 2, 2], [0, 1]) == "SUBMAT_ENODIAG"  # n > nnz
    big = 1537
    assert _plan_status(lib, [0, big], np.arange(big)) == "SUBMAT_ETOOBIG"
    assert lib.submat_plan(None, 2, None, None) != 0
    # root_sign other than -1 / +1
    o = pkg.Opts()
    lib.submat_default_opts(ctypes.byref(o))
    o.root_sign = 0
    rp = np.array([0, 1], dtype=np.int32)
    ci = np.array([0], dtype=np.int32)
    csr = pkg.CSR(1, 1, rp.ctypes.data, ci.ctypes.data, 0)
    h = ctypes.c_void_p()
    assert pkg.STATUS[lib.submat_plan(ctypes.byref(csr), 2, ctypes.byref(o), ctypes.byref(h))] == "SUBMAT_EINVAL"
    # grad_deterministic other than 0 / 1
    lib.submat_default_opts(ctypes.byref(o))
    o.grad_deterministic = 2
    assert pkg.STATUS[lib.submat_plan(ctypes.byref(csr), 2, ctypes.byref(o), ctypes.byref(h))] == "SUBMAT_EINVAL"
    # the mixed modes' largest root order
    lib.submat_default_opts(ctypes.byref(o))
    p_big = pkg.SUBMAT_MIXED_MAX_P + 1
    assert pkg.STATUS[lib.submat_plan(ctypes.byref(csr), p_big, ctypes.byref(o), ctypes.byref(h))] == "SUBMAT_EINVAL"
    assert b"SUBMAT_PREC_FP64" in lib.submat_last_error()


def test_noalloc_host_side_validation(lib):
    import paper_1710_10899_gb300 as pkg
    st = lib.submat_invroot_noalloc(4, 4, 1, 1, 2, pkg.SUBMAT_NOALLOC_MAX_M + 1, 1, 1 << 20, None)
    assert pkg.STATUS[st] == "SUBMAT_ETOOBIG"
    assert pkg.STATUS[lib.submat_invroot_noalloc(4, 4, 1, 1, 0, 8, 1, 1 << 20, None)] == "SUBMAT_EINVAL"
    assert pkg.STATUS[lib.submat_invroot_noalloc(4, 4, 1, 1, 2, 8, 1, 1, None)] == "SUBMAT_EINVAL"
    assert pkg.STATUS[lib.submat_invroot_noalloc(0, 0, None, None, 2, 8, None, None, None)] == "SUBMAT_OK"


def test_null_plan_and_arguments(lib):
    """Every plan-based entry point rejects a NULL plan or NULL arrays with SUBMAT_EINVAL
    (and a message) before touching the GPU."""
    import paper_1710_10899_gb300 as pkg
    buf = (ctypes.c_double * 4)()
    b = ctypes.addressof(buf)

    def einval(st):
        return pkg.STATUS[st] == "SUBMAT_EINVAL"

    assert einval(lib.submat_invroot(None, b, b + 16, None, 0))
    assert einval(lib.submat_invroot_host(None, b, b + 16, None))
    assert einval(lib.submat_invroot_backward(None, b, b + 16, None))
    assert einval(lib.submat_pcg(None, b, None, b, b, 0.0, 0, None, None, None))
    assert einval(lib.submat_get_report(None, None))
    assert einval(lib.submat_plan_rows(None, None, None))
    assert einval(lib.submat_plan_shape(None, None, None))
    assert lib.submat_last_error()
    lib.submat_plan_destroy(None)                 # a no-op


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: without the built library the binding raises ImportError."""
    import subprocess
    import sys
    missing = str(tmp_path / "libsubmat.so")
    code = ("import paper_1710_10899_gb300 as p\n"
            "try:\n"
            f"    p.load_library({missing!r})\n"
            "except ImportError as e:\n"
            "    print('raised', e)\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         timeout=120, check=True)
    assert out.stdout.startswith("raised") and "not found" in out.stdout


def test_plain_c_caller(lib, tmp_path):
    """include/submat.h compiles as strict C99, and a C program linked against
    libsubmat.so runs the host-side entry points (no GPU needed)."""
    import subprocess
    import paper_1710_10899_gb300 as pkg
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_check")
    libdir = os.path.dirname(pkg.LIB_PATH)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_check.c"),
                    "-o", exe, "-L", libdir, "-lsubmat", "-Wl,-rpath," + libdir],
                   check=True, capture_output=True, text=True, timeout=120)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    assert "abi_check ok" in out.stdout


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes structures have the C structs' size and field offsets (a C
    program built against include/submat.h prints them)."""
    import subprocess
    import paper_1710_10899_gb300 as pkg
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"submat_csr": pkg.CSR, "submat_opts": pkg.Opts, "submat_report": pkg.Report}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "submat.h"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe],
                   check=True, capture_output=True, text=True, timeout=120)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=60).stdout
    got = {}
    for ln in out.splitlines():
        cname, field, val = ln.split()
        got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_binding_constants_match_the_header():
    """Status codes, precision modes and size limits in the binding are the header's."""
    import paper_1710_10899_gb300 as pkg
    text = open(os.path.join(ROOT, "include", "submat.h")).read()
    enums = {k: int(v) for k, v in re.findall(r"\b(SUBMAT_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    macros = {k: int(v) for k, v in re.findall(r"#define\s+(SUBMAT_[A-Z0-9_]+)\s+(\d+)", text)}
    status = {k: v for k, v in enums.items() if not k.startswith("SUBMAT_PREC_")}
    assert {v: k for k, v in status.items()} == pkg.STATUS
    assert enums["SUBMAT_PREC_FP64"] == pkg.PREC_FP64
    assert enums["SUBMAT_PREC_MIXED_F16"] == pkg.PREC_MIXED_F16
    assert enums["SUBMAT_PREC_MIXED_F16_SYNC"] == pkg.PREC_MIXED_F16_SYNC
    assert macros["SUBMAT_MAX_M"] == pkg.SUBMAT_MAX_M
    assert macros["SUBMAT_NOALLOC_MAX_M"] == pkg.SUBMAT_NOALLOC_MAX_M
    assert macros["SUBMAT_SMALL_MAX_M"] == pkg.SUBMAT_SMALL_MAX_M
    assert macros["SUBMAT_MIXED_MAX_P"] == pkg.SUBMAT_MIXED_MAX_P


def _prototypes():
    text = open(os.path.join(ROOT, "include", "submat.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    out = {}
    for ret, name, args in re.findall(
            r"SUBMAT_API\s+([\w\s\*]+?)\s*\b(submat_\w+)\s*\(([^)]*)\)\s*;", text):
        params = [] if args.strip() in ("", "void") else [a.strip() for a in args.split(",")]
        out[name] = (" ".join(ret.split()), params)
    return out


def test_ctypes_signatures_match_the_header(lib):
    """Every argtype / restype of the binding has the width of the header's parameter (a
    mismatch, e.g. an int where int64_t is expected, would silently corrupt arguments)."""
    scalars = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double,
               "submat_status": ctypes.c_int32}
    protos = _prototypes()
    assert len(protos) >= 10
    for name, (ret, params) in protos.items():
        fn = getattr(lib, name)
        if ret == "void":
            assert fn.restype is None, name
        elif ret == "const char*":
            assert fn.restype is ctypes.c_char_p, name
        else:
            assert fn.restype is scalars[ret], name
        assert len(fn.argtypes) == len(params), name
        for decl, at in zip(params, fn.argtypes):
            ctype = decl.rsplit(None, 1)[0] if not decl.endswith("*") else decl
            if "*" in decl or ctype.strip() in ("submat_plan_t", "void*"):
                assert at is ctypes.c_void_p or issubclass(at, ctypes._Pointer), (name, decl)
            else:
                base = ctype.replace("const", "").strip()
                assert at is scalars[base], (name, decl, at)
