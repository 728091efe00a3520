"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gpulsm.h declares (no GPU needed, no compute calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    with open(os.path.join(ROOT, "include", "gpulsm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsm_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lsm_lib):
    lib = ctypes.CDLL(lsm_lib.LIB_PATH)
    names = declared_entry_points()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(lsm_lib.EXPORTED)


def test_host_only_calls_without_gpu(lsm_lib):
    assert lsm_lib.lsm_status_str(0) == "LSM_OK"
    assert lsm_lib.lsm_status_str(6) == "LSM_ERR_CAPACITY"
    lib = lsm_lib._lib
    assert lib.lsm_stats(None, None, None, None, None) == lsm_lib.LSM_ERR_ARG
    assert lib.lsm_capacity(None) == 0
    h = ctypes.c_void_p()
    assert lib.lsm_create(ctypes.byref(h), 0, 100, 0) == lsm_lib.LSM_ERR_ARG      # b = 0
    assert lib.lsm_create(None, 16, 100, 0) == lsm_lib.LSM_ERR_ARG                # no handle slot
    assert lib.lsm_create(ctypes.byref(h), 1 << 27, 100, 0) == lsm_lib.LSM_ERR_ARG  # b too large


def test_built_for_sm_103a():
    from paper_1707_05354_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_library_resolves_its_own_symbols(lsm_lib):
    """Every internal (gpulsm::) function the library calls is defined in it:
    a declaration left without a definition would only fail when loaded."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "-C", "--undefined-only", lsm_lib.LIB_PATH], capture_output=True, text=True)
    missing = [ln for ln in out.stdout.splitlines() if "gpulsm::" in ln]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path):
    """Importing the binding from a package copy without libgpulsm.so raises:
    there is no CPU fallback to fall back on."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "paper_1707_05354_gb300"
    pkg.mkdir()
    for f in ("__init__.py", "gpulsm.py"):
        shutil.copy2(os.path.join(ROOT, "paper_1707_05354_gb300", f), pkg / f)
    env = dict(os.environ)
    env.pop("PYTHONPATH", None)
    p = subprocess.run([sys.executable, "-c", "import paper_1707_05354_gb300.gpulsm"],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode != 0
    assert "ImportError" in p.stderr and "libgpulsm.so is not built" in p.stderr


def _oracle_imports(path):
    """(line, enclosing function names, enclosing if-tests) of every import of
    the oracle package in a Python file."""
    import ast
    with open(path) as f:
        tree = ast.parse(f.read())
    found = []

    def walk(node, funcs, tests):
        for ch in ast.iter_child_nodes(node):
            f2, t2 = funcs, tests
            if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)):
                f2 = funcs + [ch.name]
            if isinstance(ch, ast.If):
                t2 = tests + [ast.unparse(ch.test)]
            if isinstance(ch, ast.Import):
                mods = [a.name for a in ch.names]
            elif isinstance(ch, ast.ImportFrom):
                mods = [ch.module or ""]
            else:
                mods = []
            if any(m.split(".")[0] == "oracle" for m in mods):
                found.append((ch.lineno, f2, t2))
            walk(ch, f2, t2)

    walk(tree, [], [])
    return found


def test_product_path_never_reaches_the_oracle():
    """The package, its CUDA sources and the header never name the oracle;
    the benchmark imports it only in its CPU-baseline legs."""
    pkg = os.path.join(ROOT, "paper_1707_05354_gb300")
    for base, _, files in os.walk(pkg):
        if "__pycache__" in base or "_build" in base:
            continue
        for f in files:
            if f.endswith(".py"):
                assert not _oracle_imports(os.path.join(base, f)), f
            if f.endswith((".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(base, f)) as fh:
                    assert "oracle" not in fh.read().lower(), f
    with open(os.path.join(ROOT, "include", "gpulsm.h")) as fh:
        assert "oracle" not in fh.read().lower()
    sites = _oracle_imports(os.path.join(ROOT, "bench.py"))
    assert sites
    for line, funcs, tests in sites:
        assert funcs and funcs[0] in ("oracle_sample", "run_reference", "run_gpu", "run_batched"), line
        if funcs[0] in ("run_gpu", "run_batched"):
            assert any("no_cpu_baseline" in t for t in tests), line


def test_header_is_plain_c_and_links(lsm_lib, tmp_path):
    """include/gpulsm.h compiles as strict C99 and C++17 (no C++ or torch types
    in the signatures), and a C program links against libgpulsm.so and calls
    its host-only entry points."""
    import shutil
    import subprocess
    gcc, gxx = shutil.which("gcc"), shutil.which("g++")
    if gcc is None or gxx is None:
        pytest.skip("gcc / g++ not available")
    src = tmp_path / "abi.c"
    src.write_text(
        '#include <stdio.h>\n#include <string.h>\n#include "gpulsm.h"\n'
        "int main(void) {\n"
        "  lsm_t* h = NULL;\n"
        "  uint64_t r = 0, n = 0; uint32_t b = 0;\n"
        '  if (strcmp(lsm_status_str(LSM_OK), "LSM_OK") != 0) return 1;\n'
        '  if (strcmp(lsm_status_str(LSM_ERR_TIMEOUT), "LSM_ERR_TIMEOUT") != 0) return 2;\n'
        "  if (lsm_create(&h, 0, 100, 0) != LSM_ERR_ARG || h != NULL) return 3;\n"
        "  if (lsm_stats(NULL, &r, &n, &b, NULL) != LSM_ERR_ARG) return 4;\n"
        "  if (lsm_capacity(NULL) != 0) return 5;\n"
        '  printf("ok\\n");\n'
        "  return 0;\n}\n")
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(lsm_lib.LIB_PATH)
    exe = tmp_path / "abi"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, str(src),
                    "-L", libdir, "-lgpulsm", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    cpp = tmp_path / "abi.cpp"
    cpp.write_text('#include "gpulsm.h"\nint main() { return lsm_capacity(nullptr) == 0 ? 0 : 1; }\n')
    subprocess.run([gxx, "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-I", inc,
                    str(cpp)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)


def test_profile_codes(lsm_lib, monkeypatch):
    """lsm_profile: 0 off, 1 every group, 2 + g group g alone; the binding
    maps a group's name to its code (the library checks the handle first)."""
    assert lsm_lib._lib.lsm_profile(None, 1) == lsm_lib.LSM_ERR_ARG
    seen = []

    class Fake:
        def lsm_profile(self, h, code):
            seen.append(code)
            return 0

    monkeypatch.setattr(lsm_lib, "_lib", Fake())
    for arg in (True, False, "merge", "sort", "cleanup"):
        lsm_lib.lsm_profile(None, arg)
    g = lsm_lib.PROF_GROUPS
    assert seen == [1, 0, 2 + g.index("merge"), 2 + g.index("sort"), 2 + g.index("cleanup")]
    assert g.index("merge") == 2 and len(g) == 7   # the header's lsm_prof_group order
