"""Memory and undefined-behaviour checks of the CPU code on the CPU: the oracle
and the library's host set-up (assembly, sliced-ELL layout, renumbering) are
built with AddressSanitizer and UndefinedBehaviorSanitizer and run on a subset
of their tests; any report aborts the run (halt_on_error)."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLAGS = ["-O1", "-g", "-fPIC", "-shared", "-fopenmp", "-fsanitize=address,undefined", "-fno-omit-frame-pointer"]


def _runtime():
    if shutil.which("gcc") is None or shutil.which("g++") is None:
        pytest.skip("gcc/g++ not available")
    libs = [subprocess.run(["gcc", f"-print-file-name={n}"], capture_output=True, text=True).stdout.strip()
            for n in ("libasan.so", "libubsan.so")]
    if not all(os.path.isabs(p) and os.path.exists(p) for p in libs):
        pytest.skip("sanitizer runtimes not installed")
    return " ".join(libs)


def _env(preload, **extra):
    return dict(os.environ, LD_PRELOAD=preload, ASAN_OPTIONS="detect_leaks=0:halt_on_error=1",
                UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", **extra)


def test_oracle_under_sanitizers(tmp_path):
    preload = _runtime()
    lib = str(tmp_path / "libidp_oracle_san.so")
    subprocess.run(["gcc", *FLAGS, "-std=c11", "-ffp-contract=off", "-o", lib,
                    os.path.join(ROOT, "oracle", "idp_oracle.c"), "-lm"], check=True)
    pins = ["tests/test_oracle_matrices.py", "tests/test_oracle_symmetry.py",
            "tests/test_oracle_2d.py::test_uniform_periodic_closed_forms_2d",
            "tests/test_oracle_2d.py::test_identities_any_quad_mesh",
            "tests/test_oracle_stage.py::test_trace_identities", "tests/test_oracle_pointwise.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *pins], cwd=ROOT,
                       env=_env(preload, IDP_ORACLE_LIB=lib), capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])


def test_library_host_code_under_sanitizers(tmp_path):
    preload = _runtime()
    lib = str(tmp_path / "libhost_layout_san.so")
    csrc = os.path.join(ROOT, "paper_2007_00094_gb300", "csrc")
    subprocess.run(["g++", *FLAGS, "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", csrc, "-o", lib,
                    os.path.join(ROOT, "tests", "host_layout.cpp"), os.path.join(csrc, "idp_mesh.cpp")], check=True)
    code = f"""
import ctypes, sys
sys.path[:0] = [{ROOT!r}, {os.path.join(ROOT, 'tests')!r}]
import test_host_layout as T
lib = ctypes.CDLL({lib!r})
lib.host_layout.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, T._i64p, T._dp, ctypes.c_int, T._i64p,
                            T._i64p]
for name, make in T.MESHES.items():
    for ren in (0, 1):
        mesh = T._shuffle(make(), 7) if ren else make()
        perm, s = T._layout(lib, mesh, ren)
        assert not {{k: v for k, v in s.items() if k not in ('n_slots', 'bandwidth') and v}}, (name, ren, s)
print('ok')
"""
    r = subprocess.run([sys.executable, "-c", code], env=_env(preload), capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "ok" in r.stdout, (r.stdout[-2000:], r.stderr[-3000:])
