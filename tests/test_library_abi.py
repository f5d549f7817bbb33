"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function that include/idp.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2007_00094_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        with open(os.path.join(inc, f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(idp_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2007_00094_gb300 import idp
    assert set(_declared_functions()) == set(idp.EXPORTED)


def test_config_defaults_and_argument_checks(lib):
    from paper_2007_00094_gb300 import idp
    cfg = idp.idp_config_default()
    assert cfg.gamma == 1.4 and cfg.cfl == 0.5 and cfg.limiter_passes == 2 and cfg.newton_max == 2
    ctx = ctypes.c_void_p()
    bad = idp.idp_config_default()
    bad.gamma = 1.6667  # kernels are specialised for gamma = 7/5
    assert idp.load().idp_create(ctypes.byref(bad), None, ctypes.byref(ctx)) == 1
    bad = idp.idp_config_default()
    bad.cfl = 1.5
    assert idp.load().idp_create(ctypes.byref(bad), None, ctypes.byref(ctx)) == 1
    assert idp.load().idp_status_string(5) == b"CFL violation"


def test_sources_target_sm103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)


def _c_layout(struct, fields, tmp_path):
    """sizeof and field offsets of a struct of include/idp.h, from a C program."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    prog = tmp_path / "layout.c"
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "idp.h"', "int main(void) {",
             f'  printf("%zu", sizeof({struct}));']
    lines += [f'  printf(" %zu", offsetof({struct}, {f}));' for f in fields]
    lines += ['  printf("\\n");', "  return 0;", "}"]
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(prog)], check=True)
    return [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """The binding's idp_config and idp_bounds_report have the C compiler's size
    and field offsets (a field added on one side only would shift the rest)."""
    from paper_2007_00094_gb300 import idp
    for cls, name in ((idp.IdpConfig, "idp_config"), (idp.BoundsReport, "idp_bounds_report")):
        fields = [f[0] for f in cls._fields_]
        layout = _c_layout(name, fields, tmp_path)
        assert layout[0] == ctypes.sizeof(cls), name
        assert layout[1:] == [getattr(cls, f).offset for f in fields], name
