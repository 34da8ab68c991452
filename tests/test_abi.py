"""The C-ABI library builds, loads, and exports every function include/ipm.h declares (no GPU)."""
import os
import re
import subprocess

import pytest

from paper_1806_05896_gb300 import build, ipm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "ipm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ipm_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ipm.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", ipm.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (ipm_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(ipm.EXPORTED) == set(names)
    for n in names:
        assert hasattr(lib, n)


def test_default_options_are_the_papers(lib):
    o = ipm.default_options()
    assert (o.sigma, o.alpha0, o.eps_p, o.eps_d, o.eps_c) == (0.2, 0.995, 1e-6, 1e-6, 1e-6)
    assert (o.krylov_tol, o.cheb_steps, o.vcycles, o.smooth_pre, o.smooth_post) == (1e-10, 20, 3, 5, 5)
    assert o.mu0 == 1.0


def test_strerror_without_gpu(lib):
    assert lib.ipm_strerror(ipm.EINVAL).decode() == "invalid argument"
    assert lib.ipm_strerror(99).decode() == "unknown error"


def test_library_is_built_for_sm103a(lib):
    """The fatbinary carries sm_103a code (checked from the build flags, not by disassembly)."""
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1806_05896_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "from oracle" not in src and "import oracle" not in src


def test_server_wait_returns_the_solves_own_error(lib):
    """A request whose solver cannot be created reports the creation's status through
    ipm_server_wait, not an argument error about the control buffer. Without a GPU the
    creation fails with IPM_ENOMEM / IPM_ECUDA; with one, bounds violating u_a < 0 < u_b
    make it fail with IPM_EINVAL. Either way the returned code is the creation's."""
    import numpy as np
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    sv = ipm.Server(workers=1, budget_bytes=1 << 30)
    try:
        n = 9
        ub = 1.0 if not has_gpu else -1.0
        t = sv.submit(2, n, 1e-2, 1e-3, -1.0, ub, np.zeros(n * n))
        with pytest.raises(ipm.IpmError) as e:
            sv.wait(t)
        want = (ipm.EINVAL,) if has_gpu else (ipm.ENOMEM, ipm.ECUDA)
        assert e.value.code in want
    finally:
        sv.close()


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every public struct the binding passes through the ABI has the header's size and field
    offsets (compiled with the host C compiler against include/ipm.h)."""
    import ctypes
    pairs = [("ipm_grid", ipm.Grid), ("ipm_pde", ipm.Pde), ("ipm_bounds", ipm.Bounds),
             ("ipm_options", ipm.Options), ("ipm_report", ipm.Report),
             ("ipm_request", ipm.Request)]
    lines = []
    for cname, cls in pairs:
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"ipm.h\"\n"
                   "int main(void) {\n" + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, cls in pairs:
        assert ctypes.sizeof(cls) == got[(cname, "sizeof")], cname
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == got[(cname, field)], (cname, field)
