"""The C-ABI library loads and exports every entry point include/tps.h declares (no GPU needed).

Also checks the host-side set-up routine tps_two_body_v0 (no device work) against the oracle.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tps.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tps_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_02534_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/tps.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2111_02534_gb300", "libtps.so")],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (tps_\w+)", out))
    assert exported == set(names), f"exported but undeclared: {exported - set(names)}"


def test_binding_covers_header(lib):
    from paper_2111_02534_gb300 import tps
    assert set(tps.EXPORTED) == set(_declared())


def test_status_strings_and_defaults(lib):
    from paper_2111_02534_gb300 import tps
    assert tps._lib.tps_status_string(0) == b"ok"
    assert tps._lib.tps_status_string(-5) == b"singular preconditioner shift"
    o = tps.default_opts()
    assert o.use_prec == 1 and o.prec_shift != o.prec_shift   # NaN: adaptive shift
    # argument checks that fail before any device work
    assert tps._lib.tps_create(None, 1, 0) == tps.ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert tps._lib.tps_create(ctypes.byref(h), 3, 0) == tps.ERR_INVALID_ARG


@pytest.mark.parametrize("E0,shape,mu,sigma", [(0.1, 0, 1.0, 1.0), (1e-3, 0, 40 / 41, 1.0), (0.3, 1, 0.5, 2.0)])
def test_two_body_v0_host_setup_matches_oracle(lib, E0, shape, mu, sigma):
    from paper_2111_02534_gb300 import tps
    from oracle.two_body import tune_v0
    n, L = 256, 20.0
    got = tps.two_body_v0(1, mu, 1.0, E0, shape, sigma, n, L)
    ref = tune_v0(E0, mu, sigma, shape, n, L)
    assert got == pytest.approx(ref, rel=1e-11)
    with pytest.raises(tps.TpsError):
        tps.two_body_v0(1, mu, 1.0, -1.0, shape, sigma, n, L)


def test_two_body_v0_2d_host_setup_matches_oracle(lib):
    from paper_2111_02534_gb300 import tps
    from oracle.two_body import tune_v0
    got = tps.two_body_v0(2, 1.0, 1.0, 0.2, 0, 1.0, 24, 8.0)
    assert got == pytest.approx(tune_v0(0.2, 1.0, 1.0, 0, 24, 8.0, dim=2), rel=1e-11)


def test_binding_structs_match_header(tmp_path):
    # the ctypes mirrors of tps_solver_opts and tps_stats have the C layout: every field
    # offset and the struct sizes, from a C program compiled against include/tps.h
    import shutil
    import subprocess
    from paper_2111_02534_gb300 import tps
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    lines = ['#include <stdio.h>', '#include "tps.h"', "int main(void) {"]
    for cname, py in (("tps_solver_opts", tps.SolverOpts), ("tps_stats", tps.Stats)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in (("tps_solver_opts", tps.SolverOpts), ("tps_stats", tps.Stats)):
        assert got[(cname, "size")] == ctypes.sizeof(py)
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
