"""The C-ABI library builds, loads and exports every symbol its header
declares (no GPU needed; only host-side calls are made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"ZTOEP_API\s+[\w\s\*]+?\b(ztoep_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2506_04710_gb300 import build, ztoep
    build.build()
    return ztoep.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["ztoep_plan", "ztoep_matvec", "ztoep_solve", "ztoep_solve_host", "ztoep_footprint",
              "ztoep_plan_destroy", "ztoep_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_symbols():
        assert hasattr(lib, n), n
    from paper_2506_04710_gb300 import ztoep
    assert sorted(ztoep.EXPORTS) == declared_symbols()


def test_host_only_calls(lib):
    from paper_2506_04710_gb300 import ztoep
    assert "sm_103a" in ztoep.ztoep_version()
    assert ztoep.ztoep_status_string(0) == "ok"
    assert ztoep.ztoep_status_string(4) == "not converged"
    o = ztoep.ztoep_default_opts()
    assert o.tol == 1e-8 and o.restart == 30 and o.prec == ztoep.ZTOEP_MIXED
    d, _ = ztoep.make_desc(32, 32, 64, 512)
    fp = ztoep.ztoep_footprint(d, 1, 30)
    # resident spectrum (half the frequencies, FP64+FP32) + B (FP64+FP32) dominate
    assert 24 * 4096 * 64 * 64 // 2 < fp < 4e9
    bad, _ = ztoep.make_desc(0, 4, 8, 0)
    assert ztoep.ztoep_footprint(bad, 1, 30) == 0
    bad2, _ = ztoep.make_desc(4, 4, 8, 0, lx=6)  # 6 < 2*4-1
    assert ztoep.ztoep_footprint(bad2, 1, 30) == 0
    # grouped solve: bad counts are rejected before any device work
    assert ztoep.lib().ztoep_solve_group(0, None, ctypes.byref(o), None, None, None, None, None) == ztoep.ZTOEP_ERR_ARG
    nine = ctypes.c_void_p(1)
    assert ztoep.lib().ztoep_solve_group(9, (ctypes.c_void_p * 9)(*[nine] * 9), ctypes.byref(o),
                                         (ctypes.c_int32 * 9)(*[1] * 9), None, None, None, None) == ztoep.ZTOEP_ERR_ARG


def test_structs_match_header_layout(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler gives
    the header's structs."""
    import subprocess
    from paper_2506_04710_gb300 import ztoep
    pairs = {"ztoep_desc_t": ztoep.Desc, "ztoep_solve_opts_t": ztoep.SolveOpts,
             "ztoep_solve_info_t": ztoep.SolveInfo, "ztoep_plan_info_t": ztoep.PlanInfo,
             "ztoep_tune_t": ztoep.TuneInfo, "ztoep_sched_opts_t": ztoep.SchedOpts,
             "ztoep_request_t": ztoep.Request, "ztoep_request_state_t": ztoep.RequestState,
             "ztoep_sched_stats_t": ztoep.SchedStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ztoep.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_no_cpu_fallback_when_library_missing(tmp_path):
    from paper_2506_04710_gb300 import ztoep
    with pytest.raises(RuntimeError):
        ztoep.lib(str(tmp_path / "missing.so"))


def test_post_solve_entry_points_validate_on_the_host(lib):
    """Argument checks of the port-matrix, far-field and Schur entry points
    return ARG before any device work (no GPU needed): bad port indices,
    lengths, impedances, sizes and missing plans."""
    import ctypes
    import numpy as np
    from paper_2506_04710_gb300 import ztoep
    fake = ctypes.c_void_p(0x1000)  # never dereferenced on these paths
    fake2 = ctypes.c_void_p(0x2000)
    fake3 = ctypes.c_void_p(0x3000)
    ports = np.array([0, 4, 9], np.int32)
    ones = np.ones(3)
    z0 = np.full(3, 50.0)

    def pm(p, n, prt, ln, z):
        return lib.ztoep_port_matrices(p, n, fake, prt.ctypes.data_as(ctypes.c_void_p),
                                       ln.ctypes.data_as(ctypes.c_void_p), z.ctypes.data_as(ctypes.c_void_p),
                                       fake2, fake3, None)
    assert pm(0, 10, ports, ones, z0) == ztoep.ZTOEP_ERR_ARG
    assert pm(3, 9, ports, ones, z0) == ztoep.ZTOEP_ERR_ARG                    # port 9 >= n
    assert pm(3, 10, np.array([0, -1, 9], np.int32), ones, z0) == ztoep.ZTOEP_ERR_ARG
    assert pm(3, 10, ports, np.array([1.0, np.inf, 1.0]), z0) == ztoep.ZTOEP_ERR_ARG
    assert pm(3, 10, ports, ones, np.array([50.0, 0.0, 50.0])) == ztoep.ZTOEP_ERR_ARG
    assert lib.ztoep_port_matrices(3, 10, fake, ports.ctypes.data_as(ctypes.c_void_p),
                                   ones.ctypes.data_as(ctypes.c_void_p), z0.ctypes.data_as(ctypes.c_void_p),
                                   fake2, fake2, None) == ztoep.ZTOEP_ERR_ARG  # Y aliases S
    assert lib.ztoep_far_field_grid(None, 1, fake, 2, fake2, 1.0, 1.0, fake3, None) == ztoep.ZTOEP_ERR_ARG
    o = ztoep.ztoep_default_opts()
    assert lib.ztoep_solve_schur(None, 8, fake, fake2, ctypes.byref(o), 1, fake3, ctypes.c_void_p(0x4000),
                                 None, None) == ztoep.ZTOEP_ERR_ARG
