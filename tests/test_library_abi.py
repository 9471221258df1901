"""The C-ABI library builds, loads and exports every declared symbol; its
host-only parts behave as documented.  No kernel runs here (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
G = synth.GEOMETRY


@pytest.fixture(scope="module")
def lib():
    from paper_2511_02742_gb300 import build, hough
    build.build()
    return hough.load()


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(inc, fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(hough_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15, names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_tables_equal_oracle_tables(lib):
    """The library's fixed-point tables (built on the host) equal the oracle's,
    which are computed by independent code from the same definition."""
    from paper_2511_02742_gb300 import hough
    for n_theta, n_rho in [(180, 1000), (256, 256), (512, 512), (1024, 1024), (97, 332), (1, 4)]:
        C, S, D, K = hough.hough_tables(G, n_theta, n_rho)
        oc, os_, od, ok = oracle.tables(G, n_theta, n_rho)
        np.testing.assert_array_equal(C, oc)
        np.testing.assert_array_equal(S, os_)
        assert D == od and K == ok
    geom = dict(G, rho_min=-123.5, rho_max=321.25, phi_u_per_deg=100)
    C, S, D, K = hough.hough_tables(geom, 77, 444)
    oc, os_, od, ok = oracle.tables(geom, 77, 444)
    np.testing.assert_array_equal(C, oc)
    np.testing.assert_array_equal(S, os_)
    assert D == od and K == ok


def test_status_strings(lib):
    from paper_2511_02742_gb300 import hough
    assert hough.status_string(0) == "HOUGH_OK"
    assert hough.status_string(-1) == "HOUGH_ERR_INVALID_ARG"
    assert hough.status_string(-5) == "HOUGH_ERR_UNSUPPORTED_SHAPE"
    assert hough.status_string(12345) == "HOUGH_ERR_UNKNOWN"


def test_create_rejects_bad_arguments_before_touching_a_device(lib):
    from paper_2511_02742_gb300 import hough
    bad = [
        (dict(G, n_vanes=0), 64, 64, {}),
        (dict(G, rho_max=-600.0), 64, 64, {}),
        (G, 64, 64, dict(vote_threshold=0)),
        (G, 64, 64, dict(assoc_tol_bins=-1)),
        (G, 64, 64, dict(max_peaks=-3)),
    ]
    for geom, nt, nr, kw in bad:
        with pytest.raises(hough.HoughError) as e:
            hough.hough_create(geom, nt, nr, **kw)
        assert e.value.code == -1
    for nt, nr, kw in [(0, 64, {}), (64, 6, {}), (64, 2048, {}), (8192, 64, {}),
                       (64, 64, dict(max_peaks=257))]:
        with pytest.raises(hough.HoughError) as e:
            hough.hough_create(G, nt, nr, **kw)
        assert e.value.code == -5


def test_null_pointers_are_rejected(lib):
    assert lib.hough_create(None, 64, 64, None, None) == -1
    assert lib.hough_find(None, None, None, 0, None, None) == -1
    assert lib.hough_plan_launch(None, None) == -1
    lib.hough_destroy(None)
    lib.hough_plan_destroy(None)
    assert lib.hough_last_error(None) == -1
    assert lib.hough_launch_count(None) == 0
    C = np.zeros(4, np.int32)
    assert lib.hough_tables(None, 4, 4, C.ctypes.data_as(ctypes.c_void_p), None, None, None) == -1
    # the other entry points check their context and sizes before anything else
    assert lib.hough_find_host(None, None, None, 0, None, None) == -1
    assert lib.hough_encode(None, None, None, 0, None, None, None) == -1
    assert lib.hough_find_coarse_fine(None, None, None, 0, None, None, None) == -1
    assert lib.hough_find_iterative(None, None, None, 0, 1, None, None, None, None, None) == -1
    assert lib.hough_accumulate(None, None, None, 0, None, None, None) == -1
    assert lib.hough_extend(None, None, None, 0, None, 0, None, None) == -1
    assert lib.hough_time_slice(None, None, None, None, 0, 0, 5, 10, 1, None, None, None, 0,
                                None, None, None) == -1
    assert lib.hough_plan_create(None, None, None, 0, None, None, None) == -1
    assert lib.hough_autotune(None, None, None, 0, None, None, 1, None) == -1
    assert lib.hough_set_launch(None, None) == -1
    assert lib.hough_get_launch(None, None) == -1
    # the request loop: every call checks its server first; destroy is NULL-safe
    res = (ctypes.c_int64 * 8)()
    assert lib.hough_server_create(None, None, None) == -1
    assert lib.hough_server_submit(None, None, None) == -1
    assert lib.hough_server_wait(None, 1, 0, None) == -1
    assert lib.hough_server_poll(None, None, 0, ctypes.cast(res, ctypes.c_void_p)) == -1
    assert lib.hough_server_drain(None, 0) == -1
    assert lib.hough_server_get_stats(None, None) == -1
    lib.hough_server_destroy(None)
    assert lib.hough_server_clock_ns() > 0


def test_no_device_is_reported_not_faked(lib):
    """Without a GPU the library says so; it never computes on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2511_02742_gb300 import hough
    with pytest.raises(hough.HoughError) as e:
        hough.hough_create(G, 64, 64)
    assert e.value.code == -6


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets the C
    compiler gives the struct of include/hough.h."""
    import subprocess
    from paper_2511_02742_gb300 import hough
    structs = [hough.hough_geometry, hough.hough_thresholds, hough.hough_hits, hough.hough_tracks,
               hough.hough_launch, hough.hough_server_config, hough.hough_request,
               hough.hough_request_result, hough.hough_server_stats, hough.hough_extension]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hough.h"', 'int main(void) {']
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for field, _ in st._fields_:
            lines.append(f'printf("{n} {field} %zu\\n", offsetof({n}, {field}));')
    lines.append('printf("hough_peak size %zu\\n", sizeof(hough_peak));')
    lines.append('printf("hough_ext_track size %zu\\n", sizeof(hough_ext_track));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    got = dict(line.rsplit(" ", 1) for line in
               subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(got[f"{n} size"]) == ctypes.sizeof(st), n
        for field, _ in st._fields_:
            assert int(got[f"{n} {field}"]) == getattr(st, field).offset, (n, field)
    assert int(got["hough_peak size"]) == hough.PEAK_DTYPE.itemsize == 16
    assert int(got["hough_ext_track size"]) == hough.EXT_DTYPE.itemsize == 16


def test_binding_constants_match_the_header(tmp_path):
    """Every HOUGH_* integer constant of the binding has the value the C
    compiler gives the macro of the same name in include/hough.h, and every
    per-window flag and limit macro of the header has a binding constant."""
    import subprocess
    from paper_2511_02742_gb300 import hough
    src_h = open(os.path.join(ROOT, "include", "hough.h")).read()
    macros = re.findall(r"^#define\s+(HOUGH_\w+)\s+\S", src_h, flags=re.M)
    ours = {n: getattr(hough, n) for n in dir(hough) if n.startswith("HOUGH_")
            and isinstance(getattr(hough, n), int)}
    for n in macros:
        if n.startswith(("HOUGH_WIN_", "HOUGH_MAX_", "HOUGH_FLAG_")):
            assert n in ours, n
    names = sorted(set(macros) & set(ours))
    lines = ['#include <stdio.h>', '#include "hough.h"', 'int main(void) {']
    lines += [f'printf("{n} %lld\\n", (long long)({n}));' for n in names]
    lines += ['return 0;', '}']
    (tmp_path / "consts.c").write_text("\n".join(lines))
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    str(tmp_path / "consts.c")], check=True)
    got = dict(line.split() for line in
               subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines())
    assert len(names) >= 10
    for n in names:
        assert int(got[n]) == ours[n], n
