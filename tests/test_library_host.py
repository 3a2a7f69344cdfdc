"""Host-side tests of the C ABI (no GPU): the library loads, exports every
symbol the header declares, validates arguments before touching the device,
and its host-only helpers (batch split, tuner cache) behave."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spuma.h")


@pytest.fixture(scope="module")
def L():
    from paper_2512_22215_gb300 import build as B
    B.build()
    from paper_2512_22215_gb300._lib import lib
    return lib()


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(spuma_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_header_is_plain_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "spuma.h"\nint main(void){ spuma_solver_controls c; spuma_solver_perf p;'
                   ' (void)c; (void)p; return (int)sizeof(spuma_solver_perf) - 48; }\n')
    exe = tmp_path / "t"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    assert subprocess.run([str(exe)]).returncode == 0


def test_exports_every_declared_symbol(L):
    names = header_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(L):
    for s in range(10):
        assert len(L.spuma_status_string(s)) >= 2
    assert L.spuma_status_string(9) != b"unknown status"
    assert L.spuma_status_string(99) == b"unknown status"


def test_workspace_bytes(L):
    assert L.spuma_workspace_bytes(-1, 0, 0) == 0
    a = L.spuma_workspace_bytes(1000, 3000, 0)
    b = L.spuma_workspace_bytes(2000, 6000, 0)
    assert 0 < a < b
    big = L.spuma_workspace_bytes(8_000_000, 23_880_000, 0)
    assert 2.0e9 < big < 4.5e9


def test_create_rejects_bad_arguments_without_device(L):
    h = C.c_void_p()
    ws = (C.c_uint8 * 4096)()
    # negative size, NULL out, NULL workspace, misaligned workspace, too small
    assert L.spuma_ldu_create(-1, 0, None, None, C.addressof(ws), 4096, None, C.byref(h)) == 1
    assert L.spuma_ldu_create(4, 0, None, None, C.addressof(ws), 4096, None, None) == 1
    assert L.spuma_ldu_create(4, 0, None, None, None, 4096, None, C.byref(h)) == 1
    base = (C.addressof(ws) + 255) // 256 * 256
    assert L.spuma_ldu_create(4, 0, None, None, base + 8, 1024, None, C.byref(h)) == 1
    assert L.spuma_ldu_create(1000, 2000, 1, 1, base, 1024, None, C.byref(h)) == 4
    assert L.spuma_ldu_create(4, 3, None, None, base, 1024, None, C.byref(h)) == 1   # NULL addressing
    assert b"NULL" in L.spuma_last_error()


def test_entry_points_reject_null_handle(L):
    from paper_2512_22215_gb300._lib import Controls
    ctl = Controls(2, 0, 1e-8, 0.0, 1e-4, 100, 0, 10, 0)
    assert L.spuma_pcg_solve(None, None, None, None, None, C.byref(ctl), None, None) == 1
    assert L.spuma_amul(None, 0, None, None, None, None, None) == 1
    assert L.spuma_matrix_prepare(None, None, None, 2, None) == 1
    assert L.spuma_ldu_info(None, None, None, None) == 1
    assert L.spuma_batch_run(None, None) == 1
    bad = Controls(7, 0, 1e-8, 0.0, 1e-4, 100, 0, 10, 0)
    assert L.spuma_pcg_solve(None, None, None, None, None, C.byref(bad), None, None) == 1


def test_batch_split(L):
    w = (C.c_double * 4)(1.0, 3.0, 0.0, 4.0)
    out = (C.c_int32 * 5)()
    assert L.spuma_batch_split(4, w, 20, out) == 1
    split = list(out)
    assert split[0] == 0 and split[-1] == 20
    nb = [split[k + 1] - split[k] for k in range(4)]
    assert min(nb) >= 1
    assert nb[3] >= nb[1] >= nb[0] and nb[2] == 1
    assert L.spuma_batch_split(4, w, 3, out) == 0          # fewer blocks than systems
    # proportional: weights 1:1 -> equal
    w2 = (C.c_double * 2)(5.0, 5.0)
    out2 = (C.c_int32 * 3)()
    assert L.spuma_batch_split(2, w2, 10, out2) == 1 and list(out2) == [0, 5, 10]


def test_tune_cache_roundtrip(L, tmp_path):
    path = str(tmp_path / "tune.json").encode()
    t, p, d, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
    assert L.spuma_tune_cache_lookup(path, b"sig-a", C.byref(t), C.byref(p), C.byref(d), C.byref(ms)) == 0
    assert L.spuma_tune_cache_store(path, b"sig-a", 256, 1, 1, 12.5) == 1
    assert L.spuma_tune_cache_store(path, b"sig-b", 512, 0, 2, 3.25) == 1
    assert L.spuma_tune_cache_store(path, b"sig-c", 512, 0, 0, 3.25) == 0      # grid divisor >= 1
    import json
    data = json.loads(open(path).read())
    assert data == {"sig-a": [256, 1, 1, 12.5], "sig-b": [512, 0, 2, 3.25]}
    assert L.spuma_tune_cache_lookup(path, b"sig-b", C.byref(t), C.byref(p), C.byref(d), C.byref(ms)) == 1
    assert (t.value, p.value, d.value, ms.value) == (512, 0, 2, 3.25)


def test_tune_cache_reads_three_number_lines(L, tmp_path):
    """Entries of the older [threads, policy, ms] form read with grid divisor 1."""
    path = tmp_path / "old.json"
    path.write_text('{\n  "sig-old": [128, 0, 7.500000]\n}\n')
    t, p, d, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
    assert L.spuma_tune_cache_lookup(str(path).encode(), b"sig-old", C.byref(t), C.byref(p), C.byref(d),
                                     C.byref(ms)) == 1
    assert (t.value, p.value, d.value, ms.value) == (128, 0, 1, 7.5)


def test_batch_create_rejects_unknown_flags(L):
    from paper_2512_22215_gb300._lib import Controls
    ctl = Controls(2, 0, 1e-8, 0.0, 1e-4, 100, 0, 10, 0)
    one = (C.c_void_p * 1)(1)
    h = C.c_void_p()
    assert L.spuma_batch_create(1, one, one, one, one, one, C.byref(ctl), 1, 8, None, C.byref(h)) == 1
    assert L.spuma_batch_info(None, None, None, None, None) == 1
    assert L.spuma_batch_trials(None, 0, None, None, None, None) == 0


def test_static_solve_checks_arguments_before_the_device(L):
    """The no-allocation solve rejects bad controls and NULL arrays on the
    host, before it looks at its shared static array (no device call)."""
    from paper_2512_22215_gb300._lib import Controls
    bad = Controls(9, 0, 1e-8, 0.0, 1e-4, 100, 0, 10, 0)
    assert L.spuma_pcg_solve_static(8, 12, None, None, None, None, None, None, None, None, None) == 1
    assert L.spuma_pcg_solve_static(8, 12, 1, 1, 1, 1, 1, 1, C.byref(bad), None, None) == 1
    ok = Controls(2, 0, 1e-8, 0.0, 1e-4, 100, 0, 10, 0)
    assert L.spuma_pcg_solve_static(8, 12, None, 1, 1, 1, 1, 1, C.byref(ok), None, None) == 1
    assert L.spuma_pcg_solve_static(-1, 0, None, None, None, None, None, None, C.byref(ok), None, None) == 1


def test_launch_counter_and_timeout_setter(L):
    n0 = L.spuma_launch_count()
    assert n0 >= 0
    L.spuma_set_barrier_timeout_ns(2_000_000_000)
    assert L.spuma_launch_count() == n0


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib
    import paper_2512_22215_gb300._lib as M
    monkeypatch.setattr(M, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(M, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        M.lib()


def test_new_entry_points_reject_bad_arguments(L):
    """The pressure step, the assembly adjoint, PBiCG and GAMG validate their
    arguments on the host (no device call)."""
    from paper_2512_22215_gb300._lib import Controls
    ctl = Controls(3, 0, 1e-8, 0.0, 1e-4, 100, 0, 10, 0)
    assert L.spuma_pbicg_solve(None, None, None, None, None, None, C.byref(ctl), None, None) == 1
    assert L.spuma_fv_weights(None, None, None, None, None, None) == 1
    assert L.spuma_fv_grad(None, None, None, None, 0, None, None, None, None, None, None) == 1
    assert L.spuma_pressure_rhs(None, None, None, None, None, None, None, 0, None, None, None, None, None) == 1
    assert L.spuma_pressure_flux(None, None, None, None, None, 0, None, None, None, None, None, None, None,
                                 None, None, None) == 1
    assert L.spuma_fv_div(None, None, 0, None, None, None, None) == 1
    assert L.spuma_assemble_laplacian_adjoint(None, None, None, 0, None, None, None, None, None, None, None, None,
                                              None) == 1
    g = C.c_void_p()
    assert L.spuma_gamg_create(None, None, None, C.byref(g)) == 1
    assert L.spuma_gamg_create(None, None, None, None) == 1
    assert L.spuma_gamg_workspace_bytes(None) == 0
    assert L.spuma_gamg_bind(None, None, 0, None) == 1
    assert L.spuma_gamg_solve(None, None, None, None, None, C.byref(ctl), None, None) == 1
    assert L.spuma_gamg_info(None, None, None, 0) == 1
    assert L.spuma_gamg_destroy(None) == 0
    assert L.spuma_gamg_set_options(None, 0, 1) == 1


def test_asymmetric_workspace_is_larger(L):
    n, f = 1000, 2700
    sym = L.spuma_workspace_bytes(n, f, 0)
    asym = L.spuma_workspace_bytes(n, f, 1)
    assert asym >= sym + 48 * f + 16 * n
