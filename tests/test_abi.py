"""The C ABI boundary: the library loads and exports every function that
include/rewl.h declares; argument checking happens before any CUDA call; the
Python layer fails loudly when the library is missing (no CPU fallback)."""
import ctypes as C
import os
import re

import pytest

import paper_1312_3004_gb300 as pkg
from paper_1312_3004_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(rewl_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for n in ("rewl_create", "rewl_run", "rewl_get_lng", "rewl_destroy", "rewl_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.rewl_version().startswith(b"rewl-gb300")


@pytest.mark.slow
def test_debug_build_with_bounds_checks(monkeypatch):
    """The build with the kernels' bounds checks compiles (sm_103a) and exports
    the same entry points; REWL_DEBUG=1 makes the package load it."""
    from paper_1312_3004_gb300 import build

    path = build.build(debug=True)
    assert path.endswith("librewl_debug.so") and os.path.exists(path)
    monkeypatch.setenv("REWL_DEBUG", "1")
    monkeypatch.setattr(_lib, "_lib", None)
    lib = _lib.load()
    assert lib._name == path
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.rewl_server_release(None, 1) == 1   # host paths behave alike


@pytest.mark.parametrize("args", [
    (1, 8, 4, 0.75, 2, 1e-6, 0.8, 1000, 1),       # q < 2
    (2, 2, 4, 0.75, 2, 1e-6, 0.8, 1000, 1),       # L < 3
    (2, 8, 0, 0.75, 2, 1e-6, 0.8, 1000, 1),       # h < 1
    (2, 8, 4, 1.0, 2, 1e-6, 0.8, 1000, 1),        # overlap >= 1
    (2, 8, 4, 0.75, 0, 1e-6, 0.8, 1000, 1),       # m < 1
    (2, 8, 4, 0.75, 2, 0.0, 0.8, 1000, 1),        # lnf_final <= 0
    (2, 8, 4, 0.75, 2, 1e-6, 1.0, 1000, 1),       # flatness >= 1
    (2, 8, 4, 0.75, 2, 1e-6, 0.8, 0, 1),          # K < 1
    (2, 4, 40, 0.75, 2, 1e-6, 0.8, 1000, 1),      # window narrower than 8 bins
])
def test_invalid_arguments_are_rejected_before_any_device_work(args):
    lib = _lib.load()
    h = C.c_void_p()
    st = lib.rewl_create(*args, C.byref(h))
    assert st == 1  # REWL_ERR_ARG
    assert h.value is None
    assert len(lib.rewl_last_error()) > 0


def test_null_handles_are_rejected():
    lib = _lib.load()
    assert lib.rewl_run(None, 1, None) == 1
    assert lib.rewl_get_lng(None, None, 0, 0) == 1
    lib.rewl_destroy(None)  # NULL-safe


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/librewl.so")
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        pkg.REWL(2, 8, 4, 0.75, 2, 1e-6, 0.8, 1000, 1)


def params(**kw):
    base = dict(q=2, L=8, h=4, overlap=0.75, m=2, lnf_final=1e-6, flatness=0.8, exchange_interval=1000, seed=1)
    base.update(kw)
    return _lib.Params(**base)


def test_batch_arguments_are_checked_before_any_device_work():
    lib = _lib.load()
    out = C.c_void_p()
    assert lib.rewl_batch_create(None, 1, 0, C.byref(out)) == 1
    jobs = (_lib.Params * 2)(params(q=1), params())
    assert lib.rewl_batch_create(jobs, 0, 0, C.byref(out)) == 1  # n < 1
    assert lib.rewl_batch_create(jobs, 2, 0, C.byref(out)) == 1  # job 0 has q < 2
    assert out.value is None
    assert b"job 0" in lib.rewl_last_error()
    wide = (_lib.Params * 1)(params(q=17))
    assert lib.rewl_batch_create(wide, 1, 4, C.byref(out)) == 1  # q > 16 cannot pack in 4 bits
    ok = (_lib.Params * 1)(params())
    assert lib.rewl_batch_create_ext(ok, 1, 0, 3, C.byref(out)) == 1  # lanes must be 0, 1 or 32
    assert b"lanes" in lib.rewl_last_error()
    assert lib.rewl_batch_run(None, 1, None) == 1
    lib.rewl_batch_destroy(None)


def test_server_arguments_are_checked_before_any_device_work():
    lib = _lib.load()
    out = C.c_void_p()
    assert lib.rewl_server_create(1024, 4, C.byref(out)) == 1  # pool below 4 KiB
    assert lib.rewl_server_create(1 << 20, 0, C.byref(out)) == 1  # max_jobs < 1
    assert out.value is None
    jid = C.c_longlong()
    p = params()
    assert lib.rewl_server_submit(None, C.byref(p), 0, C.byref(jid)) == 1
    assert lib.rewl_server_step(None, 1, None, None) == 1
    assert lib.rewl_server_release(None, 1) == 1
    lib.rewl_server_destroy(None)


@pytest.mark.parametrize("kw", [dict(q=1), dict(L=2), dict(m=0), dict(overlap=1.0), dict(lnf_final=1.5),
                                dict(flatness=0.0), dict(exchange_interval=0), dict(L=4, h=40)])
def test_static_run_rejects_bad_parameters_before_any_device_work(kw):
    lib = _lib.load()
    p = params(**kw)
    buf = (C.c_double * 16)()
    conv = C.c_int(-1)
    assert lib.rewl_run_static(C.byref(p), 0, 1, buf, None, 16, C.byref(conv), None) == 1
    assert lib.rewl_run_static(None, 0, 1, buf, None, 16, C.byref(conv), None) == 1


def test_header_is_plain_c(tmp_path):
    """include/rewl.h compiles as C99 (no C++ or CUDA types cross the ABI) and a
    C program that links the library's symbols type-checks against it."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('''#include "rewl.h"
#include <stddef.h>
int main(void) {
    rewl_t h = NULL;
    int conv = 0;
    rewl_params p = {10, 8, 4, 0.75, 2, 1e-6, 0.8, 1000, 1ull};
    if (rewl_create_ext(&p, 0, &h) != REWL_OK) return 1;
    rewl_run(h, 0, &conv);
    rewl_set_allocator(NULL, NULL, NULL);
    rewl_destroy(h);
    return rewl_last_error()[0] != 0;
}
''')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-fsyntax-only", "-I",
                        os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
