"""The C-ABI library builds, loads without a GPU and exports every entry
point declared in include/spg.h (no compute calls here)."""
import ctypes
import os
import re

from paper_1905_13408_gb300 import spg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "spg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spg_[a-z_]+)\s*\(", src)))


def test_header_matches_binding_list():
    assert declared_symbols() == sorted(spg.EXPORTS)


def test_header_is_self_contained_c_and_cxx(tmp_path):
    """A C caller needs nothing but the header: it compiles as strict C99 and
    as C++17 (with extern "C" linkage), and a C program calling every entry
    point links against the library (the calls themselves are not run)."""
    import shutil
    import subprocess
    hdr = os.path.join(ROOT, "include", "spg.h")
    gcc = shutil.which("gcc")
    if gcc is None:
        import pytest
        pytest.skip("no C compiler")
    for lang, std in (("c", "-std=c99"), ("c++", "-std=c++17")):
        r = subprocess.run([gcc if lang == "c" else shutil.which("g++") or gcc, "-fsyntax-only", std, "-Wall",
                            "-Wextra", "-Werror", "-x", lang, hdr], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    lib = spg.load()
    calls = "\n".join(f"    (void)&{name};" for name in declared_symbols())
    src = tmp_path / "caller.c"
    src.write_text(f'#include "spg.h"\nint main(void)\n{{\n{calls}\n    return 0;\n}}\n')
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(tmp_path / "caller"), lib._name], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_symbol():
    lib = spg.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_create_without_gpu_fails_cleanly():
    """No CUDA device here: creation must fail with a status, not fall back."""
    import torch
    if torch.cuda.is_available():
        return
    lib = spg.load()
    p = spg.volume_params((8, 8, 8))
    h = ctypes.c_void_p()
    st = lib.spg_create(ctypes.byref(p), None, None, ctypes.byref(h))
    assert st == spg.SPG_ECUDA
    assert not h.value
    assert "CUDA" in spg.spg_last_error(None) or "device" in spg.spg_last_error(None)


def test_bad_arguments_rejected_before_device_use():
    lib = spg.load()
    h = ctypes.c_void_p()
    bad = spg.volume_params((0, 8, 8))
    assert lib.spg_create(ctypes.byref(bad), None, None, ctypes.byref(h)) == spg.SPG_EINVAL
    neg = spg.volume_params((8, 8, 8), mu=-1.0)
    assert lib.spg_create(ctypes.byref(neg), None, None, ctypes.byref(h)) == spg.SPG_EINVAL
    assert lib.spg_reweight(None) == spg.SPG_EINVAL
    assert lib.spg_iterate(None, 3) == spg.SPG_EINVAL


def test_grid_bad_arguments_rejected_before_device_use():
    lib = spg.load()
    g = ctypes.c_void_p()
    assert lib.spg_grid_create(15, 0, 2.0, None, ctypes.byref(g)) == spg.SPG_EINVAL  # odd n
    assert not g.value
    assert b"even n" in lib.spg_grid_last_error(None)
    assert lib.spg_grid_create(16, 2, 2.0, None, ctypes.byref(g)) == spg.SPG_EINVAL  # no kernel 2
    assert lib.spg_grid_create(16, 0, 0.0, None, ctypes.byref(g)) == spg.SPG_EINVAL  # h = 0
    assert lib.spg_grid_add(None, 1, None, None, None, None) == spg.SPG_EINVAL
    assert lib.spg_grid_finish(None, None, None) == spg.SPG_EINVAL
    assert lib.spg_grid_count(None) == 0
    lib.spg_grid_destroy(None)


def test_every_handle_entry_point_rejects_a_null_handle():
    """Each entry point that takes a context or accumulator handle returns
    SPG_EINVAL for a null one (or, for the void, count and message calls,
    returns without touching it), before any device work; run in a child
    process so that a crash would show as a failure here."""
    import subprocess
    import sys
    code = r'''
import ctypes
from paper_1905_13408_gb300 import spg
lib = spg.load()
bad = []
for name in spg.EXPORTS:
    f = getattr(lib, name)
    if not f.argtypes or f.argtypes[0] is not ctypes.c_void_p:
        continue
    args = [None if t in (ctypes.c_void_p,) or isinstance(t, type) and issubclass(t, ctypes._Pointer) else 0
            for t in f.argtypes]
    r = f(*args)
    if f.restype is ctypes.c_int and r != spg.SPG_EINVAL:
        bad.append((name, r))
print("BAD", bad)
'''
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "BAD []" in r.stdout, r.stdout
