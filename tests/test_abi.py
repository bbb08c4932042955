"""The C ABI library: it builds for sm_103a, loads, and exports every entry
point that include/*.h declares.  No GPU is needed (no compute calls)."""
import ctypes
import glob
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(xg_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1108_0486_gb300 import build as B
    try:
        return B.build()
    except RuntimeError as e:  # pragma: no cover
        if "nvcc not found" in str(e):
            pytest.skip(str(e))
        raise


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("xg_create_streams", "xg_seed", "xg_generate_u32", "xg_generate_uniform",
                     "xg_generate_normal", "xg_submit", "xg_poll"):
        assert required in names, required


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1108_0486_gb300 import _lib
    missing = sorted(_declared() - set(_lib.SIGNATURES))
    assert not missing, missing


def test_library_is_built_for_sm_103a(libpath):
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    arches = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert arches == {"103a"}, arches


def test_version_string(libpath):
    lib = ctypes.CDLL(libpath)
    lib.xg_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.xg_version()


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1108_0486_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), path
    code = ("import sys; sys.path.insert(0, %r); import paper_1108_0486_gb300 as p; "
            "p._lib; p.workloads; p.build; import paper_1108_0486_gb300.api; "
            "assert 'oracle' not in sys.modules" % ROOT)
    subprocess.run([sys.executable, "-c", code], check=True)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1108_0486_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _lib.lib()


def test_public_headers_are_plain_c_and_cpp(tmp_path):
    import shutil
    for compiler, lang, std in (("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++17")):
        if not shutil.which(compiler):
            pytest.skip(f"{compiler} unavailable")
        for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
            subprocess.run([compiler, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                            "-x", lang, f"-I{ROOT}/include", h], check=True)


def test_plain_c_client_links_and_gets_host_side_errors(libpath, tmp_path):
    """A C program linked against the library: argument checks and error
    reporting work without touching a GPU."""
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("gcc unavailable")
    exe = str(tmp_path / "c_abi_check")
    libdir = os.path.dirname(libpath)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", f"-I{ROOT}/include",
                    os.path.join(ROOT, "tests", "host", "c_abi_check.c"), "-o", exe,
                    f"-L{libdir}", "-lxorgens_gb300", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
