"""The C ABI library loads and exports every entry point include/*.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    inc = os.path.join(ROOT, "include")
    txt = "\n".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*([a-z_][a-z_0-9]*)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2112_10059_gb300 import build as b
    return b.build()


def test_header_declares_boundary():
    names = _declared()
    for n in ("set_grid", "set_sources", "set_targets", "set_criteria", "eval_sph"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports_version(lib_path):
    import paper_2112_10059_gb300 as sph
    lib = sph.load(lib_path)
    assert lib.sph_version().startswith(b"libsph")
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_exports_match_header():
    import paper_2112_10059_gb300 as sph
    assert sorted(sph.EXPORTS) == _declared()


def test_create_without_gpu_fails_cleanly(lib_path):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    import paper_2112_10059_gb300 as sph
    lib = sph.load(lib_path)
    h = ctypes.c_void_p()
    assert lib.sph_create(ctypes.byref(h), 0, None) != 0
    assert lib.sph_destroy(None) is None
