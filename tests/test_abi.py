"""CPU checks of the C ABI boundary: the library builds, loads without a GPU and
exports every entry point include/bem.h declares; the binding names match."""
import ctypes
import os
import re

from paper_1901_08393_gb300 import bem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    return sorted(set(re.findall(r"^\s*(?:bem_status|const char \*)\s*(bem_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("bem_mesh_upload", "bem_assemble_V", "bem_solve_capacity", "bem_zz_estimate",
                     "bem_mark_refine"):
        assert required in names
    assert set(names) == set(bem.EXPORTS + ["bem_last_error"])


def test_library_exports_every_symbol():
    from paper_1901_08393_gb300 import build

    build.build()
    L = ctypes.CDLL(bem.LIB_PATH)
    for name in _declared():
        assert hasattr(L, name), name
    assert bem.lib() is not None


def test_no_torch_types_in_header():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    assert "torch" not in src.lower().replace("pytorch", "") and "at::" not in src


def _prototypes():
    """{name: parameter count} of every entry point declared in include/bem.h."""
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    out = {}
    for m in re.finditer(r"(?:bem_status|const char \*)\s*(bem_\w+)\s*\(([^)]*)\)\s*;", src):
        params = [p for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        out[m.group(1)] = len(params)
    return out


def test_binding_argument_counts_match_the_header():
    """The ctypes signature of every entry point has as many arguments as its C
    prototype (a changed signature cannot go unnoticed by the binding)."""
    from paper_1901_08393_gb300 import build

    build.build()
    L = bem.lib()
    protos = _prototypes()
    assert set(protos) == set(_declared())
    for name, n in protos.items():
        assert len(getattr(L, name).argtypes) == n, (name, n, len(getattr(L, name).argtypes))
