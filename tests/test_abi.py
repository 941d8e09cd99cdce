"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function its header declares (no compute calls here)."""
import ctypes
import shutil

import pytest


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    from paper_2201_02460_gb300 import build, epi
    build.build()
    return epi.load()


def test_header_symbols_exported(lib):
    from paper_2201_02460_gb300 import epi
    names = epi.exported_names()
    assert "epi_search" in names and "epi_dataset_create" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_last_error_empty_and_null_args(lib):
    assert lib.epi_last_error() == b""
    # argument checks that run before any CUDA call
    h = ctypes.c_void_p()
    assert lib.epi_create(0, None, None) == 1
    assert lib.epi_dataset_create(None, None, None, 1, 1, 0, ctypes.byref(h)) == 1
    assert b"NULL" in lib.epi_last_error()
    assert lib.epi_kernel_launches(None) == 0


def test_result_record_layout():
    from paper_2201_02460_gb300 import epi
    dt = epi.RESULT_DTYPE
    assert dt.itemsize == 56
    assert dt.fields["mi"][1] == 32 and dt.fields["rank"][1] == 48


def test_product_has_no_oracle_import():
    import pathlib
    pkg = pathlib.Path(__file__).resolve().parents[1] / "paper_2201_02460_gb300"
    for p in pkg.rglob("*.py"):
        text = p.read_text()
        assert "import oracle" not in text and "from oracle" not in text, p


def _header_param_counts():
    """Parameter count of every function prototype in include/epi.h."""
    import pathlib
    import re
    text = (pathlib.Path(__file__).resolve().parents[1] / "include" / "epi.h").read_text()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    out = {}
    for m in re.finditer(r"\b(epi_[a-z0-9_]+)\s*\(([^;{}]*?)\)\s*;", text):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(lib):
    """Every function the binding declares argument types for takes as many
    arguments as its prototype in the header."""
    counts = _header_param_counts()
    assert len(counts) >= 40
    checked = 0
    for name, n in counts.items():
        fn = getattr(lib, name)
        if fn.argtypes is not None:
            assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
            checked += 1
    assert checked >= 30
