"""The C-ABI library builds, loads and exports every symbol include/coulps.h
declares; argument validation that needs no GPU rejects bad input."""
import ctypes
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _declared():
    text = (ROOT / "include" / "coulps.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(coulps_[a-z_0-9]+)\s*\(", text))
    return {n for n in names if not n.endswith("_fn")}


@pytest.fixture(scope="module")
def lib():
    from paper_1403_0711_gb300 import _build, coulps
    _build.build()
    return coulps.load()


def test_exports_match_header(lib):
    from paper_1403_0711_gb300 import coulps
    declared = _declared()
    assert declared == set(coulps.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", str(coulps.LIB_PATH)], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = declared - exported
    assert not missing, missing
    for name in declared:
        assert hasattr(lib, name)


def test_error_strings_and_version(lib):
    from paper_1403_0711_gb300 import coulps
    assert coulps.error_string(0) == "ok"
    for st in range(-8, 0):
        assert coulps.error_string(st) != "unknown status"
    assert lib.coulps_version() >= 100


def test_host_validation_without_gpu(lib):
    from paper_1403_0711_gb300 import coulps
    h = ctypes.c_void_p()
    bad = [(0, 4, 4, 1, 0), (4, 4, 4, 0, 0), (4, 4, 4, 1, 7), (513, 4, 4, 1, 0), (4, -1, 4, 1, 0)]
    for Lx, Ly, Lz, nc, prec in bad:
        assert lib.coulps_lattice_create(Lx, Ly, Lz, nc, prec, 0, None, ctypes.byref(h)) == coulps.EINVAL
        assert not h.value
    assert lib.coulps_lattice_create(4, 4, 4, 1, 0, 0, None, None) == coulps.EINVAL
    assert lib.coulps_sweep(None, 1, 1, 0) == coulps.EINVAL
    assert lib.coulps_measure(None, None) == coulps.EINVAL
    assert lib.coulps_estimate(None, None, None, None, None) == coulps.EINVAL
    assert lib.coulps_set_tile(None, 4, 4) == coulps.EINVAL
    assert lib.coulps_charges_create(None, 0, None, None, 0, ctypes.byref(h)) == coulps.EINVAL
    lib.coulps_lattice_destroy(None)
    lib.coulps_charges_destroy(None)


def test_product_path_has_no_oracle_dependency():
    # the package, its native sources and the header never import, include or
    # load anything under oracle/
    pat = re.compile(r"(^\s*(from|import)\s+oracle)|(#include[^\n]*oracle)|liborc|orc\.c",
                     re.M)
    files = list((ROOT / "paper_1403_0711_gb300").rglob("*.py")) + [
        p for p in (ROOT / "paper_1403_0711_gb300" / "csrc").glob("*") if p.is_file()] + [
        ROOT / "include" / "coulps.h"]
    for p in files:
        assert not pat.search(p.read_text()), p
