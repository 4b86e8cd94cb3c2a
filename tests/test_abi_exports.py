"""The C-ABI library builds, loads and exports every entry point include/pt.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import re
from pathlib import Path

import paper_2509_23043_gb300 as pt
from paper_2509_23043_gb300 import build as B

ROOT = Path(__file__).resolve().parents[1]


def _declared():
    src = (ROOT / "include" / "pt.h").read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for core in ("pt_create_instances", "pt_load_proposals", "pt_sweep", "pt_exchange",
                 "pt_global_propose", "pt_energies", "pt_read_state", "pt_destroy"):
        assert core in names
    assert set(names) == set(pt.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(str(path))
    for name in _declared():
        assert hasattr(lib, name), name
    assert pt.lib() is not None
    assert isinstance(pt.last_error(), str)


def test_former_library_exports_every_declared_symbol():
    # the IsingFormer inference library (include/pt_former.h) builds, loads and exports its ABI
    src = re.sub(r"/\*.*?\*/", "", (ROOT / "include" / "pt_former.h").read_text(), flags=re.S)
    names = sorted(set(re.findall(r"\b(pt_former_[a-z_]+)\s*\(", src)))
    assert "pt_former_score" in names and "pt_former_sample" in names
    B.build()
    lib = ctypes.CDLL(str(B.FORMER_LIB))
    for name in names:
        assert hasattr(lib, name), name
