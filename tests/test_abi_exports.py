"""The C-ABI library builds for sm_103a and exports every entry point that
include/hpclust.h declares (no GPU needed: nothing is called)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    text = (ROOT / "include" / "hpclust.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\b(hpc_[a-z_0-9]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ["hpc_draw_sample", "hpc_kmeanspp", "hpc_lloyd", "hpc_objective", "hpc_round",
              "hpc_create", "hpc_destroy", "hpc_sync_status"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2311_04517_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(str(path))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_abi():
    from paper_2311_04517_gb300 import hpclust
    for n in ["hpc_draw_sample", "hpc_kmeanspp", "hpc_lloyd", "hpc_objective", "hpc_round"]:
        assert callable(getattr(hpclust, n))


def test_library_has_no_oracle_dependency():
    # the product library links nothing from oracle/
    from paper_2311_04517_gb300 import _build
    path = _build.build()
    data = path.read_bytes()
    assert b"orc_" not in data
    src = "".join(p.read_text() for p in (ROOT / "paper_2311_04517_gb300").rglob("*.py"))
    assert "import oracle" not in src and "from oracle" not in src
