"""The C-ABI library loads and exports every symbol include/moma.h declares (no GPU calls)."""
import os
import re
import subprocess

import pytest

from paper_2501_07535_gb300 import build, moma

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "moma.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(moma_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_expected_entry_points():
    decl = _declared()
    for name in ("moma_ctx_create", "moma_ntt_fwd", "moma_ntt_inv", "moma_vec_addmod", "moma_vec_submod",
                 "moma_vec_mulmod", "moma_vec_axpymod", "moma_polymul", "moma_status_string"):
        assert name in decl


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(moma_\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing


def test_binding_covers_header(libpath):
    assert sorted(moma.exported_symbols()) == _declared()
    L = moma.lib()  # loads without a GPU (the CUDA runtime is initialised lazily)
    for name in _declared():
        assert hasattr(L, name)


def test_status_strings(libpath):
    assert moma.moma_status_string(0) == "MOMA_OK"
    assert moma.moma_status_string(3) == "MOMA_ERR_SIZE"
    assert moma.moma_status_string(99) == "MOMA_ERR_UNKNOWN"


def _enum(name_prefix):
    """Name -> value of the header's enumerators that start with name_prefix."""
    src = open(os.path.join(ROOT, "include", "moma.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(" + name_prefix + r"\w*)\s*=\s*(\d+)", src)}


def test_binding_codes_match_header():
    """The binding's status, operation and word-block codes equal the header's enumerators."""
    status = _enum("MOMA_ERR_") | _enum("MOMA_OK")
    assert {v: k for k, v in status.items()} == {k: v for k, v in moma.STATUS.items() if v != "MOMA_ERR_UNKNOWN"}
    ops = _enum("MOMA_OP_")
    assert ops == {"MOMA_OP_" + k.upper(): v for k, v in moma.OPS.items()}
    words = _enum("MOMA_WORD_")
    assert words == {"MOMA_WORD_" + k.upper(): v for k, v in moma.WORD_OPS.items()}


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libmoma.so every call raises: there is no CPU fallback path."""
    monkeypatch.setattr(moma, "_lib", None)
    monkeypatch.setattr(moma, "LIB_PATH", str(tmp_path / "libmoma.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        moma.lib()
    with pytest.raises(RuntimeError):
        moma.moma_status_string(0)
