"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry
point that include/msc.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "msc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(msc_[a-z_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2409_17346_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("msc_prepare_original", "msc_fix", "msc_verify", "msc_apply_edits", "msc_fix_batch",
                     "msc_destroy", "msc_free_edits"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    """Calls that touch no device: version, status names, default options."""
    lib.msc_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.msc_version()
    lib.msc_status_string.restype = ctypes.c_char_p
    assert lib.msc_status_string(6) == b"MSC_ERR_STALLED"
    from paper_2409_17346_gb300 import msc
    o = msc.Options()
    lib.msc_default_options(ctypes.byref(o))
    assert (o.tier, o.q_max, o.max_iters, o.exact_fallback) == (4, 6, 100000, 1)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2409_17346_gb300 import build, msc
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(msc, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        msc.load()
