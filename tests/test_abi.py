"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point include/qv.h declares, and rejects
bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(qv_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_core_calls():
    names = declared_symbols()
    for required in ("qv_create", "qv_apply_1q", "qv_apply_controlled", "qv_apply_circuit",
                     "qv_expect_z", "qv_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(qvlib):
    lib = ctypes.CDLL(qvlib.LIB_PATH)
    missing = [s for s in sorted(declared_symbols()) if not hasattr(lib, s)]
    assert not missing, missing


def test_struct_layouts_match_header(qvlib):
    # qv_gate: 8 int32 + 3 double + 4 * (2 double) = 32 + 24 + 64
    assert ctypes.sizeof(qvlib.qv_gate) == 120
    assert ctypes.sizeof(qvlib.qv_plan_opts) == 32
    assert ctypes.sizeof(qvlib.qv_pauli_term) == 24
    # qv_tc_stage: 40 int32 + 2 * 256 complex128
    assert ctypes.sizeof(qvlib.qv_tc_stage) == 160 + 2 * 256 * 16
    assert ctypes.sizeof(qvlib.qv_kernel_stat) == 24


def test_bad_arguments_rejected_without_device(qvlib):
    with pytest.raises(qvlib.QvError) as e:
        qvlib.qv_create(0)
    assert e.value.status == qvlib.QV_ERR_ARG and "outside" in str(e.value)
    with pytest.raises(qvlib.QvError) as e:
        qvlib.qv_create(41)
    assert e.value.status == qvlib.QV_ERR_ARG
    with pytest.raises(qvlib.QvError) as e:
        qvlib.qv_create(4, dtype=7)
    assert e.value.status == qvlib.QV_ERR_ARG
    with pytest.raises(qvlib.QvError) as e:
        qvlib.qv_wrap(0, 4)
    assert e.value.status == qvlib.QV_ERR_ARG
    with pytest.raises(qvlib.QvError) as e:
        qvlib.qv_wrap(8, 4)            # not 16-byte aligned
    assert e.value.status == qvlib.QV_ERR_ARG
    # NULL handle
    r = qvlib.lib.qv_set_basis(None, 0)
    assert r == qvlib.QV_ERR_ARG and "NULL" in qvlib.qv_last_error()
    assert qvlib.lib.qv_destroy(None) == qvlib.QV_OK
    # one-shot batch: no items, or a NULL state, is refused before any device work
    assert qvlib.lib.qv_apply_batch(None, 1, None, 0, None, None) == qvlib.QV_ERR_ARG
    items = (qvlib.qv_batch_item * 1)()
    assert qvlib.lib.qv_apply_batch(items, 1, None, 0, None, None) == qvlib.QV_ERR_ARG


def test_no_library_means_import_error(tmp_path, monkeypatch):
    """The binding refuses to import without libqv.so (no CPU fallback)."""
    import importlib.util
    src = os.path.join(ROOT, "paper_2508_15545_gb300", "qv.py")
    spec = importlib.util.spec_from_file_location("qv_copy", str(tmp_path / "qv.py"))
    (tmp_path / "qv.py").write_text(open(src).read())
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)
