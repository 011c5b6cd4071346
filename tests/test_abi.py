"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads
without a GPU, and exports every entry point include/talekpir.h declares; the
Python binding declares a signature for each of them.  No compute call is made."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        names |= set(re.findall(r"\b(tpir_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for must in ("tpir_db_create", "tpir_write", "tpir_read_batch", "tpir_read_batch_async",
                 "tpir_read_multi_async", "tpir_bloom_get", "tpir_serve_create",
                 "tpir_serve_submit_read", "tpir_serve_poll", "tpir_serve_stats"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2001_08250_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2001_08250_gb300 import talekpir
    bound = {name for name, _, _ in talekpir._SIGS}
    assert _declared() <= bound, sorted(_declared() - bound)


def test_library_built_for_sm103a_only():
    from paper_2001_08250_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings_without_gpu():
    from paper_2001_08250_gb300 import talekpir
    assert talekpir.strerror(talekpir.EFULL).startswith("cuckoo table full")
    assert "sm_103a" in talekpir.version()


def test_invalid_arguments_rejected_before_any_device_work():
    from paper_2001_08250_gb300 import talekpir
    L = talekpir.lib()
    assert L.tpir_db_create(0, 4, 1024) is None
    assert L.tpir_last_error() == talekpir.EINVAL
    assert L.tpir_db_create(16, 4, 1000) is None   # msg_bytes not a multiple of 16
    assert L.tpir_db_create(16, 0, 1024) is None
    assert L.tpir_read_batch(None, None, 1, None) == talekpir.EINVAL
    assert L.tpir_read_multi_async(None, 200, None) == talekpir.EINVAL


def test_tuned_plans_round_trip_through_json(tmp_path):
    from paper_2001_08250_gb300 import talekpir
    good = tmp_path / "plans.json"
    good.write_text(
        '{"plans": [\n'
        '{"row_words": 1024, "batch_class": 8, "lw_log2": 5, "warps_b": 8, "warps_w": 1, "warps_k": 1, "stage_rows_log2": 3},\n'
        '{"row_words": 128, "batch_class": 5, "lw_log2": 3, "warps_b": 1, "warps_w": 1, "warps_k": 8, "stage_rows_log2": 4}\n'
        ']}\n')
    talekpir.tune_clear()
    talekpir.tune_load(str(good))
    out = tmp_path / "out.json"
    talekpir.tune_save(str(out))
    text = out.read_text()
    assert '"row_words": 1024, "batch_class": 8, "lw_log2": 5, "warps_b": 8' in text
    assert '"row_words": 128, "batch_class": 5, "lw_log2": 3' in text
    # shapes the kernel cannot run are refused (warps do not multiply to 8;
    # a stage larger than the ring slot)
    bad = tmp_path / "bad.json"
    bad.write_text(
        '{"plans": [\n'
        '{"row_words": 64, "batch_class": 3, "lw_log2": 5, "warps_b": 2, "warps_w": 2, "warps_k": 1, "stage_rows_log2": 0},\n'
        '{"row_words": 64, "batch_class": 4, "lw_log2": 5, "warps_b": 1, "warps_w": 8, "warps_k": 1, "stage_rows_log2": 5}\n'
        ']}\n')
    import pytest
    with pytest.raises(talekpir.TpirError):
        talekpir.tune_load(str(bad))
    talekpir.tune_clear()
    empty = tmp_path / "empty.json"
    talekpir.tune_save(str(empty))
    assert '"row_words"' not in empty.read_text()


def test_kernel_plans_round_trip_and_refuse_unknown_schedules(tmp_path):
    """Kernel plans (the measured winner per table class) load and save with
    their tensor-core schedule: spans (1), items on CTA pairs (2), items on
    single CTAs (3); an unknown schedule or kernel is refused."""
    from paper_2001_08250_gb300 import talekpir
    import pytest
    good = tmp_path / "kplans.json"
    good.write_text(
        '{"plans": [\n'
        '{"row_words": 1024, "batch_class": 8, "n_class": 15, "kernel": 5, "tensor_mode": 3, '
        '"tensor_kc_rows": 16384, "tensor_loads": 0},\n'
        '{"row_words": 64, "batch_class": 6, "n_class": 12, "kernel": 5, "tensor_mode": 1, '
        '"tensor_kc_rows": 0, "tensor_loads": 1}\n'
        ']}\n')
    talekpir.tune_clear()
    try:
        talekpir.tune_load(str(good))
        out = tmp_path / "out.json"
        talekpir.tune_save(str(out))
        text = out.read_text()
        assert '"tensor_mode": 3, "tensor_kc_rows": 16384, "tensor_loads": 0' in text
        assert '"tensor_mode": 1, "tensor_kc_rows": 0, "tensor_loads": 1' in text
        for bad_plan in ('"kernel": 5, "tensor_mode": 4', '"kernel": 3, "tensor_mode": 0'):
            bad = tmp_path / "bad.json"
            bad.write_text('{"plans": [\n{"row_words": 64, "batch_class": 6, "n_class": 12, %s, '
                           '"tensor_kc_rows": 0, "tensor_loads": 0}\n]}\n' % bad_plan)
            with pytest.raises(talekpir.TpirError):
                talekpir.tune_load(str(bad))
    finally:
        talekpir.tune_clear()
