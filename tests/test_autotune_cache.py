"""The batched autotuner's cache file (host logic, no GPU): lines appended by
qsi_autotune_cache_store are found again by qsi_autotune_cache_lookup for the
same (n, b, a, precision, n_E) key, the last matching line wins, other keys
and unparsable lines are ignored, and a missing file finds nothing."""
import pytest

qsi = pytest.importorskip("paper_2601_04904_gb300.qsi")


def test_cache_round_trip_last_line_wins(tmp_path):
    path = str(tmp_path / "tune.txt")
    assert qsi.autotune_cache_lookup(path, 32, 256, 128, qsi.FP64_EMU, 256) is None  # no file yet
    qsi.autotune_cache_store(path, 32, 256, 128, qsi.FP64_EMU, 256, 64, 2, 6.0, 8.5)
    qsi.autotune_cache_store(path, 32, 256, 128, qsi.MIXED, 256, 16, 4, 2.0, 7.0)   # another precision
    qsi.autotune_cache_store(path, 32, 256, 128, qsi.FP64_EMU, 128, 32, 1, 12.0, 9.0)  # another n_E
    assert qsi.autotune_cache_lookup(path, 32, 256, 128, qsi.FP64_EMU, 256) == (64, 2, 6.0)
    with open(path, "a") as f:
        f.write("garbage line\nqsi-batched-tune 32 256 128 1 256 not numbers\n")
    qsi.autotune_cache_store(path, 32, 256, 128, qsi.FP64_EMU, 256, 128, 4, 12.0, 8.0)  # re-tuned
    assert qsi.autotune_cache_lookup(path, 32, 256, 128, qsi.FP64_EMU, 256) == (128, 4, 12.0)
    assert qsi.autotune_cache_lookup(path, 32, 256, 128, qsi.MIXED, 256) == (16, 4, 2.0)
    assert qsi.autotune_cache_lookup(path, 32, 256, 128, qsi.FP64_EMU, 128) == (32, 1, 12.0)
    assert qsi.autotune_cache_lookup(path, 16, 256, 128, qsi.FP64_EMU, 256) is None
    lines = open(path).read().splitlines()
    assert sum(ln.startswith("qsi-batched-tune ") for ln in lines) == 5


def test_cache_rejects_bad_arguments(tmp_path):
    with pytest.raises(qsi.QsiError):
        qsi.autotune_cache_store(str(tmp_path / "t.txt"), 1, 2, 3, 0, 4, 0, 0, -1.0, 1.0)  # wave < 1
    with pytest.raises(qsi.QsiError):
        qsi.autotune_cache_store(str(tmp_path / "missing_dir" / "t.txt"), 1, 2, 3, 0, 4, 8, 0, -1.0, 1.0)
