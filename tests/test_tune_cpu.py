"""Autotune cache of the library (host side, no GPU): save / load round trip,
merging, clearing and rejection of malformed files."""
import pytest

from paper_2410_01316_gb300 import QSError, tune_cache_clear, tune_cache_load, tune_cache_save, tune_cache_size


def test_cache_round_trip_and_merge(tmp_path):
    tune_cache_clear()
    assert tune_cache_size() == 0
    src = tmp_path / "tune.txt"
    src.write_text("# dbits n_ft pbits proj W spread_variant gemm_pair\n"
                   "10 1024 11 3 8 5 1\n"
                   "6 2048 12 3 8 0 -1\n")
    tune_cache_load(str(src))
    assert tune_cache_size() == 2
    # the same key again replaces its entry instead of adding one
    again = tmp_path / "again.txt"
    again.write_text("10 1024 11 3 8 4 0\n")
    tune_cache_load(str(again))
    assert tune_cache_size() == 2
    out = tmp_path / "out.txt"
    tune_cache_save(str(out))
    lines = [l for l in out.read_text().splitlines() if not l.startswith("#")]
    assert sorted(lines) == sorted(["10 1024 11 3 8 4 0", "6 2048 12 3 8 0 -1"])
    tune_cache_clear()
    assert tune_cache_size() == 0


@pytest.mark.parametrize("text", ["1 2 3\n", "10 1024 11 3 8 9 0\n", "10 1024 11 3 8 1 2\n"])
def test_malformed_cache_files_are_rejected(tmp_path, text):
    tune_cache_clear()
    f = tmp_path / "bad.txt"
    f.write_text(text)
    with pytest.raises(QSError):
        tune_cache_load(str(f))
    assert tune_cache_size() == 0
    with pytest.raises(QSError):
        tune_cache_load(str(tmp_path / "missing.txt"))
