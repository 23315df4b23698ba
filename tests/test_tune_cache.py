"""The autotuner's cache file (host logic, no GPU): save, load, replace,
reject malformed lines."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def amto():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_04240_b300 import amto as A
    return A


LINE = "amto-tune-v1 {n} 100 10 256 1 1 0 0 0 1 15 {G} {QW} 1 1 {us}\n"


def test_save_load_replace_and_reject(amto, tmp_path):
    amto.tune_cache_clear()
    assert amto.tune_cache_size() == 0
    empty = tmp_path / "empty.txt"
    amto.tune_cache_save(str(empty))
    assert empty.read_text() == ""
    f = tmp_path / "two.txt"
    f.write_text("# comment\n" + LINE.format(n=64, G=16, QW=1, us=80.5)
                 + LINE.format(n=32, G=32, QW=2, us=30.25))
    amto.tune_cache_load(str(f))
    assert amto.tune_cache_size() == 2
    # an entry of the same key replaces the earlier one
    g = tmp_path / "replace.txt"
    g.write_text(LINE.format(n=64, G=8, QW=4, us=70.0))
    amto.tune_cache_load(str(g))
    assert amto.tune_cache_size() == 2
    out = tmp_path / "out.txt"
    amto.tune_cache_save(str(out))
    lines = sorted(out.read_text().split("\n")[:-1])
    assert len(lines) == 2
    assert any(l.split()[1] == "64" and l.split()[12:14] == ["8", "4"] for l in lines)
    assert any(l.split()[1] == "32" and l.split()[12:14] == ["32", "2"] for l in lines)
    # malformed: wrong magic, a tile group of 12, too few fields
    for bad in ["amto-tune-v0 64 100 10 256 1 1 0 0 0 1 15 16 1 1 1 1.0\n",
                LINE.format(n=16, G=12, QW=1, us=1.0),
                "amto-tune-v1 64 100 10\n"]:
        b = tmp_path / "bad.txt"
        b.write_text(LINE.format(n=8, G=8, QW=1, us=1.0) + bad)
        with pytest.raises(RuntimeError):
            amto.tune_cache_load(str(b))
        assert amto.tune_cache_size() == 2   # nothing merged
    with pytest.raises(RuntimeError):
        amto.tune_cache_load(str(tmp_path / "missing.txt"))
    amto.tune_cache_clear()
    amto.tune_cache_load(str(out))
    assert amto.tune_cache_size() == 2
    amto.tune_cache_clear()
    assert amto.tune_cache_size() == 0
