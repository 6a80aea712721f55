"""The split-K autotuner's table through the C ABI, on the CPU (no kernel
runs): save, load, merge, clear, and rejection of malformed files."""
import pytest

from paper_2506_04840_gb300 import api


@pytest.fixture
def lib():
    api.load()
    api.tucker_tune_clear()
    api.tucker_tune_enable(False)
    yield
    api.tucker_tune_clear()
    api.tucker_tune_enable(False)


def test_round_trip_and_merge(lib, tmp_path):
    f = tmp_path / "t.txt"
    f.write_text("tucker-tune 1\n0 1000 64 1048576 40\n1 400 20 262144 3\n")
    assert api.tucker_tune_load(f) == api.TK_OK
    assert api.tucker_tune_entries() == 2
    out = tmp_path / "o.txt"
    api.tucker_tune_save(out)
    lines = out.read_text().splitlines()
    assert lines[0] == "tucker-tune 1"
    assert sorted(lines[1:]) == sorted(["0 1000 64 1048576 40", "1 400 20 262144 3"])
    # loading merges: a new class is added, an existing one replaced
    g = tmp_path / "g.txt"
    g.write_text("tucker-tune 1\n0 1000 64 1048576 10\n0 50 16 64 1\n")
    assert api.tucker_tune_load(g) == api.TK_OK
    assert api.tucker_tune_entries() == 3
    api.tucker_tune_save(out)
    assert "0 1000 64 1048576 10" in out.read_text().splitlines()
    api.tucker_tune_clear()
    assert api.tucker_tune_entries() == 0


@pytest.mark.parametrize("text", ["", "tucker-tune 2\n", "tucker-tune 1\n0 10 4 16\n",
                                  "tucker-tune 1\n0 10 4 16 0\n", "tucker-tune 1\n0 x 4 16 2\n",
                                  "tucker-tune 1\n-1 10 4 16 2\n"])
def test_malformed_file_leaves_the_table(lib, tmp_path, text):
    good = tmp_path / "good.txt"
    good.write_text("tucker-tune 1\n0 100 16 1024 4\n")
    assert api.tucker_tune_load(good) == api.TK_OK
    bad = tmp_path / "bad.txt"
    bad.write_text(text)
    assert api.tucker_tune_load(bad) == api.TK_EINVAL
    assert api.tucker_tune_entries() == 1


def test_missing_file(lib, tmp_path):
    assert api.tucker_tune_load(tmp_path / "none.txt") == api.TK_EINVAL
