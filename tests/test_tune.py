"""Launch-shape autotuner table (host side, no GPU): op list, size buckets,
set/get, save/load round trip and rejection of malformed tables."""
import pytest

from paper_2411_17164_gb300 import build


@pytest.fixture(scope="module")
def X():
    build.build()
    from paper_2411_17164_gb300 import xmgn
    xmgn.tune_clear()
    yield xmgn
    xmgn.tune_clear()


def test_ops_and_candidates(X):
    ops = X.tune_ops()
    assert ops == {"edge_fwd_order": (0, 2), "edge_bwd_order": (1, 2), "seg_sums": (2, 4), "tn_grid": (3, 2),
                   "edge_bwd_tiles": (4, 3)}
    assert X.lib().xmgn_tune_op_name(5) is None
    assert X.lib().xmgn_tune_candidates(-1) == 0
    assert X.tune_get(7, 100) == -1


def test_choice_is_kept_per_size_bucket(X):
    X.tune_clear()
    X.tune_set(2, 1000, 3)            # bucket = bit length of 1000 = 10, rows 512..1023
    assert X.tune_get(2, 512) == 3 and X.tune_get(2, 1023) == 3
    assert X.tune_get(2, 511) == 0 and X.tune_get(2, 1024) == 0  # other buckets: untuned
    assert X.tune_get(1, 1000) == 0   # other op
    X.tune_clear()
    assert X.tune_get(2, 1000) == 0


def test_set_rejects_out_of_range(X):
    with pytest.raises(X.XmgnError):
        X.tune_set(0, 100, 2)   # op 0 has two candidates
    with pytest.raises(X.XmgnError):
        X.tune_set(9, 100, 0)
    with pytest.raises(X.XmgnError):
        X.tune_set(0, 0, 0)


def test_save_load_round_trip(X, tmp_path):
    X.tune_clear()
    X.tune_set(0, 1_411_222, 1)
    X.tune_set(2, 200_000, 2)
    X.tune_set(3, 200_000, 1)
    f = tmp_path / "tune.txt"
    X.tune_save(str(f))
    lines = f.read_text().splitlines()
    assert lines[0] == "xmgn-tune 1"
    assert sorted(lines[1:]) == sorted(["edge_fwd_order 21 1", "seg_sums 18 2", "tn_grid 18 1"])
    X.tune_clear()
    assert X.tune_get(0, 1_411_222) == 0
    X.tune_load(str(f))
    assert X.tune_get(0, 1_411_222) == 1 and X.tune_get(2, 200_000) == 2 and X.tune_get(3, 200_000) == 1


@pytest.mark.parametrize("text", ["not a table\n", "xmgn-tune 1\nbogus_op 3 1\n", "xmgn-tune 1\nseg_sums 3 4\n",
                                  "xmgn-tune 1\ntn_grid 70 0\n", "xmgn-tune 2\n", "xmgn-tune 1\nseg_sums x 1\n"])
def test_load_rejects_malformed_tables_unchanged(X, tmp_path, text):
    X.tune_clear()
    X.tune_set(1, 5000, 1)
    f = tmp_path / "bad.txt"
    f.write_text(text)
    with pytest.raises(X.XmgnError):
        X.tune_load(str(f))
    assert X.tune_get(1, 5000) == 1 and X.tune_get(2, 5000) == 0
    with pytest.raises(X.XmgnError):
        X.tune_load(str(tmp_path / "missing.txt"))
