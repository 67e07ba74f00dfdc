"""The rasterizer autotuner's cache: host-only entry points of the C ABI, run
without a GPU (store, look up, save, merge-load, reject malformed input)."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gs():
    from paper_2609_30741_gb300 import build
    build.build()
    from paper_2609_30741_gb300 import gs as gsmod
    return gsmod


KEY_A = "GB300|sm103|152sm|stereo|1600x1200:n2^19:sh3"
KEY_B = "GB300|sm103|152sm|stereo|1280x720:n2^18:sh3,2048x1536:n2^22:sh3"


def test_put_get_clear(gs):
    gs.tune_cache_clear()
    assert gs.tune_cache_size() == 0
    assert gs.tune_cache_get(KEY_A) is None
    gs.tune_cache_put(KEY_A, (16, 4, 128), 1.25)
    gs.tune_cache_put(KEY_B, (8, 2, 64), 7.5)
    assert gs.tune_cache_size() == 2
    assert gs.tune_cache_get(KEY_A) == ((16, 4, 128), 1.25)
    gs.tune_cache_put(KEY_A, (32, 8, 256), 1.0)  # replaces
    assert gs.tune_cache_get(KEY_A) == ((32, 8, 256), 1.0)
    assert gs.tune_cache_size() == 2
    gs.tune_cache_clear()
    assert gs.tune_cache_size() == 0


def test_invalid_entries_are_rejected(gs):
    gs.tune_cache_clear()
    for cfg in ((16, 3, 128), (12, 4, 128), (16, 4, 100), (8, 4, 64)):
        with pytest.raises(gs.GsError):
            gs.tune_cache_put(KEY_A, cfg, 1.0)
    for key in ("", "has space", "tab\there", "new\nline"):
        with pytest.raises(gs.GsError):
            gs.tune_cache_put(key, (16, 4, 128), 1.0)
    assert gs.tune_cache_size() == 0


def test_save_and_load_round_trip(gs, tmp_path):
    gs.tune_cache_clear()
    gs.tune_cache_put(KEY_A, (16, 2, 32), 1.5)
    gs.tune_cache_put(KEY_B, (32, 4, 256), 9.25)
    path = tmp_path / "tune.txt"
    gs.tune_cache_save(str(path))
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and all(len(ln.split()) == 5 for ln in lines)
    gs.tune_cache_clear()
    gs.tune_cache_put("other|key", (8, 1, 64), 3.0)
    gs.tune_cache_load(str(path))  # merges
    assert gs.tune_cache_size() == 3
    assert gs.tune_cache_get(KEY_A) == ((16, 2, 32), 1.5)
    assert gs.tune_cache_get(KEY_B) == ((32, 4, 256), 9.25)
    assert gs.tune_cache_get("other|key") == ((8, 1, 64), 3.0)


@pytest.mark.parametrize("bad", ["k 16 4 128", "k 16 4 128 1.0 extra", "k 16 3 128 1.0", "k sixteen 4 128 1.0"])
def test_malformed_file_changes_nothing(gs, tmp_path, bad):
    gs.tune_cache_clear()
    gs.tune_cache_put(KEY_A, (16, 4, 128), 2.0)
    path = tmp_path / "bad.txt"
    path.write_text(f"{KEY_B} 8 2 64 1.0\n{bad}\n")
    with pytest.raises(gs.GsError):
        gs.tune_cache_load(str(path))
    assert gs.tune_cache_size() == 1 and gs.tune_cache_get(KEY_B) is None
    with pytest.raises(gs.GsError):
        gs.tune_cache_load(str(tmp_path / "missing.txt"))
