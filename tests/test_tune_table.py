"""The plan-parameter table of the autotuner (host side only: set, get,
save and load need no GPU)."""
import os

import pytest

import paper_1708_09746_gb300 as G


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1708_09746_gb300 import build
    build.build()
    G.load()


def test_defaults_and_set_get():
    na, nb = (1 << 20) + 3, 1 << 19
    t = G.gf2x_tune_get(na, nb)
    assert (t["fft_depth"], t["fft_buffers"], t["bcvt_tile_log"], t["bcvt_threads"],
            t["ms"]) == (7, 2, 11, 256, -1.0)
    G.gf2x_tune_set(na, nb, 5, 1, 12, 128, 1.25)
    t = G.gf2x_tune_get(na, nb)
    assert (t["fft_depth"], t["fft_buffers"], t["bcvt_tile_log"], t["bcvt_threads"],
            t["ms"]) == (5, 1, 12, 128, 1.25)
    # another size with the same shape (log2 N, log2 Pa, log2 Pb) shares the entry
    t2 = G.gf2x_tune_get(na + 1000, nb - 7)
    assert t2 == t


@pytest.mark.parametrize("bad", [(0, 2, 11, 256), (8, 2, 11, 256), (7, 0, 11, 256),
                                 (7, 3, 11, 256), (7, 2, 3, 256), (7, 2, 15, 256),
                                 (7, 2, 11, 16), (7, 2, 11, 100), (7, 2, 11, 544)])
def test_out_of_range_rejected(bad):
    with pytest.raises(G.GF2XError):
        G.gf2x_tune_set(1 << 12, 1 << 12, *bad)


def test_save_load_roundtrip(tmp_path):
    shapes = [((1 << 16) + 64, 1 << 10, 6, 1, 10, 512, 0.5),
              (1 << 14, 1 << 14, 4, 2, 13, 64, 0.125)]
    for na, nb, d, nbuf, tl, th, ms in shapes:
        G.gf2x_tune_set(na, nb, d, nbuf, tl, th, ms)
    path = str(tmp_path / "tune.txt")
    G.gf2x_tune_save(path)
    text = open(path).read().splitlines()
    assert text[0] == "gf2x-tune 1" and len(text) >= 3
    # overwrite, then load the file back
    for na, nb, *_ in shapes:
        G.gf2x_tune_set(na, nb, 7, 2, 11, 256)
    G.gf2x_tune_load(path)
    for na, nb, d, nbuf, tl, th, ms in shapes:
        t = G.gf2x_tune_get(na, nb)
        assert (t["fft_depth"], t["fft_buffers"], t["bcvt_tile_log"], t["bcvt_threads"]) == \
            (d, nbuf, tl, th)
        assert abs(t["ms"] - ms) < 1e-9


@pytest.mark.parametrize("content", ["", "gf2x-tune 2\n", "gf2x-tune 1\n5 3 3 7 2 11 256 1.0 x\n",
                                     "gf2x-tune 1\n5 3 3 9 2 11 256 1.0\n",
                                     "gf2x-tune 1\n5 3 3 7 11 256 1.0\n", "nonsense\n"])
def test_malformed_files_rejected(tmp_path, content):
    path = str(tmp_path / "bad.txt")
    with open(path, "w") as f:
        f.write(content)
    with pytest.raises(G.GF2XError):
        G.gf2x_tune_load(path)


def test_missing_file_rejected(tmp_path):
    with pytest.raises(G.GF2XError):
        G.gf2x_tune_load(str(tmp_path / "absent.txt"))
    assert not os.path.exists(str(tmp_path / "absent.txt"))
