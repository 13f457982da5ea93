"""Autotuner bookkeeping on the host (no GPU needed): manual choices, the text file round trip,
and the rejection of malformed files (nothing applied)."""
import pytest


def _xl():
    from paper_2310_08408_gb300 import build, xl
    build.build()
    xl.load()
    return xl


def test_set_get_save_load_roundtrip(tmp_path):
    xl = _xl()
    xl.tune_clear()
    assert xl.tune_get(xl.TUNE_RS_PASS1, 4096, xl.C64) == 0
    xl.tune_set(xl.TUNE_RS_PASS1, 4096, xl.C64, 1)
    xl.tune_set(xl.TUNE_CZT_ADJ_Y, 2048, xl.C128, 2)
    xl.tune_set(xl.TUNE_RS_PASS3, 512, xl.C64, 2)  # recorded, but short rows run the default
    assert xl.tune_get(xl.TUNE_RS_PASS1, 4096, xl.C64) == 1
    assert xl.tune_get(xl.TUNE_CZT_ADJ_Y, 2048, xl.C128) == 2
    assert xl.tune_get(xl.TUNE_RS_PASS3, 512, xl.C64) == 0
    assert xl.tune_get(17, 4096, xl.C64) == -1
    path = tmp_path / "tune.txt"
    xl.tune_save(str(path))
    text = path.read_text()
    assert "rs_pass1 4096 c64 1" in text and "czt_adj_y 2048 c128 2" in text
    xl.tune_clear()
    assert xl.tune_get(xl.TUNE_RS_PASS1, 4096, xl.C64) == 0
    xl.tune_load(str(path))
    assert xl.tune_get(xl.TUNE_RS_PASS1, 4096, xl.C64) == 1
    assert xl.tune_get(xl.TUNE_CZT_ADJ_Y, 2048, xl.C128) == 2
    xl.tune_clear()


@pytest.mark.parametrize("bad", ["rs_pass1 4096 c64\n", "nope 4096 c64 1 3.0\n",
                                 "rs_pass1 4000 c64 1 3.0\n", "rs_pass1 4096 c32 1 3.0\n",
                                 "rs_pass1 4096 c64 3 3.0\n"])
def test_malformed_file_applies_nothing(tmp_path, bad):
    xl = _xl()
    xl.tune_clear()
    path = tmp_path / "bad.txt"
    path.write_text("# header\nczt_fwd_x 4096 c64 2 10.0\n" + bad)
    with pytest.raises(xl.XLError):
        xl.tune_load(str(path))
    assert xl.tune_get(xl.TUNE_CZT_FWD_X, 4096, xl.C64) == 0


def test_set_rejects_bad_arguments():
    xl = _xl()
    for args in [(9, 4096, 0, 1), (0, 3000, 0, 1), (0, 4096, 5, 1), (0, 4096, 0, 3)]:
        with pytest.raises(xl.XLError):
            xl.tune_set(*args)
