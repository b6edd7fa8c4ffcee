"""The work-split tuning table and its JSON file (host side; no GPU needed)."""
import pytest


@pytest.fixture(scope="module")
def api():
    from paper_1905_10587_gb300 import build
    build()
    from paper_1905_10587_gb300 import api as a
    return a


def test_tune_table_round_trips_through_json(api, tmp_path):
    api.tune_clear()
    api.tune_set("form=1 w=64 r=16 lg=16", 5, 1, 6.5)
    api.tune_set("form=0 w=8 r=1 lg=16", 3, 0, 3.75)
    f = tmp_path / "tune.json"
    api.tune_save(f)
    text = f.read_text()
    assert text.startswith('{"krr_tune": 1') and text.count('"key"') == 2
    api.tune_clear()
    assert api.tune_get("form=1 w=64 r=16 lg=16") is None
    api.tune_load(f)
    assert api.tune_get("form=1 w=64 r=16 lg=16") == (5, 1, 6.5)
    assert api.tune_get("form=0 w=8 r=1 lg=16") == (3, 0, 3.75)
    api.tune_clear()


def test_tune_load_rejects_bad_files_and_adds_nothing(api, tmp_path):
    from paper_1905_10587_gb300.api import KRRError
    api.tune_clear()
    bad = tmp_path / "bad.json"
    bad.write_text('{"krr_tune": 1, "entries": [\n {"key": "form=1 w=64 r=8 lg=10", "splits": 2, "pv": 1, "ms": 1},\n'
                   ' {"key": "form=1 w=64 r=8 lg=11", "splits": -3, "pv": 1, "ms": 1}\n]}\n')
    with pytest.raises(KRRError):
        api.tune_load(bad)
    assert api.tune_get("form=1 w=64 r=8 lg=10") is None
    with pytest.raises(KRRError):
        api.tune_load(tmp_path / "missing.json")
    nohdr = tmp_path / "nohdr.json"
    nohdr.write_text('{"key": "form=1 w=64 r=8 lg=10", "splits": 2, "pv": 1, "ms": 1}\n')
    with pytest.raises(KRRError):
        api.tune_load(nohdr)
    with pytest.raises(KRRError):
        api.tune_set("form=1 w=64 r=8 lg=10", 2, 3, 0.0)   # pv must be 0 or 1


def test_autotune_option_is_validated(api):
    from paper_1905_10587_gb300 import _lib
    import ctypes as C
    lib = _lib.load()
    o = _lib.KrrOpts()
    lib.krr_default_opts(C.byref(o))
    assert o.autotune == 0 and o.tc_pv == 1
