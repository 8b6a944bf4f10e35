"""The stencil autotuner's choices as JSON text (hc_autotune_export /
hc_autotune_import): host code only, so these run without a GPU.

The tuner's table is process-wide; the shapes here are ones no other test
uses, so the entries kept by these tests change no other test's launches.
"""
import ctypes
import json

import pytest


@pytest.fixture(scope="module")
def hc():
    from paper_2603_25206_gb300 import build as b

    b.build()
    from paper_2603_25206_gb300 import hc as mod

    mod.lib()
    return mod


def _entry(**kw):
    e = {"n0": 3, "n1": 5, "n2": 7777, "wmax": 31, "op": "laplacian", "out": "int64", "tile_rows": 4, "waves": 2}
    e.update(kw)
    return e


def _text(entries, **top):
    d = {"format": "hc-autotune", "version": 1, "entries": entries}
    d.update(top)
    return json.dumps(d)


def _kept(hc):
    return json.loads(hc.autotune_export())["entries"]


def test_import_then_export_round_trip(hc):
    es = [_entry(), _entry(n0=4, op="multi", out="float64", tile_rows=1, waves=1),
          _entry(n0=5, op="gradmag", out="float32", tile_rows=255), _entry(n0=6, op="derivative", wmax=0)]
    assert hc.autotune_import(_text(es)) == 4
    kept = _kept(hc)
    for e in es:
        assert e in kept
    # the export reads back to the same table, byte for byte
    t = hc.autotune_export()
    assert hc.autotune_import(t) == len(kept)
    assert hc.autotune_export() == t


def test_import_replaces_a_kept_choice(hc):
    assert hc.autotune_import(_text([_entry(n0=7, tile_rows=8, waves=1)])) == 1
    assert hc.autotune_import(_text([_entry(n0=7, tile_rows=2, waves=2)])) == 1
    mine = [e for e in _kept(hc) if e["n0"] == 7 and e["n2"] == 7777]
    assert mine == [_entry(n0=7, tile_rows=2, waves=2)]


def test_whitespace_and_key_order(hc):
    t = ('\n { "entries" : [ { "waves":1 ,"tile_rows" : 16, "out":"float32", "op":"multi", "wmax": 3,\n'
         '"n2": 7777, "n1":5, "n0" : 8 } ] ,\t"version":1, "format" :"hc-autotune" }\n')
    assert hc.autotune_import(t) == 1
    assert _entry(n0=8, wmax=3, op="multi", out="float32", tile_rows=16, waves=1) in _kept(hc)
    assert hc.autotune_import(_text([])) == 0


BAD = [
    ("not json", "hello"),
    ("format", _text([_entry()], format="other")),
    ("version", _text([_entry()], version=2)),
    ("unknown top key", _text([_entry()], extra=1)),
    ("trailing", _text([_entry()]) + " x"),
    ("missing key", _text([{k: v for k, v in _entry().items() if k != "waves"}])),
    ("unknown key", _text([dict(_entry(), speed=3)])),
    ("op name", _text([_entry(op="mean")])),
    ("out name", _text([_entry(out="int32")])),
    ("tile rows 0", _text([_entry(tile_rows=0)])),
    ("tile rows 256", _text([_entry(tile_rows=256)])),
    ("waves 3", _text([_entry(waves=3)])),
    ("dimension 0", _text([_entry(n1=0)])),
    ("dimension above 2^40", _text([_entry(n0=(1 << 40) + 1)])),
    ("wmax 33", _text([_entry(wmax=33)])),
    ("negative", _text([_entry(n0=-3)])),
    ("fraction", _text([_entry()]).replace('"tile_rows": 4', '"tile_rows": 4.5')),
    ("string escape", _text([_entry()]).replace('"laplacian"', '"lap\\u0061cian"')),
    ("integer gradient magnitude", _text([_entry(op="gradmag", out="int64")])),
    ("integer one-pass kernel", _text([_entry(op="multi", out="int64")])),
    ("one bad entry among good ones", _text([_entry(n0=9), _entry(n0=10, waves=0)])),
]


@pytest.mark.parametrize("name,text", BAD, ids=[b[0] for b in BAD])
def test_malformed_text_keeps_nothing(hc, name, text):
    before = hc.autotune_export()
    L = hc.lib()
    count = ctypes.c_int(-1)
    assert L.hc_autotune_import(text.encode(), ctypes.byref(count)) == hc.HC_ERR_INVALID_ARG
    assert count.value == 0
    assert hc.autotune_export() == before


def test_export_size_query_and_small_buffer(hc):
    L = hc.lib()
    n = ctypes.c_size_t()
    assert L.hc_autotune_export(None, 0, ctypes.byref(n)) == hc.HC_OK
    assert n.value == len(hc.autotune_export())
    small = ctypes.create_string_buffer(n.value)  # no room for the NUL
    assert L.hc_autotune_export(small, n.value, ctypes.byref(n)) == hc.HC_ERR_NOMEM
    assert L.hc_autotune_export(None, 0, None) == hc.HC_ERR_INVALID_ARG
    assert L.hc_autotune_import(None, ctypes.byref(ctypes.c_int())) == hc.HC_ERR_INVALID_ARG
    assert L.hc_autotune_import(b"{}", None) == hc.HC_ERR_INVALID_ARG


def test_save_and_load_a_file(hc, tmp_path):
    assert hc.autotune_import(_text([_entry(n0=11, tile_rows=2)])) == 1
    p = tmp_path / "tune.json"
    hc.save_autotune(p)
    saved = json.loads(p.read_text())
    assert saved["format"] == "hc-autotune" and _entry(n0=11, tile_rows=2) in saved["entries"]
    assert hc.load_autotune(p) == len(saved["entries"])


def test_any_valid_table_round_trips(hc):
    """Drawn tables of valid entries read back as the same entries."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    entry = st.fixed_dictionaries({
        "n0": st.integers(1, 1 << 40), "n1": st.integers(1, 1 << 40), "n2": st.integers(100000, 1 << 40),
        "wmax": st.integers(0, 32), "op": st.sampled_from(["derivative", "laplacian"]),
        "out": st.sampled_from(["float32", "float64", "int64"]), "tile_rows": st.integers(1, 255),
        "waves": st.integers(1, 2)})

    @hyp.settings(max_examples=60, deadline=None)
    @hyp.given(st.lists(entry, max_size=6))
    def check(es):
        assert hc.autotune_import(_text(es)) == len(es)
        kept = _kept(hc)
        for e in es:
            key = {k: e[k] for k in ("n0", "n1", "n2", "wmax", "op", "out")}
            mine = [k for k in kept if {x: k[x] for x in key} == key]
            # a later entry of the same key replaces an earlier one
            last = [x for x in es if {k: x[k] for k in key} == key][-1]
            assert mine == [last]

    check()
