"""Host logic of the autotuner record: the tuning file round trip and its
checks (no GPU: ttv_tune_load/save/count/clear touch no device)."""
import pytest

import paper_2510_01495_gb300 as ttv


@pytest.fixture()
def clean():
    ttv.tune_clear()
    yield
    ttv.tune_clear()


def records(path):
    lines = open(path).read().split("\n")
    assert lines[0] == "ttv-tune 2"
    out = {}
    for ln in lines[1:]:
        if ln.strip():
            k, p, c, it, ms = ln.split()
            out[int(k, 16)] = (int(p), int(c), int(it), float(ms))
    return out


def test_roundtrip_and_merge(tmp_path, clean):
    f = tmp_path / "a.tune"
    f.write_text("ttv-tune 2\n0000000001020304 2 8 0 1.5\n00000000000a0b03 3 4 2 0.25\n")
    ttv.tune_load(str(f))
    assert ttv.tune_count() == 2
    g = tmp_path / "b.tune"
    ttv.tune_save(str(g))
    assert records(g) == {0x01020304: (2, 8, 0, 1.5), 0x000a0b03: (3, 4, 2, 0.25)}
    # loading again merges: same classes replaced, new ones added
    f.write_text("ttv-tune 2\n0000000001020304 1 2 1 0.5\n0000000000000042 4 0 0 9\n")
    ttv.tune_load(str(f))
    assert ttv.tune_count() == 3
    ttv.tune_save(str(g))
    assert records(g)[0x01020304] == (1, 2, 1, 0.5)
    ttv.tune_clear()
    assert ttv.tune_count() == 0


@pytest.mark.parametrize("text", [
    "not-a-tune 2\n",
    "ttv-tune 1\n0000000001020304 2 8 1.5\n",            # the old format
    "ttv-tune 2\n0000000001020304 9 8 0 1.5\n",        # no such path
    "ttv-tune 2\n0000000001020304 0 8 0 1.5\n",        # AUTO is not a plan
    "ttv-tune 2\n0000000001020304 2 8 -1 1.5\n",       # bad items per thread
    "ttv-tune 2\n0000000001020304 2 8 0 1.5\nzz 2\n",  # malformed line
])
def test_rejects_bad_files(tmp_path, clean, text):
    f = tmp_path / "bad.tune"
    f.write_text(text)
    with pytest.raises(ttv.TTVError) as e:
        ttv.tune_load(str(f))
    assert e.value.name == "TTV_ERR_ARG"
    assert ttv.tune_count() == 0          # nothing merged from a bad file


def test_missing_file(tmp_path, clean):
    with pytest.raises(ttv.TTVError):
        ttv.tune_load(str(tmp_path / "absent.tune"))
    with pytest.raises(ttv.TTVError):
        ttv.tune_save(str(tmp_path / "no_dir" / "x.tune"))
