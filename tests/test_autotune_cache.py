"""The autotuner cache's file format and host calls (no GPU): entries load,
merge and save; malformed or out-of-range lines are rejected whole; missing
or unwritable files report PP_EIO.  The cache only chooses how work is
assigned to the device, so nothing here touches the values computed."""
import pytest


@pytest.fixture
def pp():
    from paper_1404_0743_gb300 import build
    build.build()
    import paper_1404_0743_gb300 as pp
    pp.autotune_cache_clear()
    yield pp
    pp.autotune_cache_clear()


def _entries(path):
    rows = {}
    for line in open(path):
        line = line.rstrip("\n")
        if line and not line.startswith("#"):
            key, vals = line.split("\t")
            rows[key] = tuple(int(v) for v in vals.split())
    return rows


GOOD = (
    "# a comment\n"
    "\n"
    "sm_103x152 midgame parity=-1 max_empty=12 boards=12:1024,\t3 0 0 0 0\n"
    "sm_103x152 slice=34 d4=0 sections=4940 boards=1 h=0123456789abcdef\t2 0 0 1 0\r\n"
)


def test_load_save_round_trip(pp, tmp_path):
    src = tmp_path / "a.txt"
    src.write_text(GOOD)
    assert pp.autotune_cache_load(src) == 2
    assert pp.autotune_cache_stats() == (2, 0, 0)
    dst = tmp_path / "b.txt"
    pp.autotune_cache_save(dst)
    assert _entries(dst) == {
        "sm_103x152 midgame parity=-1 max_empty=12 boards=12:1024,": (3, 0, 0, 0, 0),
        "sm_103x152 slice=34 d4=0 sections=4940 boards=1 h=0123456789abcdef": (2, 0, 0, 1, 0),
    }
    pp.autotune_cache_clear()
    assert pp.autotune_cache_stats() == (0, 0, 0)
    assert pp.autotune_cache_load(dst) == 2
    assert not list(tmp_path.glob("*.tmp.*"))  # the temporary file was renamed away


def test_later_entries_replace(pp, tmp_path):
    a, b = tmp_path / "a.txt", tmp_path / "b.txt"
    a.write_text("k1\t1 0 0 0 0\nk2\t2 0 0 0 0\n")
    b.write_text("k2\t1 256 2 0 1\nk3\t3 0 0 0 0\n")
    pp.autotune_cache_load(a)
    pp.autotune_cache_load(b)
    out = tmp_path / "c.txt"
    pp.autotune_cache_save(out)
    assert _entries(out) == {"k1": (1, 0, 0, 0, 0), "k2": (1, 256, 2, 0, 1), "k3": (3, 0, 0, 0, 0)}


@pytest.mark.parametrize("bad", [
    "no tab here 1 0 0 0 0\n",     # key and options not separated by a tab
    "\t1 0 0 0 0\n",               # empty key
    "k\t1 0 0 0\n",                # four fields
    "k\t1 0 0 0 0 7\n",            # six fields
    "k\t4 0 0 0 0\n",              # unknown mode
    "k\t1 128 0 0 0\n",            # threads_per_block other than 0 or 256
    "k\t1 0 33 0 0\n",             # ctas_per_sm out of range
    "k\t1 0 0 3 0\n",              # stage_children out of range
    "k\t1 0 0 0 2\n",              # largest_first not 0 or 1
    "k\t1 0 x 0 0\n",              # not a number
    "k" * 2000 + "\t1 0 0 0 0\n",  # longer than a line may be
])
def test_malformed_file_merges_nothing(pp, tmp_path, bad):
    f = tmp_path / "bad.txt"
    f.write_text("good\t1 0 0 0 0\n" + bad)
    with pytest.raises(pp.PentagoError) as e:
        pp.autotune_cache_load(f)
    assert e.value.code == 1
    assert pp.autotune_cache_stats()[0] == 0


def test_missing_and_unwritable_files(pp, tmp_path):
    with pytest.raises(pp.PentagoError) as e:
        pp.autotune_cache_load(tmp_path / "absent.txt")
    assert e.value.code == 6
    with pytest.raises(pp.PentagoError) as e:
        pp.autotune_cache_save(tmp_path / "no_such_dir" / "c.txt")
    assert e.value.code == 6
