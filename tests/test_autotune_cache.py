"""The autotune cache's host side: the text file round trip, merging, and the
errors for malformed or missing files (no GPU: these calls touch no device)."""
import pytest

from paper_2107_07104_gb300 import fibers as F

GPU = "Test GPU|152 SMs|sm_103"


def _line(gpu, r_hex, hist, choice=(8, 6, 2, 3, 1), mode=0):
    h = " ".join(f"{n}:{c}" for n, c in hist)
    return f"{gpu}\t{mode} 0 0 0 3 1 {r_hex}\t{' '.join(map(str, choice))}\t{len(hist)} {h}\n"


@pytest.fixture(autouse=True)
def _empty_cache():
    F.load()
    F.fibers_autotune_cache_clear()
    yield
    F.fibers_autotune_cache_clear()


def test_load_save_round_trip(tmp_path):
    text = "fibers-autotune-cache 1\n" + _line(GPU, "0x1.d63886594af4fp-4", [(1481, 7744)]) + \
        _line(GPU, "0x1.d63886594af4fp-4", [(800, 3), (1200, 5), (2000, 1)], (12, 4, 1, 2, 1))
    src = tmp_path / "a.txt"
    src.write_text(text)
    F.fibers_autotune_cache_load(str(src))
    assert F.fibers_autotune_cache_size() == 2
    out = tmp_path / "b.txt"
    F.fibers_autotune_cache_save(str(out))
    saved = out.read_text()
    assert saved.splitlines()[0] == "fibers-autotune-cache 1"
    assert sorted(saved.splitlines()[1:]) == sorted(text.splitlines()[1:])
    F.fibers_autotune_cache_clear()
    assert F.fibers_autotune_cache_size() == 0
    F.fibers_autotune_cache_load(str(out))
    out2 = tmp_path / "c.txt"
    F.fibers_autotune_cache_save(str(out2))
    assert out2.read_text() == saved


def test_equal_keys_merge_and_distinct_keys_add(tmp_path):
    a = tmp_path / "a.txt"
    a.write_text("fibers-autotune-cache 1\n" + _line(GPU, "0x1p-3", [(100, 2)]))
    F.fibers_autotune_cache_load(str(a))
    b = tmp_path / "b.txt"
    b.write_text("fibers-autotune-cache 1\n" + _line(GPU, "0x1p-3", [(100, 2)], (16, 3, 1, 2, 1)) +
                 _line(GPU, "0x1p-3", [(100, 3)]) + _line("Other GPU|8 SMs|sm_80", "0x1p-3", [(100, 2)]) +
                 _line(GPU, "0x1p-2", [(100, 2)]) + _line(GPU, "0x1p-3", [(100, 2)], mode=1))
    F.fibers_autotune_cache_load(str(b))
    assert F.fibers_autotune_cache_size() == 5
    out = tmp_path / "out.txt"
    F.fibers_autotune_cache_save(str(out))
    assert any("\t16 3 1 2 1\t" in line for line in out.read_text().splitlines())


@pytest.mark.parametrize("body", [
    "fibers-autotune-cache 2\n",                                           # wrong header
    "fibers-autotune-cache 1\n" + _line(GPU, "0x1p-3", [(200, 1), (100, 1)]),  # lengths not ascending
    "fibers-autotune-cache 1\n" + _line(GPU, "0x1p-3", [(100, 0)]),          # empty length class
    "fibers-autotune-cache 1\n" + _line(GPU, "0x1p-3", [(100, 2)]).replace("\t1 100:2", "\t2 100:2"),  # count
    "fibers-autotune-cache 1\n" + _line(GPU, "0x1p-3", [(100, 2)]).rstrip("\n") + " junk\n",
    "fibers-autotune-cache 1\n" + "no tabs here\n",
    "",
])
def test_malformed_files_merge_nothing(tmp_path, body):
    good = tmp_path / "good.txt"
    good.write_text("fibers-autotune-cache 1\n" + _line(GPU, "0x1p-3", [(100, 2)]))
    F.fibers_autotune_cache_load(str(good))
    bad = tmp_path / "bad.txt"
    bad.write_text(body + _line(GPU, "0x1p-3", [(300, 9)]) if body.startswith("fibers-autotune-cache 1") else body)
    with pytest.raises(F.FibersError) as ei:
        F.fibers_autotune_cache_load(str(bad))
    assert ei.value.status == F.FIB_EINVAL
    assert "bad.txt" in str(ei.value)
    assert F.fibers_autotune_cache_size() == 1


def test_missing_file_and_unwritable_path(tmp_path):
    with pytest.raises(F.FibersError) as ei:
        F.fibers_autotune_cache_load(str(tmp_path / "absent.txt"))
    assert ei.value.status == F.FIB_EIO
    with pytest.raises(F.FibersError) as ei:
        F.fibers_autotune_cache_save(str(tmp_path / "no_such_dir" / "x.txt"))
    assert ei.value.status == F.FIB_EIO
