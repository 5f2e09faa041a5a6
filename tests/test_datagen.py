"""The seeded generator: scalar regeneration of single rows, prefix property,
ranges, and the torch implementation bit-identical to the numpy one."""
import numpy as np
import pytest

from paper_1709_00700_gb300 import datagen


def test_rows_regenerate_one_by_one_and_prefixes_agree():
    s = datagen.u64_stream(5, 7, 1000)
    for r in (0, 1, 517, 999):
        assert int(s[r]) == datagen.u64_at(5, 7, r)
    assert np.array_equal(datagen.u64_stream(5, 7, 300, start=200), s[200:500])
    t = datagen.table_filter_agg(5000, 3)
    assert np.array_equal(datagen.table_filter_agg(2000, 3)["price"], t["price"][:2000])


def test_ranges():
    v = datagen.uniform_int(1, 2, 100_000, -3, 4)
    assert v.min() == -3 and v.max() == 3
    li = datagen.table_lowcard_groups(10_000)
    assert li["disc"].min() == 0 and li["disc"].max() == 10 and li["tax"].max() == 8
    assert set(np.unique(li["k1"])) == {65, 66}
    z = datagen.zipf_keys(1, 3, 50_000, 1000)
    assert z.min() >= 0 and z.max() < 1000
    # Zipf s=1: the hottest key holds about 1 / H_1000 ~ 13% of the rows
    assert 0.10 < np.bincount(z).max() / len(z) < 0.17


@pytest.mark.parametrize("lo,hi", [(0, 100), (100, 10_000_000), (-7, 3), (0, 1)])
def test_torch_uniform_is_bit_identical(lo, hi):
    torch = pytest.importorskip("torch")
    a = datagen.uniform_int(9, 11, 20_000, lo, hi, np.int64, start=123)
    b = datagen.uniform_int_torch(9, 11, 20_000, lo, hi, torch.int64, start=123).numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("g", [1, 10, 1000, 100_000])
def test_torch_zipf_is_bit_identical(g):
    pytest.importorskip("torch")
    a = datagen.zipf_keys(4, 302, 30_000, g)
    b = datagen.zipf_keys_torch(4, 302, 30_000, g).numpy()
    assert np.array_equal(a, b)
