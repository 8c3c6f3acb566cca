"""Checks of the shared seeded input generators (CPU only)."""
import math

import numpy as np
import pytest

import datagen


def test_splitmix64_published_values():
    # SplitMix64 from state 0: the first outputs of the published generator
    # (state advances by the golden gamma before mixing).
    out = datagen.splitmix64(np.array([0, 0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_counter_based_and_deterministic():
    a = datagen.draw(5, 3, 0, 1000)
    b = datagen.draw(5, 3, 400, 100)
    assert np.array_equal(a[400:500], b)
    assert not np.array_equal(datagen.draw(6, 3, 0, 10), a[:10])
    t1 = datagen.fact_table(10000, seed=1)
    t2 = datagen.fact_table(10000, seed=1)
    for k in t1:
        assert np.array_equal(t1[k], t2[k])
    part = datagen.fact_table(100, seed=1, row0=5000)
    for k in part:
        assert np.array_equal(part[k], t1[k][5000:5100])


def test_chunked_equals_unchunked():
    n = (1 << 22) + 12345
    x = datagen.uniform_int(2, 1, n, 0, 99, np.int32)
    y = datagen.uniform_int(2, 1, 1000, 0, 99, np.int32, row0=n - 1000)
    assert np.array_equal(x[-1000:], y)


def test_column_ranges():
    t = datagen.fact_table(200000, seed=9)
    assert t["key"].min() >= 0 and t["key"].max() <= 99999
    assert t["price"].min() >= 100 and t["price"].max() <= 10_000_000
    assert set(np.unique(t["discount"])) == set(range(11))
    assert set(np.unique(t["quantity"])) == set(range(1, 51))
    assert t["date"].min() == 0 and t["date"].max() == 2556
    assert set(np.unique(t["flag"])) == {0, 1, 2}
    assert set(np.unique(t["status"])) == {0, 1}
    assert t["flag"].dtype == np.uint8 and t["price"].dtype == np.int64 and t["date"].dtype == np.int32


def test_feistel_is_a_bijection():
    for N in (1, 2, 3, 7, 100, 1000, 1500, 4097):
        y = datagen.feistel_perm(11, N, np.arange(N))
        assert sorted(y.tolist()) == list(range(N))


def test_dim_payload_groups():
    d = datagen.dim_table(15000, 1500, seed=2)
    c = np.bincount(d["payload"], minlength=1500)
    assert np.all(c == 10)
    assert np.array_equal(d["key"], np.arange(15000))


def test_zipf_frequencies():
    N, s, n = 1000, 0.5, 400_000
    r = datagen.zipf_ranks(4, datagen.COL_ZIPF, n, N, s)
    assert r.min() >= 0 and r.max() < N
    p = np.arange(1, N + 1, dtype=np.float64) ** -s
    p /= p.sum()
    c = np.bincount(r, minlength=N)
    for rank in (0, 1, 9, 99, 999):
        sd = math.sqrt(n * p[rank] * (1 - p[rank]))
        assert abs(c[rank] - n * p[rank]) < 5 * sd + 1


def test_torch_generator_matches_numpy():
    """The device generator (run here on CPU tensors) reproduces the NumPy values exactly."""
    torch = pytest.importorskip("torch")
    from datagen import torch_gen
    for row0 in (0, 12345, (1 << 40) + 7):
        a = datagen.fact_table(50_003, seed=datagen.DEFAULT_SEED + 3, row0=row0)
        b = torch_gen.fact_table(50_003, seed=datagen.DEFAULT_SEED + 3, device="cpu", row0=row0)
        for k in a:
            assert np.array_equal(a[k], b[k].numpy()), (k, row0)
    x = np.arange(1000, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    got = torch_gen.splitmix64(torch.from_numpy(x.view(np.int64).copy())).numpy().view(np.uint64)
    assert np.array_equal(got, datagen.splitmix64(x))


def test_string_column_shape_padding_and_vocabulary():
    s = datagen.string_column(5000, seed=9)
    assert s.shape == (5000, datagen.STR_WIDTH) and s.dtype == np.uint8
    vocab = set(datagen.string_vocab(9))
    for row in s[:500]:
        b = bytes(row)
        body = b.split(b"\0", 1)[0]
        assert b[len(body):] == b"\0" * (len(b) - len(body))  # right-padded with 0 only
        words = body.split(b" ")
        assert 1 <= len(words) <= 3 and all(w in vocab for w in words)
    assert np.array_equal(datagen.string_column(100, seed=9, row0=50), datagen.string_column(150, seed=9)[50:])
    cut = datagen.string_column(5000, seed=9, width=5)
    assert np.array_equal(cut, s[:, :5])
