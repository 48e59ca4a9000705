"""Host-side logic that needs no GPU: the autotuner's choice among timed shapes, the keys of the
stored launch tables, and the seeded input generators."""
import numpy as np

from paper_0707_0438_gb300 import abi, autotune, workloads


def test_pick_prefers_fewer_splits_within_the_tie():
    timed = [(1 << 20, 2, 24, 1.1024), (1 << 20, 2, 16, 1.1030), (1 << 20, 4, 8, 1.1200), (1 << 20, 1, 12, 1.1040)]
    # 2 x 16 is within 0.5% of the fastest and has fewer splits than 2 x 24; 1 x 12 has fewer still
    assert autotune._pick(timed)[1:3] == (1, 12)
    assert autotune._pick(timed, tie=0.0)[1:3] == (2, 24)
    # only the shapes within the tie compete: 4 x 8 is 1.6% slower
    assert autotune._pick(timed[:3])[1:3] == (2, 16)
    # equal splits: fewer groups, then time
    assert autotune._pick([(8, 8, 4, 1.0), (8, 2, 4, 1.001)])[1:3] == (2, 4)


def test_pick_batch_prefers_whole_clusters_within_the_tie():
    timed = [(1, 0, 1.004), (2, 0, 1.010), (1, 32, 1.000), (4, 16, 0.990), (2, 64, 0.994)]
    # 4 x 16 is the fastest; 2 x 64 is within 0.5% and splits less; whole clusters are 1.4% slower
    assert autotune._pick_batch(timed)[:2] == (2, 64)
    assert autotune._pick_batch(timed, tie=0.0)[:2] == (4, 16)
    # whole clusters win whenever they are within the tie, then fewer groups
    assert autotune._pick_batch(timed, tie=0.02)[:2] == (1, 0)
    assert autotune._pick_batch([(4, 0, 1.0), (1, 0, 1.001)])[:2] == (1, 0)
    assert set(autotune.BATCH_CANDIDATES) >= {(1, 0), (2, 0), (4, 0)}


def test_table_keys_per_call_kind():
    assert autotune._key("NVIDIA GB300", "mixed", 65536) == "NVIDIA GB300|mixed|65536"
    assert autotune._key("NVIDIA GB300", "mixed", 16384, "acc_pot") == "NVIDIA GB300|mixed|16384|acc_pot"
    assert set(abi.CALL_KINDS) == {"forces", "acc_pot", "adjoint"}
    assert abi.CALL_KINDS["forces"] == abi.KIRIN_CALL_FORCES == 0
    # the packaged tables are keyed this way and every entry is a valid shape
    import json
    data = json.load(open(autotune.PACKAGED))
    for key, entries in data.items():
        assert key.count("|") in (2, 3)
        n_j = int(key.split("|")[2])
        assert all(a[0] < b[0] for a, b in zip(entries, entries[1:]))
        assert entries[-1][0] == n_j
        for n_i, groups, n_split, seconds in entries:
            assert groups in (1, 2, 4, 8) and 1 <= n_split <= 1024 and seconds > 0


def test_gaussian_cloud_is_seeded():
    a = workloads.gaussian_cloud(1000, 7, eps=1e-3)
    b = workloads.gaussian_cloud(1000, 7, eps=1e-3)
    c = workloads.gaussian_cloud(1000, 8, eps=1e-3)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v) and not np.array_equal(a.x, c.x)
    assert a.n == 1000 and a.x.shape == (1000, 3) and abs(a.m.sum() - 1.0) < 1e-12 and a.eps == 1e-3
