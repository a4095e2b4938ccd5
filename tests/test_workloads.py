"""The seeded input generators: pinned to splitmix64's published test vector,
closed-form properties of the workloads, and the GPU twin of the numpy
streams (bit-identical)."""
import numpy as np
import pytest

from workloads import recipes, splitmix as sm


def test_splitmix64_published_vector():
    # first outputs of splitmix64 seeded with 1234567 (Vigna's reference)
    assert sm.sequential(1234567, 5) == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                         4593380528125082431, 16408922859458223821]


def test_counter_form_matches_sequential():
    base = sm.stream_base(7, 3)
    assert [int(x) for x in sm.stream_u64(7, 3, 0, 20)] == sm.sequential(base, 20)
    assert np.array_equal(sm.stream_u64(7, 3, 5, 10), sm.stream_u64(7, 3, 0, 15)[5:])
    idx = np.array([0, 3, 14, 2])
    assert np.array_equal(sm.stream_at(7, 3, idx), sm.stream_u64(7, 3, 0, 15)[idx])


def test_affine_sample_is_distinct():
    for n_pop in (1, 2, 1000, 1 << 20, 12_500_000):
        s = sm.affine_sample(n_pop, min(n_pop, 50000), 14)
        assert len(np.unique(s)) == len(s) and s.min() >= 0 and s.max() < n_pop


def test_set_u32_workload_shape():
    w = recipes.set_u32_workload()
    assert len(w.insert_keys) == 1_000_000 and len(w.find_keys) == 1_000_000 and len(w.erase_keys) == 500_000
    # expected duplicate pairs among 10^6 uniform u32 keys: n^2 / 2^33 ~ 116
    dups = len(w.insert_keys) - len(np.unique(w.insert_keys))
    assert 60 < dups < 180
    hit = np.isin(w.find_keys, w.insert_keys).mean()
    assert 0.49 < hit < 0.51


def test_multi_table_shape():
    s = recipes.multi_table_slots()
    assert len(s) == 1024 and s.min() >= 1 << 10 and s.max() <= (1 << 22) + 16 and (s % 16 == 0).all()
    # E[2^U(10,22)] = (2^22 - 2^10) / (12 ln 2) ~ 5.04e5 per table
    assert 4.0e5 < s.mean() < 6.0e5
    o = recipes.multi_table_ops(4096, 3)
    assert len(o.insert_keys) + len(o.find_keys) + len(o.erase_keys) == 2048
    assert np.isin(o.erase_keys, o.insert_keys).all()


@pytest.mark.gpu
def test_gpu_streams_match_numpy():
    import torch
    from workloads import gpu
    a = gpu.stream_u64(3, 0, 1000, 4097).cpu().numpy().view(np.uint64)
    assert np.array_equal(a, sm.stream_u64(3, 0, 1000, 4097))
    b = gpu.stream_u32(1, 0, 0, 5000).cpu().numpy().view(np.uint32)
    assert np.array_equal(b, sm.stream_u32(1, 0, 0, 5000))
    c = gpu.sample_u64(3, 1_000_003, 70000, 14, 0).cpu().numpy().view(np.uint64)
    assert np.array_equal(c, recipes.map_hit_keys(1_000_003, 70000))
    d = gpu.value_of(torch.from_numpy(a.view(np.int64)).cuda()).cpu().numpy().view(np.uint64)
    assert np.array_equal(d, sm.value_of(a))
