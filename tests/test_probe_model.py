"""The probe-count model (tests/probe_model.py) on the CPU: the facts the exact GPU probe
counts rest on. For linear probing, the set of occupied slots and the total displacement of the
stored keys do not depend on the order the keys were inserted in (the GPU inserts them
concurrently); the longest displacement can. And a miss at load a reads (1 + 1/(1 - a)^2) / 2
slots on average for random homes (Knuth's analysis of linear probing)."""
import numpy as np
import pytest

from probe_model import linear_probing_model, miss_reads


@pytest.mark.parametrize("seed,n_slots,n_keys", [(1, 64, 40), (2, 256, 230), (3, 1024, 512), (4, 97, 97)])
def test_occupancy_and_total_displacement_do_not_depend_on_order(seed, n_slots, n_keys):
    rng = np.random.default_rng(seed)
    homes = list(rng.integers(0, n_slots, n_keys))
    occ0, total0, _ = linear_probing_model(homes, n_slots)
    for _ in range(20):
        perm = [homes[i] for i in rng.permutation(n_keys)]
        occ, total, _ = linear_probing_model(perm, n_slots)
        assert np.array_equal(occ, occ0) and total == total0
    assert occ0.sum() == n_keys


def test_longest_displacement_can_depend_on_order():
    # homes 0, 0, 1: inserted as (0, 0, 1) the third key moves 1 slot; as (1, 0, 0) the last
    # key moves 2 slots
    assert linear_probing_model([0, 0, 1], 8)[2] == 1
    assert linear_probing_model([1, 0, 0], 8)[2] == 2
    assert linear_probing_model([0, 0, 1], 8)[1] == linear_probing_model([1, 0, 0], 8)[1] == 5


@pytest.mark.parametrize("load", [0.25, 0.5, 0.75])
def test_miss_cost_matches_knuths_formula(load):
    rng = np.random.default_rng(int(load * 100))
    n_slots = 1 << 15
    homes = list(rng.integers(0, n_slots, int(load * n_slots)))
    occ, _, _ = linear_probing_model(homes, n_slots)
    probes = [miss_reads(occ, int(h), n_slots) for h in rng.integers(0, n_slots, 20000)]
    want = (1 + 1 / (1 - load) ** 2) / 2
    assert abs(np.mean(probes) - want) < 0.08 * want


def test_miss_reads_cut_at_the_bound_and_wrap():
    occ = np.array([True, True, False, False, True, True, True, True])
    assert miss_reads(occ, 4, 99) == 7  # 4, 5, 6, 7, 0, 1 occupied, then 2 empty
    assert miss_reads(occ, 4, 3) == 3
    assert miss_reads(occ, 2, 99) == 1
