"""The serving loop's host-side policies, checked without a GPU through the C-ABI
(sldm_cache_plan, sldm_batch_plan): the LRU admission under a byte budget and
the FIFO same-key batching, each against a plain re-statement in Python and
against the invariants the server relies on."""
from collections import OrderedDict

import numpy as np
import pytest


def _sl():
    from paper_2106_06184_gb300 import sldm
    return sldm


def lru_model(keys, sizes, budget):
    """Least recently used eviction, restated: hit moves to the front; a miss evicts
    from the back until the entry fits; an entry larger than the budget is refused."""
    c = OrderedDict()
    used = 0
    act, ev = [], []
    for k, b in zip(keys, sizes):
        if k in c:
            c.move_to_end(k)
            act.append(0)
            ev.append(0)
            continue
        if budget > 0 and b > budget:
            act.append(2)
            ev.append(0)
            continue
        n = 0
        while budget > 0 and used + b > budget:
            _, bb = c.popitem(last=False)
            used -= bb
            n += 1
        c[k] = b
        used += b
        act.append(1)
        ev.append(n)
    return np.array(act), np.array(ev)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cache_plan_matches_lru_model(seed):
    sl = _sl()
    rng = np.random.default_rng(2106_06184 + seed)
    nkeys = 12
    size_of = rng.integers(1, 40, nkeys) * 1000
    keys = rng.zipf(1.5, 400) % nkeys
    sizes = size_of[keys]
    for budget in (0, 60_000, 150_000):
        act, ev = sl.cache_plan(keys, sizes, budget)
        ra, re = lru_model(keys.tolist(), sizes.tolist(), budget)
        assert np.array_equal(act, ra) and np.array_equal(ev, re)
        if budget == 0:
            assert ev.sum() == 0 and (act != 2).all()


def batch_model(keys, nrhs, max_batch):
    q = list(range(len(keys)))
    out = [None] * len(keys)
    b = 0
    while q:
        first = q[0]
        take = [first]
        n = nrhs[first]
        if n < max_batch:
            for i in q[1:]:
                if keys[i] == keys[first] and n + nrhs[i] <= max_batch:
                    take.append(i)
                    n += nrhs[i]
        for i in take:
            out[i] = b
            q.remove(i)
        b += 1
    return np.array(out)


@pytest.mark.parametrize("max_batch", [1, 8, 32])
def test_batch_plan_matches_fifo_model(max_batch):
    sl = _sl()
    rng = np.random.default_rng(2106_06184 + max_batch)
    keys = rng.integers(0, 6, 300)
    nrhs = rng.integers(1, 17, 300)
    got = sl.batch_plan(keys, nrhs, max_batch)
    assert np.array_equal(got, batch_model(keys.tolist(), nrhs.tolist(), max_batch))
    for b in np.unique(got):
        idx = np.nonzero(got == b)[0]
        assert len(set(keys[idx])) == 1                               # one key per batch
        assert nrhs[idx].sum() <= max_batch or len(idx) == 1           # fits, or a lone large request
    # batches are formed oldest-first: the first request of batch b precedes that of batch b + 1
    firsts = [np.nonzero(got == b)[0][0] for b in range(got.max() + 1)]
    assert firsts == sorted(firsts)


def test_policies_reject_invalid_input():
    sl = _sl()
    with pytest.raises(sl.SldmError):
        sl.batch_plan([1, 2], [1, 0], 8)
    with pytest.raises(sl.SldmError):
        sl.cache_plan([1], [10], -1)
