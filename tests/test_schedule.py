"""Host logic of the FP64 Cholesky's static schedule (cimmino_cholesky_schedule), on CPU:
every block is factored exactly once (whole, or as two halves that open two different CTA
lists), the reported makespan is the largest list's cost under the documented weights, and
the packing is no worse than longest-first list scheduling; the split decisions follow the
stated rule (no split among equal blocks that outnumber nothing, a dominant block split)."""
import heapq

import numpy as np
import pytest

g = pytest.importorskip("paper_1710_07769_gb300")

W_DIAG, W_TRSM, W_SYNC = 1.41, 0.59, 0.09


def costs(nt, ntr, nfu):
    diag = W_DIAG * nt
    return diag + W_TRSM * ntr + nfu, diag


def check(nt, ntr, nfu, maxcta, lists, nsplit, mk):
    cost, diag = costs(np.asarray(nt, float), np.asarray(ntr, float), np.asarray(nfu, float))
    nblk = len(nt)
    assert 0 < len(lists) <= maxcta and all(lists)
    seen = {}
    loads = []
    for k, L in enumerate(lists):
        t = 0.0
        for q, (b, part, nparts) in enumerate(L):
            seen.setdefault(b, []).append((k, q, part, nparts))
            if nparts == 1:
                t += cost[b]
            else:
                t += diag[b] + 0.5 * (cost[b] - diag[b]) + W_SYNC * nt[b]
        loads.append(t)
    assert sorted(seen) == list(range(nblk))
    splits = 0
    for b, occ in seen.items():
        if len(occ) == 1:
            assert occ[0][2:] == (0, 1)
        else:
            splits += 1
            assert len(occ) == 2 and sorted(o[2] for o in occ) == [0, 1]
            assert all(o[3] == 2 and o[1] == 0 for o in occ)      # first in its list
            assert occ[0][0] != occ[1][0]                         # two different CTAs
    assert splits == nsplit
    assert mk == pytest.approx(max(loads), rel=1e-9)
    return cost


def lpt(cost, m):
    h = [(0.0, k) for k in range(m)]
    for c in sorted(cost, reverse=True):
        f, k = heapq.heappop(h)
        heapq.heappush(h, (f + c, k))
    return max(f for f, _ in h)


def test_workload_like_blocks_pack_near_the_mean():
    rng = np.random.default_rng(3)
    nblk, maxcta = 512, 152
    nt = np.full(nblk, 32)
    ntr = rng.integers(20, 90, nblk)
    nfu = (ntr.astype(float) ** 2 / 60).astype(np.int64)
    ntr[:2], nfu[:2] = (194, 178), (609, 520)   # two blocks above the mean load per CTA
    lists, nsplit, mk = g.cholesky_schedule(nt, ntr, nfu, maxcta)
    cost = check(nt, ntr, nfu, maxcta, lists, nsplit, mk)
    assert nsplit >= 1 and mk < cost.max()
    assert mk <= lpt(cost, maxcta) + 1e-9
    assert mk >= cost.sum() / maxcta - 1e-9
    assert mk <= 1.06 * cost.sum() / maxcta


def test_equal_blocks_fewer_than_ctas_are_not_split():
    nt, ntr, nfu = [16] * 128, [40] * 128, [300] * 128
    lists, nsplit, mk = g.cholesky_schedule(nt, ntr, nfu, 152)
    cost = check(nt, ntr, nfu, 152, lists, nsplit, mk)
    assert nsplit == 0 and len(lists) == 128 and mk == pytest.approx(cost[0])


def test_dominant_block_is_split_and_others_are_not():
    nt, ntr, nfu = [32, 4, 4], [194, 2, 2], [609, 1, 1]
    lists, nsplit, mk = g.cholesky_schedule(nt, ntr, nfu, 152)
    check(nt, ntr, nfu, 152, lists, nsplit, mk)
    assert nsplit == 1 and [L[0][0] for L in lists[:2]] == [0, 0]


def test_no_split_when_not_allowed_and_one_cta():
    rng = np.random.default_rng(4)
    nt = rng.integers(1, 40, 50)
    ntr = rng.integers(0, 100, 50)
    nfu = rng.integers(0, 900, 50)
    lists, nsplit, mk = g.cholesky_schedule(nt, ntr, nfu, 152, allow_split=False)
    cost = check(nt, ntr, nfu, 152, lists, nsplit, mk)
    assert nsplit == 0 and mk == pytest.approx(cost.max())
    lists, nsplit, mk = g.cholesky_schedule(nt, ntr, nfu, 1)
    cost = check(nt, ntr, nfu, 1, lists, nsplit, mk)
    assert len(lists) == 1 and nsplit == 0 and mk == pytest.approx(cost.sum())


def test_invalid_counts_are_rejected():
    with pytest.raises(g.CimminoError) as e:
        g.cholesky_schedule([0], [0], [0], 152)
    assert e.value.code == g.EINVAL
    with pytest.raises(g.CimminoError) as e:
        g.cholesky_schedule([4], [1], [1], 0)
    assert e.value.code == g.EINVAL
