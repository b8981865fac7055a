"""The symmetric pair form's work decomposition (kmc_plan_sym), checked on the
CPU by brute force: every ordered pair of cells of a lysosome (the cell with
itself included) is evaluated exactly once, as a forward term of an
off-diagonal item, as a reverse term of one, or inside a row group's diagonal
item; every reverse slot is written by exactly one item and read by exactly
the update items of its cell; every target lies in exactly one update item,
whose forward slots are exactly its row group's items. No GPU is needed."""
import numpy as np
import pytest

from paper_1407_2737_gb300 import build as kbuild
from paper_1407_2737_gb300 import kmc

CELL = kmc.KMC_CELL


@pytest.fixture(scope="module", autouse=True)
def _built():
    kbuild.build()


def _slot_offset(h, gc):
    """Reverse slots of the cells before cell h: one per row group below each
    cell, summed cell by cell."""
    return sum(hp // gc for hp in range(h))


def _check(n, gc, src_cells):
    items, upd, n_rev, cut_i, cut_u = kmc.kmc_plan_sym(n, gc, src_cells)
    assert len(items) > 0 and len(upd) > 0
    # forward slot = the item's index
    assert np.array_equal(items[:, 4], np.arange(len(items)))
    written = {}
    rbase_of = {}
    covered = {l: np.zeros(((v + CELL - 1) // CELL,) * 2, dtype=np.int32) for l, v in enumerate(n)}
    for u, (l, g, h0, h1, fwd, rbase, _, _) in enumerate(items):
        nc = (n[l] + CELL - 1) // CELL
        assert 0 <= g * gc < nc
        rbase_of.setdefault(l, rbase)
        assert rbase_of[l] == rbase
        M = covered[l]
        tcells = [c for c in range(g * gc, (g + 1) * gc) if c < nc]
        if h0 == -1:
            assert h1 == -1
            for t in tcells:
                for s in tcells:
                    M[t, s] += 1
            continue
        assert (g + 1) * gc <= h0 < h1 <= nc
        if src_cells > 0:
            assert h1 - h0 <= src_cells
        assert len(tcells) == gc  # off-diagonal rows are whole
        for h in range(h0, h1):
            for t in tcells:
                M[t, h] += 1  # forward: target cell t from source cell h
                M[h, t] += 1  # reverse: source cell h from target cell t
            slot = rbase + _slot_offset(h, gc) + g
            assert slot not in written
            written[slot] = (l, h, g)
    for l, M in covered.items():
        assert np.all(M == 1), (l, np.argwhere(M != 1)[:5])
    assert len(written) == n_rev and set(written) == set(range(n_rev))
    # lysosomes' reverse ranges do not overlap
    ranges = sorted((rbase_of[l], rbase_of[l] + _slot_offset((n[l] + CELL - 1) // CELL, gc))
                    for l in rbase_of)
    assert all(a[1] <= b[0] for a, b in zip(ranges, ranges[1:]))
    # update items: every target once, inside one cell, with the right slots
    seen = {l: np.zeros(v, dtype=np.int32) for l, v in enumerate(n)}
    for (l, t0, nt, fwd0, nfwd, rev0, nrev, gt0) in upd:
        assert 1 <= nt <= 32 and t0 % 32 == 0 and (t0 % CELL) + nt <= CELL and t0 + nt <= n[l]
        seen[l][t0:t0 + nt] += 1
        h = t0 // CELL
        g = h // gc
        assert gt0 == t0 - g * gc * CELL and 0 <= gt0 and gt0 + nt <= gc * CELL
        rows = [u for u in range(len(items)) if items[u, 0] == l and items[u, 1] == g]
        assert list(range(fwd0, fwd0 + nfwd)) == rows
        assert items[fwd0, 2] == -1  # the diagonal item first
        assert nrev == h // gc
        reads = [written[s] for s in range(rev0, rev0 + nrev)]
        assert reads == [(l, h, gp) for gp in range(nrev)]
    for l, v in seen.items():
        assert np.all(v == 1)
    # chains: the same lysosome boundaries in both lists
    assert cut_i[0] == 0 and cut_u[0] == 0 and cut_i[-1] == len(items) and cut_u[-1] == len(upd)
    assert len(cut_i) == len(cut_u) and 2 <= len(cut_i) <= min(len(n), kmc.KMC_MAX_CHAINS) + 1
    for a, b in zip(cut_i[1:-1], cut_u[1:-1]):
        assert items[a - 1, 0] != items[a, 0] and upd[b - 1, 0] != upd[b, 0]
        assert items[a, 0] == upd[b, 0]
    return items, upd


@pytest.mark.parametrize("gc", [4, 8])
@pytest.mark.parametrize("src_cells", [0, 1, 3, 8])
def test_every_cell_pair_once(gc, src_cells):
    rng = np.random.default_rng(gc * 10 + src_cells)
    for trial in range(4):
        n = [int(v) for v in rng.integers(1, 2600, size=int(rng.integers(1, 12)))]
        n[0] = [1, 63, 64, 65][trial]
        _check(n, gc, src_cells)


def test_large_lysosome_plan():
    items, upd = _check([50000], 8, 32)
    # 782 cells, 98 row groups: the diagonal items plus ceil(cells above / 32) per group
    nc, gc = (50000 + CELL - 1) // CELL, 8
    expect = sum(1 + -(-(nc - (g + 1) * gc) // 32) if nc > (g + 1) * gc else 1
                 for g in range(-(-nc // gc)))
    assert len(items) == expect and len(upd) == -(-50000 // 32)


def test_plan_rejects_bad_arguments():
    for args in [([100], 3, 0), ([100], 8, -1), ([0], 4, 0), ([], 4, 0)]:
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_plan_sym(*args)
        assert e.value.status == kmc.KMC_EINVAL, args
