"""The host-side work decomposition that kmc_run launches (kmc_plan_items),
checked on the CPU: every target of every lysosome lands in exactly one group,
every group's parts cover its sources once and in order, chains are cut at
lysosome boundaries, and the wave split follows its rule. No GPU is needed."""
import math

import numpy as np
import pytest

from paper_1407_2737_gb300 import build as kbuild
from paper_1407_2737_gb300 import kmc

FP32, FP64 = kmc.KMC_FP32_MIXED, kmc.KMC_FP64_PLAIN


@pytest.fixture(scope="module", autouse=True)
def _built():
    kbuild.build()


def _check_plan(n, prec, tpl, chunk, bps, n_sms):
    items, cut = kmc.kmc_plan_items(n, prec, tpl, chunk, bps, n_sms)
    gsize = 32 * tpl
    nrec = [(v + 1) // 2 if prec == FP32 else v for v in n]
    # lysosomes in order of size, largest first, ties in input order
    seen = []
    for l in items[:, 0]:
        if not seen or seen[-1] != l:
            assert l not in seen, "a lysosome's items are not contiguous"
            seen.append(int(l))
    assert seen == sorted(range(len(n)), key=lambda l: -n[l])
    covered = [np.zeros(v, dtype=np.int32) for v in n]
    u = 0
    gid = 0
    while u < len(items):
        l, t0, nt, g, j0, j1, part, parts = items[u]
        assert g == gid and part == 0 and parts >= 1
        assert t0 % gsize == 0 and 1 <= nt <= gsize and t0 + nt <= n[l]
        assert nt == gsize or t0 + nt == n[l]  # only a lysosome's last group is short
        covered[l][t0:t0 + nt] += 1
        end = 0
        for s in range(parts):
            li, ti, nti, gi, a, b, si, pi = items[u + s]
            assert (li, ti, nti, gi, si, pi) == (l, t0, nt, g, s, parts)
            assert a == end and b > a  # contiguous, non-empty parts in order
            end = b
        assert end == nrec[l]
        if chunk > 0:
            rchunk = chunk // 2 if prec == FP32 else chunk
            nominal = max(1, math.ceil(nrec[l] / rchunk))
            if len(n) == 1 and n_sms > 0:
                assert nominal <= parts <= nrec[l]  # a single chain may fill its last wave
            else:
                assert parts == nominal
        u += parts
        gid += 1
    for c in covered:
        assert np.all(c == 1)
    # chains: at most min(n_lys, KMC_MAX_CHAINS), cut where the lysosome changes
    assert cut[0] == 0 and cut[-1] == len(items)
    assert all(a < b for a, b in zip(cut, cut[1:]))
    assert 1 <= len(cut) - 1 <= min(len(n), kmc.KMC_MAX_CHAINS)
    for q in cut[1:-1]:
        assert items[q - 1, 0] != items[q, 0]
    return items, cut


@pytest.mark.parametrize("prec,tpl", [(FP32, 1), (FP32, 2), (FP32, 3), (FP64, 1)])
@pytest.mark.parametrize("chunk", [0, 64, 256, 1024])
def test_random_batches_cover_every_pair_once(prec, tpl, chunk):
    rng = np.random.default_rng(100 + tpl + chunk)
    for trial in range(12):
        n = [int(v) for v in rng.integers(1, 3000, size=int(rng.integers(1, 20)))]
        if trial % 3 == 0:
            n[0] = 1  # single-NP lysosome
        _check_plan(n, prec, tpl, chunk, 5, 152 if trial % 2 else 0)


def test_equal_lysosomes_give_one_chain_each():
    items, cut = _check_plan([2000] * 8, FP32, 1, 1024, 5, 152)
    assert len(cut) == 9
    for q in range(8):
        assert len(set(items[cut[q]:cut[q + 1], 0])) == 1
    # 63 groups of 32 targets per lysosome, sources in two parts of 512 records
    assert len(items) == 8 * 63 * 2


def test_chains_balance_source_records():
    rng = np.random.default_rng(5)
    n = [int(v) for v in rng.lognormal(np.log(800), 0.5, size=512).clip(2, 6000)]
    items, cut = _check_plan(n, FP32, 1, 0, 5, 152)
    rec = (items[:, 5] - items[:, 4]).astype(np.int64)
    total = rec.sum()
    per_chain = [rec[a:b].sum() for a, b in zip(cut, cut[1:])]
    assert len(per_chain) == kmc.KMC_MAX_CHAINS
    # whole lysosomes per chain: within one lysosome's work of the even share
    per_lys = np.bincount(items[:, 0], weights=rec, minlength=len(n))
    assert max(per_chain) <= total / len(per_chain) + per_lys.max()


@pytest.mark.parametrize("n,bps", [(152 * 32 * 3 + 5 * 32, 5), (152 * 32 + 40 * 32, 5),
                                   (152 * 32 * 4 + 100 * 32, 5), (152 * 32 * 2 + 151 * 32, 3)])
def test_wave_split_of_a_single_lysosome(n, bps):
    """chunk = 0, one chain: with G = q P + r groups on P SMs, the r last
    (smallest) groups are cut into the s parts (2..8) that minimise the
    busiest SM's load ceil(r s / P) / s, as long as q + ceil(r s / P) blocks
    fit on an SM; otherwise nothing is split."""
    P = 152
    items, _ = _check_plan([n], FP32, 1, 0, bps, P)
    G = math.ceil(n / 32)
    q, r = divmod(G, P)
    best_s, best = 1, 1.0
    for s in range(2, 9):
        if r == 0:
            break
        per_sm = math.ceil(r * s / P)
        if q + per_sm > bps:
            break
        if per_sm / s < best - 1e-9:
            best, best_s = per_sm / s, s
    parts = items[:, 7]
    split_groups = sorted(set(items[parts > 1, 3]))
    if best_s == 1:
        assert len(split_groups) == 0
    else:
        assert split_groups == list(range(G - r, G))
        assert np.all(parts[items[:, 3] >= G - r] == best_s)
    assert len(items) == (G - r) + r * best_s


def test_no_wave_split_without_sms_or_with_chains():
    items, _ = _check_plan([152 * 32 * 3 + 5 * 32], FP32, 1, 0, 5, 0)
    assert np.all(items[:, 7] == 1)
    items, _ = _check_plan([152 * 32 * 3 + 5 * 32, 100], FP32, 1, 0, 5, 152)
    assert np.all(items[:, 7] == 1)  # two chains: no device-wide wave to even out


def test_plan_rejects_bad_arguments():
    for args in [([100], FP64, 2, 0, 5, 0), ([100], FP64, 3, 0, 5, 0), ([100], FP32, 4, 0, 5, 0),
                 ([100], FP32, 1, 100, 5, 0),
                 ([100, 0], FP32, 1, 0, 5, 0), ([100], FP32, 1, 0, 0, 0), ([], FP32, 1, 0, 5, 0),
                 ([100], 7, 1, 0, 5, 0)]:
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_plan_items(*args)
        assert e.value.status == kmc.KMC_EINVAL, args


@pytest.mark.parametrize("n,tpl,chunk,bps", [(50000, 2, 8192, 2), (50000, 2, 4096, 4),
                                             (50000, 1, 1024, 5), (8000, 1, 2048, 5),
                                             (3000, 3, 256, 4)])
def test_single_chain_split_fills_whole_waves(n, tpl, chunk, bps):
    """One lysosome split by chunk over several waves: the last groups take one
    part more each until the items fill whole waves of n_sms x blocks_per_sm
    (the last wave would otherwise hold a few full-size items while the rest
    of the GPU waits), so the smaller items come last."""
    n_sms = 152
    items, cut = _check_plan([n], FP32, tpl, chunk, bps, n_sms)
    slots = n_sms * bps
    groups = [items[u] for u in range(len(items)) if items[u, 6] == 0]
    parts = np.array([g[7] for g in groups])
    nominal = math.ceil(((n + 1) // 2) / (chunk // 2))
    if len(groups) * nominal > slots:
        assert len(items) % slots == 0
        assert np.all(np.diff(parts) >= 0)  # the groups with more parts come last
        assert parts.max() - parts.min() <= 1 + (slots // len(groups))
    else:
        assert np.all(parts == nominal)
