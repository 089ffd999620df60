"""Work partition of the fused chain's persistent iteration (host arithmetic,
no GPU): every (256-column tile, 32-row block) unit has exactly one CTA, the
owner formula the kernel uses finds it, a CTA shares at most its first and
last tile with other CTAs, its partial slots fit `segs`, and the rows it
stages at once fit `chunk`."""
import numpy as np
import pytest

from paper_2509_20500_gb300 import spl

TW = 256   # columns of a tile: one warp span of the fused chain kernels, 8 columns per lane


def _owner(u, U, G):
    # the kernel's inverse of u0(b) = floor(b U / G)
    return ((u + 1) * G + U - 1) // U - 1


def _check(n, sms, bps):
    pl = spl.chain_run_plan(n, sms, bps)
    G, T, RB, segs, chunk, vlen = (pl[k] for k in ("grid", "tiles", "row_blocks", "segs", "chunk", "vlen"))
    assert vlen >= n and vlen % 128 == 0 and RB == vlen // 32
    assert T == (n + TW - 1) // TW
    U = T * RB
    assert 1 <= G <= min(bps * sms, 512, U)
    start = [b * U // G for b in range(G + 1)]
    assert start[0] == 0 and start[-1] == U
    assert all(start[b + 1] > start[b] for b in range(G))      # no CTA without work
    umax = max(start[b + 1] - start[b] for b in range(G))
    assert chunk == min(8192, 32 * umax)
    # owner formula against the actual ranges (sampled units for large U)
    rng = np.random.default_rng(n + sms)
    us = set(rng.integers(0, U, size=min(U, 4000)).tolist()) | {0, U - 1} | set(start[1:-1])
    bs = np.searchsorted(np.asarray(start), np.asarray(sorted(us)), side="right") - 1
    for u, b in zip(sorted(us), bs):
        assert _owner(u, U, G) == b, (n, u)
    shared = {}
    for b in range(G):
        u0, u1 = start[b], start[b + 1]
        tf, tl = u0 // RB, (u1 - 1) // RB
        assert tl - tf + 1 <= segs
        own_first = u0 == tf * RB and u1 >= (tf + 1) * RB
        own_last = u1 == (tl + 1) * RB and u0 <= tl * RB
        for t in (tf, tl):
            if not (own_first if t == tf else own_last):
                shared.setdefault(t, set()).add(b)
    # a shared tile's contributors are the CTAs owner(first unit) .. owner(last unit)
    for t, cs in shared.items():
        bf, bl = _owner(t * RB, U, G), _owner((t + 1) * RB - 1, U, G)
        assert cs == set(range(bf, bl + 1)) and len(cs) >= 2, (n, t)
    return pl


@pytest.mark.parametrize("n", [2, 3, 100, 127, 128, 129, 1000, 1500, 2000, 3000, 4100, 9000, 10000, 16000,
                               18000, 50000, 200000])
def test_partition_invariants(n):
    for sms, bps in ((152, 2), (148, 2), (152, 1), (7, 2), (1, 1)):
        _check(n, sms, bps)


def test_partition_sizes_used_by_the_gpu_tests():
    # N = 10000: two tiles per CTA at most; N = 26000: more rows than one
    # window (274 units of 32 rows > 256)
    p = _check(10000, 152, 2)
    assert (p["grid"], p["tiles"], p["segs"], p["chunk"]) == (304, 40, 2, 1344)
    p = _check(26000, 152, 2)
    assert p["chunk"] == 8192 and p["segs"] == 2 and p["tiles"] * p["row_blocks"] > 256 * p["grid"]


def test_plan_rejects_bad_arguments():
    for args in ((1, 152, 2), (2000, 0, 2), (2000, 152, 0), ((1 << 24) + 1, 152, 2)):
        with pytest.raises(spl.SplError):
            spl.chain_run_plan(*args)


# ---------------------------------------------------------------- multi-chain lockstep partition

def _tile_contributors(n_bins, active, G):
    """Largest number of CTAs one column tile of each active chain meets when
    the units of the active chains, chain after chain, are split as
    [b U / G', (b+1) U / G') over G' = min(G, U) CTAs (the kernel's partition)."""
    T = [(n + TW - 1) // TW for n in n_bins]
    RB = [spl.chain_run_plan(n, 1, 1)["vlen"] // 32 for n in n_bins]
    U = sum(T[g] * RB[g] for g in active)
    Ge = min(G, U)
    owner = lambda u: ((u + 1) * Ge + U - 1) // U - 1
    out, base = {}, 0
    for g in active:
        t = np.arange(T[g], dtype=np.int64)
        first = base + t * RB[g]
        last = first + RB[g] - 1
        out[g] = int((owner(last) - owner(first) + 1).max())
        base += T[g] * RB[g]
    return out


@pytest.mark.parametrize("n_bins,sms,bps", [
    ([10000] * 12, 152, 2),                                   # the dead-time sweep
    ([18000, 2, 37, 333, 2000, 1024], 152, 2),                # one large chain and tiny ones
    ([2, 5, 40, 130, 700], 152, 2),                           # fewer units than CTAs
    ([16000, 500], 4, 1),
])
def test_chains_plan_slots_bound_every_step(n_bins, sms, bps):
    """Whatever subset of the chains is still iterating, no tile meets more
    CTAs than the partial slots the plan gives its chain."""
    import itertools
    slots = spl.chains_plan(n_bins, sms, bps)
    G = sms * bps
    n = len(n_bins)
    subsets = [list(c) for r in range(1, n + 1) for c in itertools.combinations(range(n), r)]
    if len(subsets) > 300:
        rng = np.random.default_rng(5)
        subsets = [subsets[i] for i in rng.choice(len(subsets), 300, replace=False)] + [list(range(n))] + \
                  [[g] for g in range(n)]
    for act in subsets:
        for g, c in _tile_contributors(n_bins, act, G).items():
            assert c <= slots[g], (act, g, c, slots[g])
    assert np.all(slots >= 1) and np.all(slots <= G)


def test_chains_plan_rejects_bad_arguments():
    with pytest.raises(spl.SplError):
        spl.chains_plan([100] * 33, 152, 2)       # more than one launch takes
    with pytest.raises(spl.SplError):
        spl.chains_plan([1, 100], 152, 2)         # a chain needs 2 bins
    with pytest.raises(spl.SplError):
        spl.chains_plan([100], 0, 2)
