"""The certificates of the selection, as a property of the algorithm (host model, no GPU).

The library takes its decisions on float32 gradients g with bounds e (|g - key| <= e, key the FP64
value): a pixel is a possible candidate when g < e and is recomputed when |g| <= e; a pair of
neighbouring candidates whose gap is not certified enters the neighbour lists marked, both are
recomputed, and the rounds settle marked entries on the exact keys; a recomputed key >= 0 drops its
candidate. This test models those rules on random keys full of near-ties and checks that the accepted
set is always the greedy one of the RC section on the exact keys (ascending key, then pixel, skipping
the Chebyshev neighbours of accepted pixels)."""
import numpy as np
import pytest


def _order_uncertain(gp, ep, gq, eq):
    f = np.float32
    return abs(f(gp) - f(gq)) <= f(f(f(ep) + f(eq)) * f(1.00000024))


def _exact_greedy(keys, pix, nbrs):
    accepted, blocked = set(), set()
    for s in sorted((i for i in range(len(keys)) if keys[i] < 0), key=lambda i: (keys[i], pix[i])):
        if s in blocked:
            continue
        accepted.add(s)
        blocked.update(nbrs[s])
    return accepted


def _certified(keys, g, e, pix, nbrs):
    n = len(keys)
    cand = [i for i in range(n) if g[i] < e[i]]
    is_cand = set(cand)
    queued = {i for i in cand if abs(g[i]) <= e[i]}
    lists = {}
    for s in cand:
        row = []
        for o in nbrs[s]:
            if o not in is_cand:
                continue
            if _order_uncertain(g[s], e[s], g[o], e[o]):
                row.append(("marked", o))
                queued.add(s)
            elif (np.float64(g[o]), pix[o]) < (np.float64(g[s]), pix[s]):
                row.append(("smaller", o))
        lists[s] = row
    key = {i: (keys[i] if i in queued else np.float64(g[i])) for i in cand}
    state = {i: ("rejected" if i in queued and not keys[i] < 0 else "undecided") for i in cand}
    smaller = {s: [o for kind, o in lists[s] if kind == "smaller" or (key[o], pix[o]) < (key[s], pix[s])]
               for s in cand}
    while any(v == "undecided" for v in state.values()):
        changed = False
        for s in cand:
            if state[s] != "undecided":
                continue
            st = [state[o] for o in smaller[s]]
            if "accepted" in st:
                state[s], changed = "rejected", True
            elif all(v == "rejected" for v in st):
                state[s], changed = "accepted", True
        assert changed, "the rounds made no progress"
    return {i for i in cand if state[i] == "accepted"}


@pytest.mark.parametrize("seed", range(12))
def test_certified_selection_equals_the_exact_greedy(seed):
    rng = np.random.default_rng(seed)
    H = W = 24
    occupied = rng.random((H, W)) < 0.45
    ys, xs = np.nonzero(occupied)
    pix = list(ys * W + xs)
    where = {p: i for i, p in enumerate(pix)}
    nbrs = []
    for y, x in zip(ys, xs):
        row = []
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                q = (y + dy) * W + (x + dx)
                if (dy or dx) and 0 <= y + dy < H and 0 <= x + dx < W and q in where:
                    row.append(where[q])
        nbrs.append(row)
    n = len(pix)
    # exact keys: few distinct values near 0 and near each other, so that signs and orders are
    # often within the bounds; some exact ties and exact zeros
    keys = rng.choice([-3e-3, -1e-3, -2e-4, 0.0, 1e-4, 5e-4], n) + rng.choice([0.0, 1e-9, -1e-9, 3e-7], n)
    keys = keys.astype(np.float64)
    e = (rng.random(n) * 4e-7).astype(np.float32)
    # the float gradient: within its bound of the key, rounded to float32 (the bound widened to cover it)
    g = (keys + (rng.random(n) * 2 - 1) * e.astype(np.float64) * 0.999).astype(np.float32)
    e = np.maximum(e, np.abs(g.astype(np.float64) - keys).astype(np.float32) * np.float32(1.0000002))
    assert (np.abs(g.astype(np.float64) - keys) <= e.astype(np.float64)).all()
    assert _certified(keys, g, e, pix, nbrs) == _exact_greedy(keys, pix, nbrs)


@pytest.mark.parametrize("seed", range(8))
def test_block_sweeps_in_any_interleaving_reach_the_greedy_set(seed):
    # The rounds without grid barriers: candidates are split into contiguous ranges (one per
    # block); in every step one randomly chosen block sweeps its range once, in a random thread
    # order, reading the states as they are. Decisions depend only on smaller-key neighbours, so
    # whatever the interleaving the result is the greedy set, and a sweep of some block always
    # decides something while candidates are left (no block can wait for ever).
    rng = np.random.default_rng(100 + seed)
    n = 400
    pos = rng.permutation(30 * 30)[:n]
    pix = list(pos)
    where = {p: i for i, p in enumerate(pix)}
    nbrs = []
    for p in pix:
        y, x = divmod(int(p), 30)
        nbrs.append([where[(y + dy) * 30 + x + dx] for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                     if (dy or dx) and 0 <= y + dy < 30 and 0 <= x + dx < 30 and (y + dy) * 30 + x + dx in where])
    keys = -rng.integers(1, 40, n).astype(np.float64)          # many exact ties, broken by pixel
    order = sorted(range(n), key=lambda i: pix[i])              # candidates numbered in pixel order
    smaller = [[o for o in nbrs[s] if (keys[o], pix[o]) < (keys[s], pix[s])] for s in range(n)]
    state = ["undecided"] * n
    blocks = np.array_split(np.array(order), 7)
    left = n
    while left:
        progress = False
        for b in rng.permutation(len(blocks)):
            for s in rng.permutation(blocks[b]):
                if state[s] != "undecided":
                    continue
                st = [state[o] for o in smaller[s]]
                if "accepted" in st:
                    state[s] = "rejected"
                elif all(v == "rejected" for v in st):
                    state[s] = "accepted"
                else:
                    continue
                left -= 1
                progress = True
        assert progress, "no block could decide anything"
    assert {i for i in range(n) if state[i] == "accepted"} == _exact_greedy(keys, pix, nbrs)
