"""Pins of the oracle's simple-point tests, ranked selection and whole iterations."""
import itertools

import numpy as np
import pytest
from scipy import ndimage

CROSS2 = ndimage.generate_binary_structure(2, 1)
FULL2 = ndimage.generate_binary_structure(2, 2)
CROSS3 = ndimage.generate_binary_structure(3, 1)
FULL3 = ndimage.generate_binary_structure(3, 3)


def _yokoi4(nb9):
    # neighbours E, NE, N, NW, W, SW, S, SE (counter-clockwise), index 8 wraps to E
    g = np.asarray(nb9).reshape(3, 3)
    ring = [g[1, 2], g[0, 2], g[0, 1], g[0, 0], g[1, 0], g[2, 0], g[2, 1], g[2, 2]]
    ring = [int(v) for v in ring] + [int(g[1, 2])]
    return sum(ring[k] - ring[k] * ring[k + 1] * ring[k + 2] for k in (0, 2, 4, 6))


def test_simple_2d_all_configs_match_yokoi(orc):
    # Yokoi's connectivity number for 4-connectivity is 1 exactly at 4-simple points.
    for code in range(256):
        bits = [(code >> i) & 1 for i in range(8)]
        nb = bits[:4] + [1] + bits[4:]
        assert orc.simple_2d(nb) == (_yokoi4(nb) == 1), nb


def _count(X, structure):
    return ndimage.label(X, structure=structure)[1]


@pytest.mark.parametrize("density,seed", [(0.4, 0), (0.55, 1), (0.7, 2)])
def test_simple_2d_global_component_counts(orc, density, seed):
    rng = np.random.default_rng(seed)
    for _ in range(6):
        X = np.zeros((16, 16), bool)
        X[2:-2, 2:-2] = rng.random((12, 12)) < density
        c4, c8 = _count(X, CROSS2), _count(~X, FULL2)
        for y, x in zip(*np.nonzero(X)):
            s = orc.simple_2d(X[y - 1:y + 2, x - 1:x + 2].astype(np.uint8))
            Y = X.copy()
            Y[y, x] = False
            same = _count(Y, CROSS2) == c4 and _count(~Y, FULL2) == c8
            assert s == same, (y, x)


def _euler6(X):
    X = X.astype(np.int64)
    V = X.sum()
    E = sum(int((np.take(X, range(0, X.shape[a] - 1), a) * np.take(X, range(1, X.shape[a]), a)).sum()) for a in range(3))
    F = 0
    for a, b in ((0, 1), (0, 2), (1, 2)):
        sl = lambda i, j: X[tuple(slice(i if ax == a else (j if ax == b else 0),
                                       X.shape[ax] - 1 + i if ax == a else (X.shape[ax] - 1 + j if ax == b else X.shape[ax]))
                                 for ax in range(3))]
        F += int((sl(0, 0) * sl(1, 0) * sl(0, 1) * sl(1, 1)).sum())
    Cc = 1
    for dz, dy, dx in itertools.product((0, 1), repeat=3):
        Cc = Cc * X[dz:X.shape[0] - 1 + dz, dy:X.shape[1] - 1 + dy, dx:X.shape[2] - 1 + dx]
    return int(V) - E + F - int(Cc.sum())


@pytest.mark.parametrize("density,seed", [(0.35, 0), (0.5, 1), (0.65, 2), (0.8, 3)])
def test_simple_3d_keeps_global_invariants(orc, density, seed):
    # necessary condition: deleting a simple voxel keeps the 6-components of X, the
    # 26-components of the complement and the Euler characteristic of X (the converse fails:
    # one tunnel can be cut while another is made, so the link test below is the full pin)
    rng = np.random.default_rng(100 + seed)
    simple_seen = 0
    for _ in range(3):
        X = np.zeros((9, 9, 9), bool)
        X[1:-1, 1:-1, 1:-1] = rng.random((7, 7, 7)) < density
        c6, c26, chi = _count(X, CROSS3), _count(~X, FULL3), _euler6(X)
        for z, y, x in zip(*np.nonzero(X)):
            if not orc.simple_3d(X[z - 1:z + 2, y - 1:y + 2, x - 1:x + 2].astype(np.uint8)):
                continue
            Y = X.copy()
            Y[z, y, x] = False
            assert _count(Y, CROSS3) == c6 and _count(~Y, FULL3) == c26 and _euler6(Y) == chi, (z, y, x)
            simple_seen += 1
    assert simple_seen > 20


_AX = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


def _link_contractible(nb):
    """Link of the centre in the cubical complex of X with 6-adjacency: vertices are the
    6-neighbours in X, edges the unit squares through the centre, triangles the unit cubes
    through the centre. The centre is simple iff this link is contractible: nonempty,
    connected, Euler characteristic 1 and not the whole octahedron."""
    g = np.asarray(nb).reshape(3, 3, 3)
    at = lambda v: bool(g[v[0] + 1, v[1] + 1, v[2] + 1])
    add = lambda *vs: tuple(sum(c) for c in zip(*vs))
    V = [k for k in range(6) if at(_AX[k])]
    E = []
    for a, b in itertools.combinations(range(6), 2):
        if a // 2 == b // 2:
            continue
        if at(_AX[a]) and at(_AX[b]) and at(add(_AX[a], _AX[b])):
            E.append((a, b))
    T = 0
    for a, b, c in itertools.product((0, 1), (2, 3), (4, 5)):
        vs = [_AX[a], _AX[b], _AX[c], add(_AX[a], _AX[b]), add(_AX[a], _AX[c]), add(_AX[b], _AX[c]),
              add(_AX[a], _AX[b], _AX[c])]
        T += all(at(v) for v in vs)
    if not V or T == 8:
        return False
    comp = {v: v for v in V}
    def find(v):
        while comp[v] != v:
            v = comp[v]
        return v
    for a, b in E:
        comp[find(a)] = find(b)
    if len({find(v) for v in V}) != 1:
        return False
    return len(V) - len(E) + T == 1


@pytest.mark.parametrize("density", [0.2, 0.4, 0.5, 0.6, 0.8])
def test_simple_3d_equals_contractible_link(orc, density):
    rng = np.random.default_rng(int(density * 100))
    for _ in range(4000):
        nb = (rng.random((3, 3, 3)) < density).astype(np.uint8)
        assert orc.simple_3d(nb) == _link_contractible(nb), nb.ravel().tolist()


def test_simple_2d_equals_contractible_link(orc):
    for code in range(256):
        bits = [(code >> i) & 1 for i in range(8)]
        nb = np.array(bits[:4] + [1] + bits[4:], np.uint8).reshape(3, 3)
        g = np.zeros((3, 3, 3), np.uint8)
        g[1] = nb
        # a planar configuration embedded in 3D: its 2D (4,8) test equals the link test
        assert orc.simple_2d(nb) == _link_contractible(g)


def test_simple_3d_hand_cases(orc):
    cube = np.zeros((3, 3, 3), np.uint8)
    assert not orc.simple_3d(cube)                      # isolated voxel: deleting removes a component
    assert not orc.simple_3d(np.ones((3, 3, 3), np.uint8))   # interior voxel: deleting makes a cavity
    face = np.zeros((3, 3, 3), np.uint8)
    face[:2] = 1                                         # on a flat face
    assert orc.simple_3d(face)
    line = np.zeros((3, 3, 3), np.uint8)
    line[1, 1, 0] = 1
    assert orc.simple_3d(line)                           # end of a line
    line[1, 1, 2] = 1
    assert not orc.simple_3d(line)                       # middle of a line
    diag = np.zeros((3, 3, 3), np.uint8)
    diag[0, 0, 0] = 1
    assert not orc.simple_3d(diag)                       # only a corner neighbour: 6-isolated


def test_simple_3d_symmetry(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        nb = (rng.random((3, 3, 3)) < 0.5).astype(np.uint8)
        s = orc.simple_3d(nb)
        for perm in itertools.permutations(range(3)):
            t = np.transpose(nb, perm)
            for flips in itertools.product((False, True), repeat=3):
                u = t
                for ax, f in enumerate(flips):
                    if f:
                        u = np.flip(u, ax)
                assert orc.simple_3d(np.ascontiguousarray(u)) == s


def _candidates(orc, p, L, idx, l, c, g):
    out = []
    k = 0
    N = idx.size
    while k < N:
        e = k
        while e < N and idx[e] == idx[k]:
            e += 1
        best = min(range(k, e), key=lambda j: (g[j], c[j]))
        if g[best] < 0 and orc.admissible(p, L, int(idx[best]), int(l[best]), int(c[best])):
            out.append((float(g[best]), int(idx[best]), int(c[best])))
        k = e
    return out


def _rounds_select(cands, shape, rng):
    """Accept a candidate once all smaller Chebyshev neighbours are decided and none is accepted."""
    key = {i: (g, i) for g, i, _ in cands}
    coord = {i: np.unravel_index(i, shape) for _, i, _ in cands}
    nbrs = {i: [j for j in key if j != i and max(abs(a - b) for a, b in zip(coord[i], coord[j])) <= 1]
            for i in key}
    state = {i: 0 for i in key}      # 0 undecided, 1 accepted, 2 rejected
    while any(v == 0 for v in state.values()):
        order = [i for i in key if state[i] == 0]
        rng.shuffle(order)
        for i in order:
            smaller = [j for j in nbrs[i] if key[j] < key[i]]
            if any(state[j] == 1 for j in smaller):
                state[i] = 2
            elif all(state[j] == 2 for j in smaller):
                state[i] = 1
    return sorted(i for i, v in state.items() if v == 1)


@pytest.mark.parametrize("shape,seed", [((20, 22), 0), ((24, 24), 1), ((8, 9, 10), 2)])
def test_select_equals_order_free_rounds(orc, shape, seed):
    rng = np.random.default_rng(seed)
    L = np.zeros(shape, np.int32)
    if len(shape) == 2:
        L[4:14, 3:12] = 1
        L[9:18, 13:19] = 2
    else:
        L[2:6, 2:7, 2:6] = 1
        L[3:7, 5:9, 5:9] = 2
    I = rng.normal(0, 1, shape).astype(np.float32)
    p = orc.make_params(I, L, cutoff=2.0, nlabels=3)
    idx, l, c = orc.extract(p, L)
    g = rng.normal(-0.3, 1.0, idx.size)
    g[1::6] = g[0::6][: g[1::6].size]     # exact ties between neighbours, broken by pixel index
    acc_idx, acc_c, ncand = orc.select(p, L, idx, l, c, g)
    cands = _candidates(orc, p, L, idx, l, c, g)
    assert ncand == len(cands)
    for trial in range(3):
        assert _rounds_select(cands, shape, np.random.default_rng(trial)) == sorted(acc_idx.tolist())
    # independence and greedy maximality
    acc = set(acc_idx.tolist())
    coords = {i: np.unravel_index(i, shape) for i in acc}
    for i, j in itertools.combinations(acc, 2):
        assert max(abs(a - b) for a, b in zip(coords[i], coords[j])) > 1
    cmap = {i: cc for _, i, cc in cands}
    for i, cc in zip(acc_idx.tolist(), acc_c.tolist()):
        assert cmap[i] == cc


def _label_components_ok(L, conn, labels):
    st = CROSS2 if L.ndim == 2 else CROSS3
    for m in labels:
        if m == 0:
            continue
        X = L == m
        if X.any():
            assert ndimage.label(X, structure=st)[1] == 1, m


def _holes(L, labels):
    fs = FULL2 if L.ndim == 2 else FULL3
    out = {}
    for m in labels:
        if m:
            out[m] = ndimage.label(np.pad(L != m, 1, constant_values=True), structure=fs)[1]
    return out


@pytest.mark.parametrize("case", ["disks", "grid2d", "grid3d", "ps"])
def test_iterations_keep_invariants(orc, case):
    from paper_1403_0240_gb300 import synth
    if case == "disks":
        w = synth.disks()
        iters = 50
    elif case == "grid2d":
        w = synth.disks(96, 100, seed=5)
        w.labels0 = synth.square_grid_labels(96, 100, 24, 12)
        iters = 25
    elif case == "grid3d":
        w = synth.ellipsoids(24, 26, 28, seed=6)
        w.labels0 = synth.cube_grid_labels(24, 26, 28, 12, 6)
        iters = 12
    else:
        w = synth.ellipses(128, 128, seed=7)
        w.labels0 = synth.square_grid_labels(128, 128, 32, 16)
        iters = 10
    p = orc.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius)
    run = orc.Run(p, w.image, w.labels0)
    labels = range(int(w.labels0.max()) + 1)
    holes0 = _holes(run.L, labels)
    counts0 = np.bincount(run.L.ravel(), minlength=len(labels))
    for _ in range(iters):
        before = run.L.copy()
        s, _ = run.step()
        assert (before != run.L).sum() == s["n_accepted"]
        _label_components_ok(run.L, w.connectivity, labels)
        assert _holes(run.L, labels) == holes0
        counts = np.bincount(run.L.ravel(), minlength=len(labels))
        assert counts.sum() == counts0.sum() and (counts[1:] > 0).all()


def test_iterate_applies_the_mode_rule(orc):
    # a whole run switches and converges exactly where the hand-pinned rule (orc_advance_mode,
    # tests/golden/osc_switch.txt) puts it for the run's own accepted-move counts
    from paper_1403_0240_gb300 import synth
    w = synth.disks()
    p = orc.make_params(w.image, w.labels0, "pc", 4, 0.04, 3.0, osc_window=4)
    run = orc.Run(p, w.image, w.labels0)
    got, acc = [], []
    for t in range(400):
        s, _ = run.step()
        got.append((s["mode_used"], s["converged"]))
        acc.append(s["n_accepted"])
    assert got == orc.mode_sequence(4, acc)
    assert got[-1] == (1, 1), "the L2 fallback converges on this scene"
    assert any(m == 0 for m, _ in got) and any(m == 1 for m, _ in got)


def test_degenerate_sobolev_run_equals_l2_run(orc):
    from paper_1403_0240_gb300 import synth
    w = synth.disks()
    pa = orc.make_params(w.image, w.labels0, "pc", 4, 0.04, 1.0, gradient="sobolev")
    pb = orc.make_params(w.image, w.labels0, "pc", 4, 0.04, 1.0, gradient="l2")
    ra, rb = orc.Run(pa, w.image, w.labels0), orc.Run(pb, w.image, w.labels0)
    for _ in range(30):
        ra.step()
        rb.step()
        assert np.array_equal(ra.L, rb.L)


def _rect_labels(shape, seed, n_rect=12):
    """Random non-overlapping rectangles (some 1x1) on background 0: every label one component."""
    rng = np.random.default_rng(seed)
    L = np.zeros(shape, np.int32)
    lab = 1
    for _ in range(200):
        if lab > n_rect:
            break
        h, w = (1, 1) if rng.random() < 0.4 else tuple(rng.integers(1, 5, 2))
        y, x = rng.integers(0, shape[0] - h + 1), rng.integers(0, shape[1] - w + 1)
        y0, y1, x0, x1 = max(0, y - 1), min(shape[0], y + h + 1), max(0, x - 1), min(shape[1], x + w + 1)
        if (L[y0:y1, x0:x1] != 0).any():
            continue
        L[y:y + h, x:x + w] = lab
        lab += 1
    return L


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_vanishing_admits_exactly_the_last_pixels(orc, seed):
    L = _rect_labels((24, 26), seed)
    I = np.zeros(L.shape, np.float32)
    strict = orc.make_params(I, L, "pc", topology=0)
    vanish = orc.make_params(I, L, "pc", topology=1)
    counts = np.bincount(L.ravel())
    singles = 0
    for x in range(L.size):
        l = int(L.flat[x])
        if l == 0:
            continue
        a0 = orc.admissible(strict, L, x, l, 0)
        a1 = orc.admissible(vanish, L, x, l, 0)
        if counts[l] == 1:
            singles += 1
            assert not a0 and a1          # an isolated region: only vanishing removes it
        else:
            assert a0 == a1               # everything else is unchanged
    assert singles > 0


def test_a_one_pixel_region_vanishes_only_when_allowed(orc):
    I = np.zeros((20, 20), np.float32)
    L = np.zeros((20, 20), np.int32)
    L[10, 10] = 1                          # a one-pixel region in a flat background
    L[2:6, 2:6] = 2
    for topology, gone in [(0, False), (1, True)]:
        p = orc.make_params(I, L, "pc", lam=0.5, cutoff=1.0, topology=topology, nlabels=3)
        run = orc.Run(p, I, L)
        run.step()
        assert (int((run.L == 1).sum()) == 0) == gone


@pytest.mark.parametrize("shape,seed", [((30, 34), 0), ((30, 34), 1), ((9, 10, 11), 2)])
def test_relabel_matches_connected_components(orc, shape, seed):
    # random blobs where several labels are split into pieces; the relabelling must leave one
    # component per label, keep each label on the piece with its smallest pixel index, and number
    # the other pieces upward in ascending order of their smallest pixel indices
    rng = np.random.default_rng(seed)
    L = (rng.random(shape) < 0.45).astype(np.int32) * rng.integers(1, 5, shape).astype(np.int32)
    st = CROSS2 if L.ndim == 2 else CROSS3
    p = orc.make_params(np.zeros(shape, np.float32), L, "pc", nlabels=5, topology=2)
    out, n = orc.relabel(p, L, 5)
    pieces = []                                     # (smallest index, label, mask) of every piece
    for m in range(1, 5):
        lab, k = ndimage.label(L == m, structure=st)
        for c in range(1, k + 1):
            mask = lab == c
            pieces.append((int(np.flatnonzero(mask.ravel())[0]), m, mask))
    pieces.sort(key=lambda t: t[0])
    first = {}
    nxt = 5
    expect = L.copy()
    for lo, m, mask in pieces:
        if m not in first:
            first[m] = lo
        else:
            expect[mask] = nxt
            nxt += 1
    assert n == nxt
    assert np.array_equal(out, expect)
    assert np.array_equal(out == 0, L == 0)


def test_split_admits_the_neck_of_a_dumbbell(orc):
    L = np.zeros((12, 20), np.int32)
    L[3:9, 2:8] = 1
    L[3:9, 12:18] = 1
    L[6, 8:12] = 1                                  # a one-pixel-wide neck
    I = np.zeros(L.shape, np.float32)
    x = 6 * 20 + 10                                  # a neck pixel
    strict = orc.make_params(I, L, "pc", nlabels=2, topology=0)
    split = orc.make_params(I, L, "pc", nlabels=2, topology=2)
    assert not orc.admissible(strict, L, x, 1, 0)
    assert orc.admissible(split, L, x, 1, 0)
    corner = 3 * 20 + 2                              # a simple point stays admissible either way
    assert orc.admissible(strict, L, corner, 1, 0) and orc.admissible(split, L, corner, 1, 0)
    inner = 5 * 20 + 4                               # removing an interior pixel would make a hole
    assert not orc.admissible(strict, L, inner, 1, 0) and not orc.admissible(split, L, inner, 1, 0)


@pytest.mark.parametrize("topology", [2, 3])
def test_split_iterations_keep_one_component_per_label(orc, topology):
    from paper_1403_0240_gb300 import synth
    # one label over two disks joined by a thin bridge of background intensity: the bridge
    # pixels leave the region and the region splits into two labels
    w = synth.disks(96, 128, seed=3)
    I = np.zeros((96, 128), np.float32)
    I[20:76, 10:50] = 1.0
    I[20:76, 78:118] = 1.0
    L = np.zeros(I.shape, np.int32)
    L[30:66, 18:110] = 1                             # one rectangle across both blobs
    p = orc.make_params(I + w.image * 0.1, L, "pc", 4, 0.02, 3.0, topology=topology, nlabels=2)
    run = orc.Run(p, I + w.image * 0.1, L)
    total = L.size
    for _ in range(40):
        run.step()
        n = run.state()["nlabels"]
        counts = np.bincount(run.L.ravel(), minlength=n)
        assert counts.sum() == total
        for m in range(1, n):
            if counts[m]:
                assert ndimage.label(run.L == m, structure=CROSS2)[1] == 1
    assert run.state()["nlabels"] >= 3                # the region has split
