"""Pins of the CPU oracle to facts the paper and the mathematics fix.

None of these compares the oracle with itself: each expected value comes
from a closed form, exact rational arithmetic, a worked example printed in
the paper, or the O(n^2) definition checked against the grid search.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1803_04120_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lattice(m: int, d: int, spacing: float = 1.0, origin: float = 0.0) -> np.ndarray:
    """All points of the m^d integer lattice (times spacing)."""
    axes = [np.arange(m, dtype=np.float64) * spacing + origin] * d
    grid = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.ravel() for g in grid], axis=1)


def keys_to_pairs(keys):
    keys = np.asarray(keys, dtype=np.uint64)
    return (keys >> np.uint64(32)).astype(np.int64), (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)


# ---------------------------------------------------------------- predicate

def rn(x: Fraction) -> Fraction:
    """Round a rational to the nearest double (ties to even)."""
    return Fraction(float(x))


def exact_predicate(a, b, eps) -> bool:
    """The Section III predicate evaluated with exact rationals, rounding
    each operation to double on its own: sub, square, add, left to right."""
    s = Fraction(0)
    for x, y in zip(a, b):
        t = rn(Fraction(x) - Fraction(y))
        s = rn(s + rn(t * t))
    return s <= rn(Fraction(eps) * Fraction(eps))


def test_predicate_matches_exact_rounding_near_threshold():
    rng = np.random.default_rng(11)
    for d in (1, 2, 3, 6, 8):
        for _ in range(300):
            a = rng.uniform(-50, 50, d)
            dirn = rng.normal(size=d)
            dirn /= np.linalg.norm(dirn)
            eps = float(rng.uniform(0.1, 10))
            # b at distance eps*(1 +- a few ulps) from a
            b = a + dirn * eps * (1.0 + float(rng.integers(-8, 9)) * 2.0 ** -52)
            assert orc.within(a, b, eps) == exact_predicate(a, b, eps)


def test_predicate_is_not_contracted_to_fma():
    # Found by exhaustive search with exact rationals: with t = (a0, a1),
    # fl(fl(a0^2) + fl(a1^2)) lies one ulp above fl(eps^2), while the
    # contracted form fma(a1, a1, fl(a0^2)) lies on it.  Without contraction
    # the pair is not a member.
    a = [0.9433567169983137, 0.6489745531369242]
    b = [0.0, 0.0]
    eps = 1.1450283254684606
    t0, t1 = Fraction(a[0]), Fraction(a[1])
    nofma = rn(rn(t0 * t0) + rn(t1 * t1))
    fma = rn(rn(t0 * t0) + t1 * t1)
    E2 = rn(Fraction(eps) ** 2)
    assert nofma > E2 >= fma
    assert orc.within(a, b, eps) is False
    assert exact_predicate(a, b, eps) is False


def test_inclusive_at_exact_distance():
    # integer coordinates: every squared distance is exact; dist == eps is a member
    assert orc.within([0.0, 0.0], [3.0, 4.0], 5.0)
    assert not orc.within([0.0, 0.0], [3.0, 4.0], 5.0 - 2.0 ** -40)


# ---------------------------------------------------------------- lattices

@pytest.mark.parametrize("d,m", [(1, 9), (2, 7), (3, 5), (4, 4), (5, 3)])
def test_unit_lattice_closed_form(d, m):
    # spacing 1, eps = 1: each point pairs with itself and its 2d axis
    # neighbours that exist; total = m^d + 2 d (m-1) m^(d-1).
    pts = lattice(m, d)
    expect = m ** d + 2 * d * (m - 1) * m ** (d - 1)
    bf = orc.bruteforce(pts, 1.0)
    gj = orc.grid_join(pts, 1.0)
    assert bf.size == expect
    assert np.array_equal(bf, gj)
    # interior points have exactly 2d + 1 members
    i, _ = keys_to_pairs(bf)
    deg = np.bincount(i, minlength=len(pts))
    interior = np.all((pts > 0) & (pts < m - 1), axis=1)
    if interior.any():
        assert np.all(deg[interior] == 2 * d + 1)


@pytest.mark.parametrize("d,m", [(10, 2), (12, 2), (9, 3)])
def test_unit_lattice_closed_form_beyond_8_dimensions(d, m):
    # the brute-force definition, which checks the joins of more than 8
    # dimensions, against the same closed form
    pts = lattice(m, d)
    bf = orc.bruteforce(pts, 1.0)
    assert bf.size == m ** d + 2 * d * (m - 1) * m ** (d - 1)
    i, j = keys_to_pairs(bf)
    # every member pair differs by exactly 1 in one coordinate, or is a self-pair
    diff = np.abs(pts[i] - pts[j]).sum(axis=1)
    assert np.all((diff == 0) | (diff == 1))


@pytest.mark.parametrize("d,m", [(2, 6), (3, 4)])
def test_lattice_just_below_spacing_gives_only_self_pairs(d, m):
    pts = lattice(m, d, spacing=1.0, origin=-3.0)
    eps = 1.0 - 2.0 ** -40
    for res in (orc.bruteforce(pts, eps), orc.grid_join(pts, eps)):
        i, j = keys_to_pairs(res)
        assert res.size == m ** d and np.all(i == j)


def test_2d_lattice_with_rounded_sqrt2_includes_diagonals():
    # fl(sqrt 2)^2 rounds above 2, so diagonal neighbours (s = 2 exactly) are
    # members: an interior point has 9 members, total
    # m^2 + 4 m (m-1) + 4 (m-1)^2.  Just below sqrt 2 they are not.
    m = 6
    pts = lattice(m, 2)
    eps = math.sqrt(2.0)
    assert rn(Fraction(eps) ** 2) > 2
    expect = m * m + 4 * m * (m - 1) + 4 * (m - 1) ** 2
    assert orc.bruteforce(pts, eps).size == expect
    assert orc.grid_join(pts, eps).size == expect
    below = float(np.nextafter(eps, 0.0))
    assert rn(Fraction(below) ** 2) < 2
    assert orc.grid_join(pts, below).size == m ** 2 + 4 * m * (m - 1)


# ---------------------------------------------------------------- invariants

def check_symmetric_with_self(keys, n):
    i, j = keys_to_pairs(keys)
    assert np.all(np.diff(keys.astype(np.uint64).view(np.int64)) > 0) or keys.size <= 1
    swapped = np.sort((j.astype(np.uint64) << np.uint64(32)) | i.astype(np.uint64))
    assert np.array_equal(swapped, keys)
    selfs = keys[i == j]
    assert selfs.size == n
    assert (keys.size - n) % 2 == 0


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8])
def test_grid_equals_bruteforce_random(d):
    rng = np.random.default_rng(100 + d)
    for trial in range(4):
        n = int(rng.integers(1, 400))
        scale = float(rng.choice([1.0, 10.0, 1000.0]))
        pts = rng.uniform(-scale, scale, size=(n, d))
        if trial == 1:
            pts[n // 2:] = pts[: n - n // 2]          # duplicate points
        if trial == 2:
            pts = np.round(pts)                       # many exact ties
        eps = float(scale * rng.choice([0.01, 0.1, 0.5, 3.0]))
        bf = orc.bruteforce(pts, eps)
        gj = orc.grid_join(pts, eps, nthreads=3)
        assert np.array_equal(bf, gj), (d, trial, n, eps)
        check_symmetric_with_self(bf, n)


def test_points_on_cell_boundaries():
    # points planted exactly eps apart across cell boundaries, and at
    # eps*(1 +- 1 ulp), in every dimension
    rng = np.random.default_rng(7)
    for d in (2, 3, 5):
        eps = 0.3
        base = rng.uniform(0, 3, size=(60, d))
        extra = []
        for p in base:
            k = int(rng.integers(0, d))
            for f in (1.0, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -52):
                q = p.copy()
                q[k] += eps * f
                extra.append(q)
        pts = np.concatenate([base, np.array(extra)])
        assert np.array_equal(orc.bruteforce(pts, eps), orc.grid_join(pts, eps))


def test_digest_and_neighbors_agree_with_bruteforce():
    pts = datagen.uniform(3000, 3, seed=5) / 10.0
    eps = 0.9
    bf = orc.bruteforce(pts, eps)
    cnt, deg, h = orc.grid_digest(pts, eps, nthreads=4)
    i, _ = keys_to_pairs(bf)
    assert cnt == bf.size
    assert np.array_equal(deg, np.bincount(i, minlength=len(pts)).astype(np.uint32))
    assert h == orc.pair_hash(bf)
    # mix64 matches the published splitmix64 finaliser on a known value:
    # splitmix64 seeded with 0 first outputs 0xE220A8397B1DCDAF = mix64(G)
    assert orc.mix64(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF
    q = np.array([0, 17, 2999, 1234], dtype=np.uint32)
    offs, ids = orc.grid_neighbors(pts, eps, q)
    for k, qq in enumerate(q):
        want = bf[i == qq] & np.uint64(0xFFFFFFFF)
        assert np.array_equal(ids[offs[k]:offs[k + 1]].astype(np.uint64), want)


def test_invalid_inputs_rejected():
    pts = np.zeros((4, 2))
    with pytest.raises(ValueError):
        orc.grid_join(pts, 0.0)
    with pytest.raises(ValueError):
        orc.grid_join(pts, float("nan"))
    bad = pts.copy()
    bad[1, 1] = np.inf
    with pytest.raises(ValueError):
        orc.grid_join(bad, 1.0)


# ---------------------------------------------------------------- worked example

def test_worked_example_section_4d():
    fx = json.load(open(os.path.join(GOLDEN, "worked_example_sec4d.json")))
    pts = np.array(fx["points"], dtype=np.float64)
    paper = fx["paper"]
    ng, cells = orc.grid_cells(pts, fx["eps"])
    assert list(ng) == paper["cells_per_dim"]
    ids = sorted(set(int(c) for c in cells))
    assert len(ids) == paper["non_empty_cells"]
    assert ids == fx["constructed"]["non_empty_linear_ids"]
    # C_h numbering is 1-based in lexicographic order of linear ids
    assert ids.index(paper["query_cell_linear_id"]) + 1 == paper["query_cell_rank_1based"]
    assert ids[6 - 1] == paper["C6_linear_id"]
    assert sorted(np.nonzero(cells == paper["C6_linear_id"])[0].tolist()) == sorted(paper["C6_points"])
    # id 30 decodes to column 2, row 4 with dimension 1 fastest
    qid = paper["query_cell_linear_id"]
    cx, cy = qid % ng[0], qid // ng[0]
    assert (cx, cy) == (2, 4)
    assert [[cx - 1, cx + 1], [cy - 1, cy + 1]] == paper["O"]
    occupied_x = sorted(set(int(c) % ng[0] for c in cells))
    occupied_y = sorted(set(int(c) // ng[0] for c in cells))
    ocm = [[x for x in range(cx - 1, cx + 2) if x in occupied_x],
           [y for y in range(cy - 1, cy + 2) if y in occupied_y]]
    assert [[r[0], r[-1]] for r in ocm] == paper["O_cap_M"]
    cand = [x + ng[0] * y for y in ocm[1] for x in ocm[0]]
    assert sorted(cand) == paper["candidate_linear_ids"]
    assert [c for c in sorted(cand) if c in ids] == paper["non_empty_candidates"]


# ---------------------------------------------------------------- statistics

def test_uniform_square_mean_neighbours_closed_form():
    # Two independent uniform points in an L x L square are within eps
    # (eps <= L) with probability (pi eps^2 L^2 - 8/3 eps^3 L + eps^4 / 2) / L^4.
    # The 20,000-point, eps = 2 workload therefore has an expected member
    # count of n + n (n - 1) P; the realised count must agree within 1.5 %.
    cfg = datagen.CONFIG1
    pts = datagen.make_points(cfg)
    L, eps, n = 100.0, cfg["eps"], cfg["n"]
    P = (math.pi * eps ** 2 * L ** 2 - 8.0 / 3.0 * eps ** 3 * L + eps ** 4 / 2.0) / L ** 4
    expect = n + n * (n - 1) * P
    cnt, _, _ = orc.grid_digest(pts, eps, with_degree=False)
    assert abs(cnt - expect) / expect < 0.015, (cnt, expect)


@pytest.mark.slow
def test_config1_grid_equals_bruteforce():
    cfg = datagen.CONFIG1
    pts = datagen.make_points(cfg)
    bf = orc.bruteforce(pts, cfg["eps"])
    gj = orc.grid_join(pts, cfg["eps"])
    assert np.array_equal(bf, gj)
    check_symmetric_with_self(bf, cfg["n"])


# ---------------------------------------------------------------- UNICOMP reading

def unicomp_visits(c, ng, guard_dims=None):
    """Cells a UNICOMP home cell c visits, by the n-dimensional rule of
    Section V-B: stage k runs when coordinate k of c is odd and visits the
    cells whose coordinates below k range over c +- 1, whose coordinate k
    differs from c's by one, and whose coordinates above k equal c's.
    guard_dims[k] names the coordinate whose parity guards stage k (the
    paper's text uses k itself; its 3-D listing prints y for the z stage)."""
    d = len(c)
    out = []
    for k in range(d):
        g = k if guard_dims is None else guard_dims[k]
        if c[g] % 2 == 0:
            continue
        ranges = [range(c[j] - 1, c[j] + 2) for j in range(k)]
        ranges.append([c[k] - 1, c[k] + 1])
        for idx in np.ndindex(*[len(r) for r in ranges]):
            b = [ranges[j][idx[j]] for j in range(k + 1)] + list(c[k + 1:])
            if all(0 <= b[j] < ng[j] for j in range(d)):
                out.append(tuple(b))
    return out


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_unicomp_visits_each_adjacent_cell_pair_once(d):
    rng = np.random.default_rng(300 + d)
    ng = [int(rng.integers(3, 7)) for _ in range(d)]
    cells = [tuple(int(x) for x in c) for c in np.ndindex(*ng) if rng.random() < 0.6]
    occ = set(cells)
    seen = {}
    for a in cells:
        for b in unicomp_visits(a, ng):
            if b in occ:
                key = frozenset((a, b))
                seen[key] = seen.get(key, 0) + 1
    adjacent = set()
    for a in cells:
        for b in cells:
            if a != b and max(abs(x - y) for x, y in zip(a, b)) <= 1:
                adjacent.add(frozenset((a, b)))
    assert set(seen) == adjacent
    assert all(v == 1 for v in seen.values())
    # each visit comes from exactly one of its two cells: work halves
    full = sum(1 for a in cells for b in cells if a != b and max(abs(x - y) for x, y in zip(a, b)) <= 1)
    assert 2 * sum(seen.values()) == full


def test_unicomp_3d_listing_guard_as_printed_misses_pairs():
    # The 3-D listing guards its third stage with "y is odd"; read literally
    # it visits some pairs twice and others never, so the z stage must be
    # guarded by z (as the prose says).
    ng = [4, 4, 4]
    cells = list(np.ndindex(*ng))
    seen = {}
    for a in cells:
        for b in unicomp_visits(a, ng, guard_dims=[0, 1, 1]):
            key = frozenset((a, b))
            seen[key] = seen.get(key, 0) + 1
    n_adjacent = sum(1 for a in cells for b in cells
                     if a < b and max(abs(x - y) for x, y in zip(a, b)) <= 1)
    assert len(seen) < n_adjacent or any(v != 1 for v in seen.values())


# ------------------------------------------------------------------ two-set join
# The two-set oracle is pinned to the self-join definition: R ⋈ R is the
# self-join, the self-join of R ∪ S decomposes into R ⋈ R, S ⋈ S, R ⋈ S and
# S ⋈ R, swapping the sets swaps the pairs, and boundary points follow the
# inclusive predicate.

def _split_keys(keys):
    return keys >> np.uint64(32), keys & np.uint64(0xffffffff)


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
def test_join2_of_a_set_with_itself_is_the_self_join(d):
    rng = np.random.default_rng(100 + d)
    r = rng.uniform(0, 5, size=(300, d))
    eps = 1.3
    assert np.array_equal(orc.bruteforce2(r, r, eps), np.sort(orc.bruteforce(r, eps)))


@pytest.mark.parametrize("d", [1, 2, 4, 7])
def test_join2_decomposes_the_self_join_of_the_union(d):
    rng = np.random.default_rng(200 + d)
    r = rng.uniform(0, 6, size=(170, d))
    s = rng.uniform(2, 8, size=(230, d))
    s[:5] = r[:5]                         # coincident points across the sets
    eps = 1.7
    u = np.concatenate([r, s])
    i, j = _split_keys(np.sort(orc.bruteforce(u, eps)))
    nr = np.uint64(len(r))
    cross = (i < nr) & (j >= nr)
    want = np.sort((i[cross] << np.uint64(32)) | (j[cross] - nr))
    got = orc.bruteforce2(r, s, eps)
    assert np.array_equal(got, want)
    # swapping the sets swaps the pairs
    i2, j2 = _split_keys(orc.bruteforce2(s, r, eps))
    assert np.array_equal(np.sort((j2 << np.uint64(32)) | i2), got)


def test_join2_boundary_and_empty():
    r = np.array([[0.0, 0.0]])
    eps = 1.0
    on = np.array([[1.0, 0.0]])                       # distance exactly eps: member
    off = np.array([[np.nextafter(1.0, 2.0), 0.0]])   # one ulp beyond: not
    assert len(orc.bruteforce2(r, on, eps)) == 1
    assert len(orc.bruteforce2(r, off, eps)) == 0
    far = np.array([[10.0, 10.0], [20.0, 0.0]])
    assert len(orc.bruteforce2(r, far, eps)) == 0
