"""Band plans of the symmetric products, on the host (pb_sym_band_plan; no GPU).

The symmetric products evaluate the upper triangle of square tile pairs
(I <= J, numbered row by row) in bands of whole row tiles.  These tests check
the library's plan and, by restating the kernels' index arithmetic (the tile
pair numbering, the persistent CTAs' equal ranges, the offsets of a band's
column sides and split-row slots) in Python, that a banded product covers
every tile pair once, stays inside its buffers, and gives every row each of
its row sides and column sides exactly once.  The figures pinned at 81,920
and 300,176 triangles are the ones the GPU reported for those contexts.
"""
import pytest

pb = pytest.importorskip("paper_1301_5885_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import importlib
    importlib.import_module("paper_1301_5885_gb300.build").build()


# ---- the kernels' index arithmetic, restated ---------------------------------
def row_start(i, tiles):
    return i * tiles - i * (i - 1) // 2


def row_of(p, tiles):
    lo, hi = 0, tiles - 1
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if row_start(mid, tiles) <= p:
            lo = mid
        else:
            hi = mid - 1
    return lo


def offdiag(i, j, tiles):
    return row_start(i, tiles) + (j - i) - i - 1


def sk_begin(c, w, g):
    return (c * w) // g


def sk_cta_of(p, w, g):
    return ((p + 1) * g + w - 1) // w - 1


def band_slots(tiles, r0, r1):
    return (row_start(r1, tiles) - r1) - (row_start(r0, tiles) - r0)


def emulate(tiles, ctas, cuts):
    """Run the banded schedule on index level; return the set of covered tile pairs."""
    work = tiles * (tiles + 1) // 2
    g_full = min(ctas, work)
    slots = max(band_slots(tiles, a, b) for a, b in zip(cuts, cuts[1:]))
    covered = set()
    colacc = {}
    for r0, r1 in zip(cuts, cuts[1:]):
        wb = row_start(r0, tiles)
        w = row_start(r1, tiles) - wb
        joff = wb - r0
        g = min(g_full, w)
        jpart, islots, iside = {}, {}, {}
        for c in range(g):
            p, pend = wb + sk_begin(c, w, g), wb + sk_begin(c + 1, w, g)
            if p >= pend:
                continue
            i_first = row_of(p, tiles)
            while p < pend:
                i = row_of(p, tiles)
                row_end = row_start(i + 1, tiles)
                stop = min(pend, row_end)
                assert r0 <= i < r1
                seg = []
                for q in range(p, stop):
                    j = i + (q - row_start(i, tiles))
                    assert i <= j < tiles and (i, j) not in covered
                    covered.add((i, j))
                    seg.append(j)
                    if j != i:
                        k = offdiag(i, j, tiles) - joff
                        assert 0 <= k < slots and k not in jpart
                        jpart[k] = (i, j)
                p = stop
                c0, c1 = sk_cta_of(row_start(i, tiles) - wb, w, g), sk_cta_of(row_end - 1 - wb, w, g)
                if c0 == c1:
                    assert i not in iside
                    iside[i] = seg
                else:
                    s = 2 * c + (0 if i == i_first else 1)
                    assert s < 2 * g_full and s not in islots
                    islots[s] = (i, seg)
        # the finishing kernel: rows of the band, folds of the later row tiles
        for r in range(r0, tiles):
            parts = []
            for ip in range(r0, min(r, r1)):
                k = offdiag(ip, r, tiles) - joff
                assert 0 <= k < slots and jpart[k] == (ip, r)
                parts.append(ip)
            if r >= r1:
                colacc[r] = (colacc.get(r, []) if r0 > 0 else []) + parts
                continue
            c0 = sk_cta_of(row_start(r, tiles) - wb, w, g)
            c1 = sk_cta_of(row_start(r + 1, tiles) - 1 - wb, w, g)
            if c0 == c1:
                rows = iside[r]
            else:
                rows = []
                for cc in range(c0, c1 + 1):
                    first = row_of(wb + sk_begin(cc, w, g), tiles)
                    i, seg = islots[2 * cc + (0 if r == first else 1)]
                    assert i == r
                    rows += seg
            cols = (colacc.get(r, []) if r0 > 0 else []) + parts
            assert sorted(rows) == list(range(r, tiles))       # row sides (r, j), j >= r, once each
            assert sorted(cols) == list(range(r))              # column sides (i, r), i < r, once each
    assert len(covered) == work
    return covered


def _check_cuts(cuts, tiles):
    assert cuts[0] == 0 and cuts[-1] == tiles
    assert all(a < b for a, b in zip(cuts, cuts[1:]))


# ---- the plan ------------------------------------------------------------------
@pytest.mark.parametrize("n,tile,ctas,bands_expected,bytes_expected", [
    (300_176, 512, 456, 79, 44_122_112),     # the benchmark solute, default plan
    (81_920, 512, 456, 6, 38_248_448),       # the 81,920-triangle sphere
    (20_416, 512, 456, 1, None),             # too little work per CTA for bands
])
def test_default_plans_pinned_to_the_gpu_contexts(n, tile, ctas, bands_expected, bytes_expected):
    cuts, nbytes = pb.pb_sym_band_plan(n, tile, ctas, 4, 1 << 30, 0)
    _check_cuts(cuts, -(-n // tile))
    assert len(cuts) - 1 == bands_expected
    if bytes_expected is not None:
        assert nbytes == bytes_expected


def test_one_pass_scratch_is_the_column_sides_of_every_tile_pair():
    cuts, nbytes = pb.pb_sym_band_plan(300_176, 512, 456, 4, 0, 1)
    assert cuts == [0, 587]
    assert nbytes == 716_754_944       # reported by the GPU context in one pass
    tiles, b = 587, 512
    r256 = lambda x: (x + 255) // 256 * 256
    assert nbytes == r256(tiles * 2 * b * 8) + r256(456 * 4 * b * 8) + r256(tiles * (tiles - 1) // 2 * 2 * b * 4)


@pytest.mark.parametrize("elem", [4, 8])
@pytest.mark.parametrize("limit_mib", [600, 200, 100, 50, 30])
def test_a_bound_is_met_or_one_row_per_band(elem, limit_mib):
    n, tile, ctas = 300_176, 512 if elem == 4 else 256, 456
    limit = limit_mib << 20
    one = pb.pb_sym_band_plan(n, tile, ctas, elem, 0, 1)[1]
    cuts, nbytes = pb.pb_sym_band_plan(n, tile, ctas, elem, limit, 1)
    tiles = -(-n // tile)
    _check_cuts(cuts, tiles)
    if one <= limit:
        assert cuts == [0, tiles]
    elif len(cuts) - 1 < tiles - 1:
        assert nbytes <= limit
    assert nbytes <= one


def test_unrequested_bands_never_need_more_scratch_than_one_pass():
    for n in (16_384, 30_000, 48_000, 60_000, 81_920, 150_000):
        for tile, ctas in ((256, 608), (512, 456)):
            one = pb.pb_sym_band_plan(n, tile, ctas, 4, 0, 1)[1]
            for limit in (0, 1, one // 2, 1 << 30):
                assert pb.pb_sym_band_plan(n, tile, ctas, 4, limit, 0)[1] <= one


@pytest.mark.parametrize("req", [2, 3, 4, 7, 10_000])
def test_requested_bands(req):
    for n, tile in ((20_416, 512), (20_416, 256), (9_000, 128)):
        tiles = -(-n // tile)
        cuts, _ = pb.pb_sym_band_plan(n, tile, 456, 4, 0, req)
        _check_cuts(cuts, tiles)
        assert len(cuts) - 1 >= min(req, tiles - 1)


@pytest.mark.parametrize("tiles", [1, 2, 3, 7, 12, 19])
@pytest.mark.parametrize("ctas", [1, 3, 5, 16, 40, 1000])
def test_banded_schedules_cover_every_pair_once(tiles, ctas):
    """Every band request from one pass to one row tile per band, on the
    kernels' index arithmetic."""
    n = tiles * 128 - 5 if tiles > 1 else 100
    for req in (1, 2, 3, 5, 1000):
        cuts, _ = pb.pb_sym_band_plan(n, 128, ctas, 4, 0, req)
        _check_cuts(cuts, tiles)
        emulate(tiles, ctas, cuts)


def test_bad_arguments_are_rejected():
    for args in ((0, 512, 456, 4), (1000, 100, 456, 4), (1000, 512, 0, 4), (1000, 512, 456, 2)):
        with pytest.raises(pb.PBError):
            pb.pb_sym_band_plan(*args)
