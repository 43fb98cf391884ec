"""The warp-tile row plan of the device layout (lp_plan_rows,
lp_plan_rows_shape), on the host.

Besides the plan's own invariants, a NumPy model of the engine's lane
arithmetic (spmv_warp.cuh: group g of 2^v lanes reduces row p0 + g of a
pass, lane gl of the group touches entries lo + gl + c * 2^v * nit + u * 2^v;
a segment tile's 32 lanes touch entries lo + lane + c * 256 + u * 32 of its
segment) checks that every entry of every row is read exactly once, so a plan
the kernels would mis-cover fails here, without a GPU.
"""
import numpy as np
import pytest

KWARP_ITEMS = 8
KCTA = 512
SHAPES = [(8, 512), (8, 2048), (16, 512), (16, 2048), (32, 512), (32, 2048), (64, 512),
          (64, 2048)]


@pytest.fixture(scope="module")
def pkg():
    import paper_2604_23951_gb300 as p

    p.load()
    return p


def unpack(word):
    return word & 0xFF, (word >> 8) & 0xF, word >> 12


def covered(lo, hi, vl, nit):
    """entries touched by each lane of one group (engine model)"""
    seen = []
    for gl in range(vl):
        k0 = lo + gl
        while k0 < hi:
            for u in range(nit):
                k = k0 + u * vl
                if k < hi:
                    seen.append(k)
            k0 += vl * nit
    return seen


def check_order(lengths, perm):
    lengths = np.asarray(lengths)
    assert sorted(perm.tolist()) == list(range(lengths.size))
    L = lengths[perm]
    # longest first; equal lengths keep their original order
    assert np.all(np.diff(L) <= 0)
    for v in np.unique(L):
        assert np.all(np.diff(perm[L == v]) > 0)
    return L


def check_plan(lengths, perm, tiles, nlong, run_max=8, tile_nnz=512, seg_base=None):
    L = check_order(lengths, perm)
    rows = L.size
    llong = 32 * run_max
    offs = np.concatenate([[0], np.cumsum(L)])
    hit = np.zeros(int(offs[-1]), dtype=np.int64)
    if seg_base is not None:
        nseg_rows = seg_base.size - 1
        assert nlong == 0
        assert np.all(L[:nseg_rows] > llong) and np.all(L[nseg_rows:] <= llong)
        row = nseg_rows
    else:
        assert np.all(L[:nlong] > KCTA) and np.all(L[nlong:] <= KCTA)
        row = nlong
        for r in range(nlong):  # CTA rows: the whole row, one CTA
            hit[offs[r]:offs[r + 1]] += 1
    segs_seen = []
    for r0, word in tiles:
        if word < 0:  # segment tile
            g = int(word) & 0x7FFFFFFF
            r = int(r0)
            assert seg_base is not None and seg_base[r] <= g < seg_base[r + 1]
            s = g - seg_base[r]
            lo = offs[r] + s * llong
            hi = min(lo + llong, offs[r + 1])
            assert lo < hi
            seen = covered(lo, hi, 32, KWARP_ITEMS)
            hit[np.asarray(seen, dtype=np.int64)] += 1
            segs_seen.append(g)
            continue
        nrows, vlog, nit = unpack(int(word))
        assert r0 == row and 1 <= nrows <= 32 and 0 <= vlog <= 5 and 1 <= nit <= KWARP_ITEMS
        vl = 1 << vlog
        rpp = 32 >> vlog
        Lt = L[r0:r0 + nrows]
        if Lt[0] > llong:  # unsegmented long row: a single-row tile
            assert nrows == 1 and vlog == 5
        else:
            # lanes per row: the least 2^v with 2^v * run_max >= L; balanced chunks
            assert vl * run_max >= Lt[0] and (vlog == 0 or (vl // 2) * run_max < Lt[0])
            chunks = max(1, -(-int(Lt[0]) // (vl * KWARP_ITEMS)))
            assert nit == max(1, -(-int(Lt[0]) // (vl * chunks)))
            assert nrows <= max(1, tile_nnz // max(int(Lt[0]), 1))
            if Lt[0] > KWARP_ITEMS:
                assert np.all(2 * Lt >= Lt[0])
        for p0 in range(0, nrows, rpp):
            for gq in range(rpp):
                q = p0 + gq
                if q >= nrows:
                    continue
                lo, hi = offs[r0 + q], offs[r0 + q + 1]
                seen = covered(lo, hi, vl, nit)
                hit[np.asarray(seen, dtype=np.int64)] += 1
        row += nrows
    assert row == rows
    if seg_base is not None:
        assert sorted(segs_seen) == list(range(int(seg_base[-1])))
    assert np.all(hit == 1)


def lengths_mix(rng, rows):
    parts = [rng.integers(0, 9, rows // 2), rng.integers(9, 300, rows // 3),
             rng.lognormal(2.0, 1.2, rows // 6).astype(np.int64)]
    L = np.concatenate(parts + [np.array([0, 1, 256, 257, 512, 513, 1024, 1025, 2048, 2049, 4097, 9000])])
    rng.shuffle(L)
    return L


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_plan_covers_every_entry_once(pkg, seed):
    rng = np.random.default_rng(seed)
    L = lengths_mix(rng, 600)
    perm, tiles, nlong = pkg.plan_rows(L)
    check_plan(L, perm, tiles, nlong)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("segmented", [True, False])
def test_shaped_plans_cover_every_entry_once(pkg, shape, segmented):
    rng = np.random.default_rng(7)
    L = lengths_mix(rng, 900)
    perm, tiles, nlong, sb = pkg.plan_rows_shape(L, shape[0], shape[1], segmented)
    check_plan(L, perm, tiles, nlong, shape[0], shape[1], sb if segmented else None)
    # the row order does not depend on the shape (one stored matrix serves all)
    assert np.array_equal(perm, pkg.plan_rows(L)[0])


def test_plan_edge_cases(pkg):
    for L in ([], [0], [0, 0, 0], [5], [300], [512], [513], [5000], [1] * 70, [8] * 33, [9] * 33,
              [256, 255, 257], list(range(0, 300))):
        L = np.asarray(L, dtype=np.int64)
        perm, tiles, nlong = pkg.plan_rows(L)
        check_plan(L, perm, tiles, nlong)
        for rmax, tnnz in SHAPES:
            perm, tiles, nlong, sb = pkg.plan_rows_shape(L, rmax, tnnz, True)
            check_plan(L, perm, tiles, nlong, rmax, tnnz, sb)


def test_plan_rejects_negative_lengths(pkg):
    with pytest.raises(pkg.LPError):
        pkg.plan_rows(np.array([3, -1]))
    with pytest.raises(pkg.LPError):
        pkg.plan_rows_shape(np.array([3, 1]), 0, 512, True)
