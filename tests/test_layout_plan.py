"""The warp-tile row plan of the device layout (lp_plan_rows), on the host.

Besides the plan's own invariants, a NumPy model of the engine's lane
arithmetic (spmv_warp.cuh: group g of 2^v lanes reduces row p0 + g of a
pass, lane gl of the group touches entries lo + gl + c * 2^v * nit + u * 2^v)
checks that every entry of every row is read exactly once by one group, so
a plan the kernels would mis-cover fails here, without a GPU.
"""
import numpy as np
import pytest

KWARP_ITEMS = 8
KLONG = 32 * KWARP_ITEMS
KCTA = 512


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


def check_plan(lengths, perm, tiles, nlong):
    lengths = np.asarray(lengths)
    rows = lengths.size
    assert sorted(perm.tolist()) == list(range(rows))
    L = lengths[perm]
    assert np.all(L[:nlong] > KCTA) and np.all(L[nlong:] <= KCTA)
    # classes in order, lengths non-increasing after the long classes
    cls = np.where(L > KCTA, 2, np.where(L > KLONG, 1, 0))
    assert np.all(np.diff(cls) <= 0)
    rest = L[cls == 0]
    assert np.all(np.diff(rest) <= 0)
    # stable within a class
    for c in (0, 1, 2):
        idx = perm[cls == c]
        if c == 0:
            for v in np.unique(rest):
                sub = idx[rest == v]
                assert np.all(np.diff(sub) > 0)
        else:
            assert np.all(np.diff(idx) > 0)
    row = nlong
    offs = np.concatenate([[0], np.cumsum(L)])
    for r0, word in tiles:
        nrows, vlog, nit = unpack(int(word))
        assert r0 == row and 1 <= nrows <= 32 and 0 <= vlog <= 5 and 1 <= nit <= KWARP_ITEMS
        vl = 1 << vlog
        rpp = 32 >> vlog
        Lt = L[r0:r0 + nrows]
        if Lt[0] > KLONG:
            assert nrows == 1 and vlog == 5 and nit == KWARP_ITEMS
        else:
            # one chunk covers every row of the tile; lanes per row minimal
            assert vl * nit >= Lt.max()
            assert vlog == 0 or (vl // 2) * KWARP_ITEMS < Lt[0]
            assert nit == max(1, -(-int(Lt[0]) // vl))
        for p0 in range(0, nrows, rpp):
            for g in range(rpp):
                q = p0 + g
                if q >= nrows:
                    continue
                lo, hi = offs[r0 + q], offs[r0 + q + 1]
                seen = covered(lo, hi, vl, nit)
                assert sorted(seen) == list(range(lo, hi))
        row += nrows
    assert row == rows


def lengths_mix(rng, rows):
    parts = [rng.integers(0, 9, rows // 2), rng.integers(9, 300, rows // 3),
             rng.lognormal(2.0, 1.2, rows // 6).astype(np.int64)]
    L = np.concatenate(parts + [np.array([0, 1, 256, 257, 512, 513, 4097, 9000])])
    rng.shuffle(L)
    return L


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_plan_covers_every_entry_once(pkg, seed):
    rng = np.random.default_rng(seed)
    L = lengths_mix(rng, 600)
    perm, tiles, nlong = pkg.plan_rows(L)
    check_plan(L, perm, tiles, nlong)


def test_plan_edge_cases(pkg):
    for L in ([], [0], [0, 0, 0], [5], [300], [512], [513], [5000], [1] * 70, [8] * 33, [9] * 33,
              [256, 255, 257], list(range(0, 300))):
        L = np.asarray(L, dtype=np.int64)
        perm, tiles, nlong = pkg.plan_rows(L)
        check_plan(L, perm, tiles, nlong)


def test_plan_rejects_negative_lengths(pkg):
    with pytest.raises(pkg.LPError):
        pkg.plan_rows(np.array([3, -1]))
