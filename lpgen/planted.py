"""Planted LP instances (problem form of eq. (1); optimality by eq. (2)).

Construction shared by every generator:

* draw x* inside its column bounds, some entries at a bound;
* draw z* with z*_j > 0 only where x*_j sits at a finite lower bound,
  z*_j < 0 only where it sits at a finite upper bound, 0 elsewhere
  (either sign on fixed columns, 0 on free ones);
* draw y* and place the row bounds from (A x*)_i by the sign of y*_i:
  y*_i > 0 -> row_lo_i = (A x*)_i, y*_i < 0 -> row_hi_i = (A x*)_i,
  y*_i = 0 -> (A x*)_i strictly inside, equality rows -> both equal;
* c = A^T y* + z*.

Then (x*, y*, z*) satisfies eq. (2) exactly (up to rounding in forming
A x* and A^T y*), so p* = c^T x* is the optimal value.

Seeds: configuration i uses BASE_SEED + i; item j of a batch or a request
stream uses its configuration seed + 1000 * j.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2604_23951

# column bound kinds
COL_NONNEG, COL_BOX, COL_UPPER, COL_FREE, COL_FIXED, COL_LOWER = range(6)
# row kinds
ROW_EQ, ROW_RANGED, ROW_GE, ROW_LE = range(4)


@dataclass
class PlantedLP:
    """CSR problem data plus the planted optimum."""

    m: int
    n: int
    row_ptr: np.ndarray  # int64, m + 1
    col_idx: np.ndarray  # int32, nnz (sorted within each row, no duplicates)
    val: np.ndarray  # float64, nnz
    c: np.ndarray
    obj_offset: float
    row_lo: np.ndarray
    row_hi: np.ndarray
    col_lo: np.ndarray
    col_hi: np.ndarray
    x_star: np.ndarray | None = None
    y_star: np.ndarray | None = None
    z_star: np.ndarray | None = None
    p_star: float = float("nan")
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def csr(self):
        import scipy.sparse as sp

        return sp.csr_matrix(
            (self.val, self.col_idx.astype(np.int64), self.row_ptr), shape=(self.m, self.n)
        )

    def nbytes(self) -> int:
        return int(
            self.row_ptr.nbytes + self.col_idx.nbytes + self.val.nbytes
            + 5 * 8 * max(self.m, 0) + 3 * 8 * max(self.n, 0)
        )


# ----------------------------------------------------------------------------
# sparsity patterns


def _distinct_cols(rng: np.random.Generator, lengths: np.ndarray, n: int):
    """Row i receives lengths[i] distinct columns drawn uniformly from [0, n)."""
    lengths = np.minimum(lengths.astype(np.int64), n)
    m = lengths.shape[0]
    rows_all = []
    cols_all = []
    need = lengths.copy()
    have_keys = np.empty(0, dtype=np.int64)
    for _ in range(64):
        tot = int(need.sum())
        if tot == 0:
            break
        r = np.repeat(np.arange(m, dtype=np.int64), need)
        cidx = rng.integers(0, n, size=tot, dtype=np.int64)
        keys = np.concatenate([have_keys, r * n + cidx])
        keys.sort()
        keep = np.ones(keys.shape[0], dtype=bool)
        keep[1:] = keys[1:] != keys[:-1]
        keys = keys[keep]
        have_keys = keys
        cnt = np.bincount(keys // n, minlength=m)
        need = np.maximum(lengths - cnt, 0)
        # too many cannot happen: each pass only asks for the deficit
    rows = have_keys // n
    cols = have_keys % n
    rows_all.append(rows)
    cols_all.append(cols)
    return np.concatenate(rows_all), np.concatenate(cols_all)


def _coo_to_csr(m: int, n: int, rows, cols, vals):
    keys = rows.astype(np.int64) * n + cols.astype(np.int64)
    order = np.argsort(keys, kind="stable")
    keys = keys[order]
    keep = np.ones(keys.shape[0], dtype=bool)
    keep[1:] = keys[1:] != keys[:-1]
    keys = keys[keep]
    vals = np.asarray(vals)[order][keep]
    r = keys // n
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=m), out=row_ptr[1:])
    return row_ptr, (keys % n).astype(np.int32), vals.astype(np.float64)


def _row_of(row_ptr):
    m = row_ptr.shape[0] - 1
    return np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))


# ----------------------------------------------------------------------------
# planting


def _plant_columns(rng, kinds, p_low=0.4, p_up=0.2):
    n = kinds.shape[0]
    lo = np.full(n, -np.inf)
    hi = np.full(n, np.inf)
    x = np.zeros(n)
    z = np.zeros(n)
    g = rng.standard_normal(n)
    h = np.abs(rng.standard_normal(n))
    w = np.exp(rng.standard_normal(n)) + 0.5
    u = rng.random(n)
    zmag = np.abs(rng.standard_normal(n)) + 1e-3

    k = kinds == COL_NONNEG
    lo[k] = 0.0
    at = k & (u < p_low)
    x[k] = h[k]
    x[at] = 0.0
    z[at] = zmag[at]

    k = kinds == COL_BOX
    lo[k] = g[k] - 1.0
    hi[k] = lo[k] + w[k]
    at_l = k & (u < p_low * 0.75)
    at_u = k & (u >= p_low * 0.75) & (u < p_low * 0.75 + p_up)
    inner = k & ~at_l & ~at_u
    x[inner] = lo[inner] + w[inner] * (0.1 + 0.8 * rng.random(int(inner.sum())))
    x[at_l] = lo[at_l]
    z[at_l] = zmag[at_l]
    x[at_u] = hi[at_u]
    z[at_u] = -zmag[at_u]

    k = kinds == COL_UPPER
    hi[k] = g[k]
    at = k & (u < p_low)
    x[k] = hi[k] - h[k]
    x[at] = hi[at]
    z[at] = -zmag[at]

    k = kinds == COL_FREE
    x[k] = g[k]

    k = kinds == COL_FIXED
    lo[k] = g[k]
    hi[k] = g[k]
    x[k] = g[k]
    z[k] = rng.standard_normal(int(k.sum()))

    k = kinds == COL_LOWER
    lo[k] = g[k]
    at = k & (u < p_low)
    x[k] = lo[k] + h[k]
    x[at] = lo[at]
    z[at] = zmag[at]
    return lo, hi, x, z


def _plant_rows(rng, kinds, ax, empty_mask=None):
    m = kinds.shape[0]
    lo = np.empty(m)
    hi = np.empty(m)
    y = rng.standard_normal(m)
    s = rng.random(m)
    w1 = np.exp(rng.standard_normal(m)) + 0.1
    w2 = np.exp(rng.standard_normal(m)) + 0.1

    k = kinds == ROW_EQ
    lo[k] = ax[k]
    hi[k] = ax[k]

    k = kinds == ROW_RANGED
    pos = k & (s < 0.3)
    neg = k & (s >= 0.3) & (s < 0.6)
    mid = k & (s >= 0.6)
    y[pos] = np.abs(y[pos]) + 1e-3
    lo[pos] = ax[pos]
    hi[pos] = ax[pos] + w1[pos]
    y[neg] = -np.abs(y[neg]) - 1e-3
    hi[neg] = ax[neg]
    lo[neg] = ax[neg] - w1[neg]
    y[mid] = 0.0
    lo[mid] = ax[mid] - w1[mid]
    hi[mid] = ax[mid] + w2[mid]

    k = kinds == ROW_GE
    act = k & (s < 0.6)
    y[act] = np.abs(y[act]) + 1e-3
    lo[act] = ax[act]
    y[k & ~act] = 0.0
    lo[k & ~act] = ax[k & ~act] - w1[k & ~act]
    hi[k] = np.inf

    k = kinds == ROW_LE
    act = k & (s < 0.6)
    y[act] = -np.abs(y[act]) - 1e-3
    hi[act] = ax[act]
    y[k & ~act] = 0.0
    hi[k & ~act] = ax[k & ~act] + w1[k & ~act]
    lo[k] = -np.inf

    if empty_mask is not None and empty_mask.any():
        y[empty_mask] = 0.0
        # feasible for A x = 0: keep equality rows at 0, widen the others
        e_eq = empty_mask & (kinds == ROW_EQ)
        lo[e_eq] = 0.0
        hi[e_eq] = 0.0
        e_o = empty_mask & (kinds != ROW_EQ)
        lo[e_o] = np.where(np.isfinite(lo[e_o]), -w1[e_o], -np.inf)
        hi[e_o] = np.where(np.isfinite(hi[e_o]), w2[e_o], np.inf)
    return lo, hi, y


def _finish(name, m, n, row_ptr, col_idx, val, row_kinds, col_kinds, rng,
            p_low=0.4, p_up=0.2, meta=None):
    col_lo, col_hi, x, z = _plant_columns(rng, col_kinds, p_low, p_up)
    rows = _row_of(row_ptr)
    ax = np.bincount(rows, weights=val * x[col_idx], minlength=m).astype(np.float64)
    empty = np.diff(row_ptr) == 0
    row_lo, row_hi, y = _plant_rows(rng, row_kinds, ax, empty)
    c = np.bincount(col_idx, weights=val * y[rows], minlength=n).astype(np.float64) + z
    p = float(c @ x)
    return PlantedLP(m=m, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, c=c,
                     obj_offset=0.0, row_lo=row_lo, row_hi=row_hi, col_lo=col_lo,
                     col_hi=col_hi, x_star=x, y_star=y, z_star=z, p_star=p,
                     name=name, meta=meta or {})


# ----------------------------------------------------------------------------
# public generators


def equality_nonneg(m: int, n: int, seed: int, lmin: int = 5, lmax: int = 15,
                    p_zero: float = 0.4, name: str = "equality_nonneg") -> PlantedLP:
    """Equality rows, x >= 0, row lengths uniform in {lmin..lmax}, N(0,1) values.

    x*: a fraction p_zero of the entries are 0 (with z*_j = |N(0,1)|), the rest
    |N(0,1)|; y* ~ N(0,1); b = A x*, c = A^T y* + z*.
    """
    rng = np.random.default_rng(seed)
    lengths = rng.integers(lmin, lmax + 1, size=m)
    r, cidx = _distinct_cols(rng, lengths, n)
    vals = rng.standard_normal(r.shape[0])
    row_ptr, col_idx, val = _coo_to_csr(m, n, r, cidx, vals)
    rng2 = np.random.default_rng(seed + 7)
    x = np.abs(rng2.standard_normal(n))
    zero = rng2.random(n) < p_zero
    x[zero] = 0.0
    z = np.zeros(n)
    z[zero] = np.abs(rng2.standard_normal(int(zero.sum())))
    y = rng2.standard_normal(m)
    rows = _row_of(row_ptr)
    b = np.bincount(rows, weights=val * x[col_idx], minlength=m).astype(np.float64)
    c = np.bincount(col_idx, weights=val * y[rows], minlength=n).astype(np.float64) + z
    return PlantedLP(m=m, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, c=c,
                     obj_offset=0.0, row_lo=b.copy(), row_hi=b.copy(),
                     col_lo=np.zeros(n), col_hi=np.full(n, np.inf), x_star=x,
                     y_star=y, z_star=z, p_star=float(c @ x), name=name)


def c1_small(seed: int = BASE_SEED + 1) -> PlantedLP:
    """200 x 400, 5-15 nnz per row (~2,000 nnz), equality rows, x >= 0."""
    return equality_nonneg(200, 400, seed, 5, 15, 0.4, name="c1_planted_200x400")


def _calibrate(fn, target, lo, hi, iters=60):
    """Bisection on a monotone increasing fn."""
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if fn(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


_Q = (np.arange(200_000) + 0.5) / 200_000.0


def _lognormal_lengths_mean(sigma, median, lcap, lmin=3):
    from scipy.special import ndtri

    q = ndtri(_Q)
    return float(np.clip(np.rint(median * np.exp(sigma * q)), lmin, lcap).mean())


def general_structure(m: int, n: int, seed: int, nnz_target: int | None = None,
                      median: float = 8.0, frac_empty: float = 0.02,
                      frac_singleton: float = 0.08, frac_doubleton: float = 0.03,
                      frac_eq: float = 0.6, frac_fixed: float = 0.05,
                      one_sided: float = 0.0, lcap: int = 10_000,
                      name: str = "general") -> PlantedLP:
    """Presolvable planted LP: the row/column mix of the 200k x 500k workload.

    Rows: frac_empty empty, frac_singleton with one entry, frac_doubleton
    equality rows with two entries, the rest with lognormal lengths of the given
    median (sigma calibrated so the total is about nnz_target, lengths >= 3).
    Non-doubleton rows are equality with probability frac_eq, else two-sided
    ranged (or, with probability one_sided, one-sided >= / <=).
    Coefficients: random sign times lognormal(0, 1).
    Columns: 40% [0,inf), 20% [l,u], 15% (-inf,u], 15% free, frac_fixed fixed,
    the rest [l,inf).
    """
    rng = np.random.default_rng(seed)
    if nnz_target is None:
        nnz_target = 25 * m
    n_empty = int(round(frac_empty * m))
    n_single = int(round(frac_singleton * m))
    n_double = int(round(frac_doubleton * m))
    n_rest = m - n_empty - n_single - n_double
    rest_target = max(nnz_target - n_single - 2 * n_double, 3 * max(n_rest, 1))
    lc = min(lcap, n)
    if n_rest > 0:
        mean_needed = rest_target / n_rest
        lo_mean = _lognormal_lengths_mean(0.0, median, lc)
        if mean_needed <= lo_mean:
            sigma = 0.0
        else:
            sigma = _calibrate(lambda s: _lognormal_lengths_mean(s, median, lc),
                               mean_needed, 0.0, 4.0, 40)
    else:
        sigma = 0.0
    perm = rng.permutation(m)
    kind_len = np.empty(m, dtype=np.int64)
    kind_len[perm[:n_empty]] = 0
    kind_len[perm[n_empty:n_empty + n_single]] = 1
    kind_len[perm[n_empty + n_single:n_empty + n_single + n_double]] = 2
    rest_rows = perm[n_empty + n_single + n_double:]
    lens = np.clip(np.rint(median * np.exp(sigma * rng.standard_normal(n_rest))), 3, lc)
    kind_len[rest_rows] = lens.astype(np.int64)
    is_double = np.zeros(m, dtype=bool)
    is_double[perm[n_empty + n_single:n_empty + n_single + n_double]] = True

    r, cidx = _distinct_cols(rng, kind_len, n)
    mag = np.exp(rng.standard_normal(r.shape[0]))
    sgn = np.where(rng.random(r.shape[0]) < 0.5, -1.0, 1.0)
    row_ptr, col_idx, val = _coo_to_csr(m, n, r, cidx, sgn * mag)

    s = rng.random(m)
    row_kinds = np.where(s < frac_eq, ROW_EQ, ROW_RANGED).astype(np.int64)
    if one_sided > 0:
        t = rng.random(m)
        row_kinds[(row_kinds == ROW_RANGED) & (t < one_sided / 2)] = ROW_GE
        row_kinds[(row_kinds == ROW_RANGED) & (t >= one_sided / 2) & (t < one_sided)] = ROW_LE
    row_kinds[is_double] = ROW_EQ

    t = rng.random(n)
    cuts = np.cumsum([0.40, 0.20, 0.15, 0.15, frac_fixed])
    col_kinds = np.searchsorted(cuts, t, side="right").astype(np.int64)
    col_kinds = np.minimum(col_kinds, COL_LOWER)
    meta = {"sigma": sigma, "n_empty": n_empty, "n_singleton": n_single,
            "n_doubleton": n_double}
    return _finish(name, m, n, row_ptr, col_idx, val, row_kinds, col_kinds, rng, meta=meta)


def c2_presolvable(seed: int = BASE_SEED + 2, scale: float = 1.0) -> PlantedLP:
    """200k x 500k, ~5M nnz presolvable planted LP (scale shrinks m, n, nnz)."""
    m = max(int(round(200_000 * scale)), 8)
    n = max(int(round(500_000 * scale)), 16)
    return general_structure(m, n, seed, nnz_target=int(round(5_000_000 * scale)),
                             name=f"c2_presolvable_{m}x{n}")


def _powerlaw_mean(kmin, alpha, kmax):
    l = np.floor(kmin * _Q ** (-1.0 / (alpha - 1.0)))
    return float(np.minimum(l, kmax).mean())


def c3_powerlaw(seed: int = BASE_SEED + 3, m: int = 2_000_000, n: int = 5_000_000,
                row_nnz_target: int = 40_000_000, n_dense: int = 5_000,
                dense_len: int = 2_000, alpha: float = 2.1, kmax: int = 10_000,
                name: str | None = None) -> PlantedLP:
    """Large planted LP: power-law row lengths plus dense-ish columns.

    Row lengths floor(kmin * U^(-1/(alpha-1))) capped at kmax, kmin calibrated
    so the rows hold about row_nnz_target entries; n_dense columns get
    dense_len extra entries each in distinct random rows.  Values +-U[0.1, 10];
    equality rows; box bounds [0, U] with U ~ lognormal(0, 1).
    """
    rng = np.random.default_rng(seed)
    kmax = min(kmax, n)
    kmin = _calibrate(lambda k: _powerlaw_mean(k, alpha, kmax), row_nnz_target / m,
                      1.0, 1000.0, 50)
    lens = np.minimum(np.floor(kmin * rng.random(m) ** (-1.0 / (alpha - 1.0))), kmax)
    lens = np.maximum(lens, 1).astype(np.int64)
    r1, c1 = _distinct_cols(rng, lens, n)
    dense_cols = rng.permutation(n)[:n_dense]
    # dense columns: distinct rows per column, drawn as "rows of the transpose"
    dl = np.full(n_dense, min(dense_len, m), dtype=np.int64)
    dc_local, dr = _distinct_cols(rng, dl, m)
    r = np.concatenate([r1, dr])
    cc = np.concatenate([c1, dense_cols[dc_local]])
    mag = rng.uniform(0.1, 10.0, size=r.shape[0])
    sgn = np.where(rng.random(r.shape[0]) < 0.5, -1.0, 1.0)
    row_ptr, col_idx, val = _coo_to_csr(m, n, r, cc, sgn * mag)
    col_kinds = np.full(n, COL_BOX, dtype=np.int64)
    row_kinds = np.full(m, ROW_EQ, dtype=np.int64)
    lp = _finish(name or f"c3_powerlaw_{m}x{n}", m, n, row_ptr, col_idx, val,
                 row_kinds, col_kinds, rng, meta={"kmin": kmin, "n_dense": n_dense})
    # box bounds [0, U], U ~ lognormal(0, 1): re-plant the columns on that box
    rng3 = np.random.default_rng(seed + 11)
    U = np.exp(rng3.standard_normal(n))
    u = rng3.random(n)
    x = U * (0.1 + 0.8 * rng3.random(n))
    z = np.zeros(n)
    zmag = np.abs(rng3.standard_normal(n)) + 1e-3
    at0 = u < 0.3
    atU = (u >= 0.3) & (u < 0.5)
    x[at0] = 0.0
    z[at0] = zmag[at0]
    x[atU] = U[atU]
    z[atU] = -zmag[atU]
    rows = _row_of(row_ptr)
    b = np.bincount(rows, weights=val * x[col_idx], minlength=m).astype(np.float64)
    y = rng3.standard_normal(m)
    y[np.diff(row_ptr) == 0] = 0.0
    lp.c = np.bincount(col_idx, weights=val * y[rows], minlength=n).astype(np.float64) + z
    lp.row_lo = b
    lp.row_hi = b.copy()
    lp.col_lo = np.zeros(n)
    lp.col_hi = U
    lp.x_star, lp.y_star, lp.z_star = x, y, z
    lp.p_star = float(lp.c @ x)
    return lp


def c4_batch(count: int = 512, seed: int = BASE_SEED + 4, m_lo: int = 100,
             m_hi: int = 20_000, first: int = 0):
    """Independent planted LPs: m log-uniform in [m_lo, m_hi], n = 2m,
    4-30 nnz per row, N(0,1) values, equality rows, x >= 0.  Items
    first .. first + count - 1 of the seeded sequence (the same LPs whatever
    slice they are generated in)."""
    rng = np.random.default_rng(seed)
    ms = np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), size=first + count)).astype(np.int64)
    out = []
    for j in range(first, first + count):
        m = int(ms[j])
        out.append(equality_nonneg(m, 2 * m, seed + 1000 * (j + 1), 4, 30, 0.4,
                                   name=f"c4_item{j}_{m}x{2 * m}"))
    return out


def c4_sizes(count: int = 512, seed: int = BASE_SEED + 4, m_lo: int = 100,
             m_hi: int = 20_000):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), size=count)).astype(np.int64)


@dataclass
class StreamRequest:
    index: int
    arrival_s: float
    nnz_target: int
    m: int
    n: int
    seed: int

    def make(self) -> PlantedLP:
        return general_structure(self.m, self.n, self.seed, nnz_target=self.nnz_target,
                                 name=f"c5_req{self.index}_{self.m}x{self.n}")


def c5_stream(count: int = 2000, seed: int = BASE_SEED + 5, rate: float = 200.0,
              nnz_lo: float = 1e3, nnz_hi: float = 1e7):
    """Poisson arrivals at `rate` per second; nnz log-uniform in [nnz_lo, nnz_hi];
    each request has the presolvable structure with m = nnz/25, n = 2.5 m."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    nnz = np.exp(rng.uniform(np.log(nnz_lo), np.log(nnz_hi), size=count)).astype(np.int64)
    reqs = []
    for j in range(count):
        m = max(int(nnz[j] // 25), 8)
        reqs.append(StreamRequest(j, float(t[j]), int(nnz[j]), m, int(round(2.5 * m)),
                                  seed + 1000 * (j + 1)))
    return reqs


def tiny_box(m: int, n: int, seed: int, density: float = 0.7) -> PlantedLP:
    """Tiny LP with every column boxed (finite l, u) and mixed row kinds:
    equality, ranged, >= and <=.  Small enough for vertex enumeration."""
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    for i in range(m):
        if not mask[i].any():
            mask[i, rng.integers(n)] = True
    r, cidx = np.nonzero(mask)
    vals = np.round(rng.standard_normal(r.shape[0]) * 4) / 2
    vals[vals == 0] = 1.0
    row_ptr, col_idx, val = _coo_to_csr(m, n, r, cidx, vals)
    row_kinds = rng.integers(0, 4, size=m)
    col_kinds = np.full(n, COL_BOX, dtype=np.int64)
    return _finish(f"tiny_box_{m}x{n}_{seed}", m, n, row_ptr, col_idx, val, row_kinds,
                   col_kinds, rng, p_low=0.35, p_up=0.35)


def medium_structure(m: int, n: int, seed: int, nnz_target: int | None = None,
                     frac_parallel: float = 0.08, frac_slack: float = 0.05,
                     frac_parallel_cols: float = 0.0) -> PlantedLP:
    """general_structure (with one-sided rows) plus two planted structures:

    * parallel copies: frac_parallel * m extra rows, each a copy of a random
      row with two or more entries scaled by s in {-3, -0.5, 0.25, 2, 7},
      with bounds that hold x* strictly (one side possibly infinite) and
      y* = 0 on the copy;
    * slack columns: frac_slack * m extra columns, each a single entry in an
      inequality row whose y*_i is nonzero, with x* = 0 and either x >= 0 or
      x free; for x >= 0 the coefficient's sign and z* = |a y*_i| / 2 make
      c_j = a y*_i + z*_j of the sign that pushes x_j against the row.

    * parallel columns (frac_parallel_cols * n extra columns, 0 by default):
      copies s a_j of random columns with two or more entries, cost s c_j, so
      z*_k = s z*_j; x*_k = 0 with bounds [0, u] when z*_k > 0, [l, 0] when
      z*_k < 0 and [-w, w] when z*_k = 0.

    The planted optimum (x*, y*, z*) stays optimal, so p* is unchanged.
    """
    import scipy.sparse as sp

    base = general_structure(m, n, seed, nnz_target=nnz_target, one_sided=0.3,
                             name="medium")
    rng = np.random.default_rng(seed + 7)
    A = base.csr()
    lens = np.diff(base.row_ptr)
    ax = A @ base.x_star
    # parallel copies
    src = rng.choice(np.nonzero(lens >= 2)[0], int(round(frac_parallel * m)))
    scale = rng.choice(np.array([-3.0, -0.5, 0.25, 2.0, 7.0]), src.shape[0])
    B = sp.diags(scale) @ A[src]
    w1 = np.exp(rng.standard_normal(src.shape[0])) + 0.1
    w2 = np.exp(rng.standard_normal(src.shape[0])) + 0.1
    open_side = rng.random(src.shape[0])
    lo_c = ax[src] - w1
    hi_c = ax[src] + w2
    lo_c[open_side < 0.25] = -np.inf
    hi_c[(open_side >= 0.25) & (open_side < 0.5)] = np.inf
    # bounds of s * (a_i x): scale and swap for s < 0
    blo = np.where(scale > 0, scale * lo_c, scale * hi_c)
    bhi = np.where(scale > 0, scale * hi_c, scale * lo_c)
    blo[np.isnan(blo)] = -np.inf
    bhi[np.isnan(bhi)] = np.inf
    # slack columns
    ineq = np.nonzero((base.row_lo != base.row_hi) & (base.y_star != 0.0) & (lens >= 1))[0]
    rows_s = rng.choice(ineq, min(int(round(frac_slack * m)), ineq.shape[0]), replace=False)
    k = rows_s.shape[0]
    mag = np.exp(0.5 * rng.standard_normal(k))
    free = rng.random(k) < 0.3
    ys = base.y_star[rows_s]
    # x >= 0: y* > 0 (lower side active) takes a < 0, y* < 0 takes a > 0
    a_s = np.where(ys > 0, -mag, mag)
    z_s = np.where(free, 0.0, 0.5 * np.abs(a_s * ys))
    c_s = a_s * ys + z_s
    S = sp.csr_matrix((a_s, (rows_s, np.arange(k))), shape=(m, k))
    top = sp.hstack([A, S])
    bot = sp.hstack([B, sp.csr_matrix((src.shape[0], k))])
    M = sp.vstack([top, bot]).tocsr()
    x = np.concatenate([base.x_star, np.zeros(k)])
    z = np.concatenate([base.z_star, z_s])
    y = np.concatenate([base.y_star, np.zeros(src.shape[0])])
    c = np.concatenate([base.c, c_s])
    col_lo = np.concatenate([base.col_lo, np.where(free, -np.inf, 0.0)])
    col_hi = np.concatenate([base.col_hi, np.full(k, np.inf)])
    npc = int(round(frac_parallel_cols * n))
    if npc > 0:
        clen = np.diff(base.csr().tocsc().indptr)
        srcc = rng.choice(np.nonzero(clen >= 2)[0], npc)
        sc = rng.choice(np.array([-2.0, -0.5, 0.5, 3.0]), npc)
        P = (M.tocsc()[:, srcc] @ sp.diags(sc)).tocsr()
        M = sp.hstack([M, P]).tocsr()
        zp = sc * z[srcc]
        w = np.exp(rng.standard_normal(npc)) + 0.1
        lo_p = np.where(zp > 0, 0.0, -w)
        hi_p = np.where(zp < 0, 0.0, w)
        hi_p = np.where(zp > 0, w, hi_p)
        lo_p = np.where(zp < 0, -w, lo_p)
        x = np.concatenate([x, np.zeros(npc)])
        z = np.concatenate([z, zp])
        c = np.concatenate([c, sc * c[srcc]])
        col_lo = np.concatenate([col_lo, lo_p])
        col_hi = np.concatenate([col_hi, hi_p])
    M.sort_indices()
    M.eliminate_zeros()
    mm, nn = M.shape
    return PlantedLP(m=mm, n=nn, row_ptr=M.indptr.astype(np.int64),
                     col_idx=M.indices.astype(np.int32), val=M.data.astype(np.float64), c=c,
                     obj_offset=0.0, row_lo=np.concatenate([base.row_lo, blo]),
                     row_hi=np.concatenate([base.row_hi, bhi]), col_lo=col_lo, col_hi=col_hi,
                     x_star=x, y_star=y, z_star=z, p_star=float(c @ x),
                     name=f"medium_{mm}x{nn}",
                     meta={"parallel": int(src.shape[0]), "slack": int(k)})


def amplified_postsolve(m: int = 300, n: int = 700, seed: int = BASE_SEED + 41,
                        shrink: float = 30.0, fixed_value: float = 1.0,
                        fixed_cost: float = 0.7) -> PlantedLP:
    """An LP whose presolve shrinks nothing but the row norm it is measured by.

    Start from equality_nonneg(m, n, seed) (rows A x = b, x >= 0) and append
    one fixed column (l = u = fixed_value) with entry a_i = -(1 - 1/shrink)
    b_i / fixed_value in every row; the original rows become A x + a x_f =
    b / shrink.  Removing the fixed column gives back rows with right-hand
    side b, so the reduced LP's bhat is `shrink` times the original's while
    every row residual is the same: a point at relative KKT error eps on the
    reduced LP can be up to shrink * eps off on the original.  The planted
    optimum (x*, fixed_value), y*, z* (z_f free on a fixed column) stays
    optimal; p* = c^T x* + fixed_cost * fixed_value.
    """
    import scipy.sparse as sp

    base = equality_nonneg(m, n, seed)
    b = base.row_lo
    a = -(1.0 - 1.0 / shrink) * b / fixed_value
    A = sp.hstack([base.csr(), sp.csr_matrix(a.reshape(-1, 1))]).tocsr()
    A.sort_indices()
    rhs = b + a * fixed_value
    x = np.concatenate([base.x_star, [fixed_value]])
    y = base.y_star
    c = np.concatenate([base.c, [fixed_cost]])
    z = np.concatenate([base.z_star, [fixed_cost - float(a @ y)]])
    return PlantedLP(m=m, n=n + 1, row_ptr=A.indptr.astype(np.int64),
                     col_idx=A.indices.astype(np.int32), val=A.data.astype(np.float64), c=c,
                     obj_offset=0.0, row_lo=rhs.copy(), row_hi=rhs.copy(),
                     col_lo=np.concatenate([base.col_lo, [fixed_value]]),
                     col_hi=np.concatenate([base.col_hi, [fixed_value]]), x_star=x, y_star=y,
                     z_star=z, p_star=float(c @ x), name="amplified_postsolve",
                     meta={"shrink": shrink})
