"""Seeded synthetic LP batches for the batched PDHG solver and its oracle.

This module only *builds inputs*: a shared sparse constraint matrix A (CSR),
base vectors c, l, u, x_lo, x_hi, and per-LP override records.  It holds none
of the solver's arithmetic; both the CUDA library and the CPU oracle read what
it produces.  Every generator draws from ``numpy.random.default_rng(seed)``.

Problem form (Sec. 3, Eq. main_lp):  min c^T x  s.t.  l <= A x <= u,
x_lo <= x <= x_hi, infinite bounds written as +-inf.

Override records (one per LP of a batch; Sec. 5.1 and 5.2):
  kind 0  base LP, unchanged;
  kind 1  bound change on variable ``var``: the child's box for that variable
          is [max(x_lo[var], lo), min(x_hi[var], hi)] (strong branching,
          Sec. 5.1: up child lo = ceil(x_rel), down child hi = floor(x_rel));
  kind 2  objective replaced by sign * e_var (bound tightening, Sec. 5.2:
          sign +1 gives min x_var, sign -1 gives max x_var).

Workload recipes (shapes follow the paper's strong-branching and OBBT use):
  ``sb_small``   m=200, n=400, 4-6 nnz per column, FP64, 16 SB children.
  ``sb_powerlaw`` m=20k, n=50k, power-law row lengths on [2,500], 64 children.
  ``obbt_square`` m=n=100k, 10 nnz per row, 10% free variables, 1024 LPs.
  ``sb_large``   m=1M, n=2M, rows of 3-8 nnz plus 500 dense rows of 10k nnz,
                 128 children.
The paper's instances (generator families, NN verification, MIPLIB) are not
available; these synthetic batches stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

KIND_BASE = 0
KIND_BOUND = 1
KIND_OBJECTIVE = 2


@dataclass
class LPData:
    """One shared LP: CSR matrix plus base vectors (all float64, int64/int32)."""

    m: int
    n: int
    row_ptr: np.ndarray  # int64, m+1
    col_idx: np.ndarray  # int32, nnz
    vals: np.ndarray  # float64, nnz
    c: np.ndarray
    row_lo: np.ndarray
    row_hi: np.ndarray
    var_lo: np.ndarray
    var_hi: np.ndarray
    x0: np.ndarray | None = None  # generating point (feasible by construction)
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        a = np.zeros((self.m, self.n))
        for i in range(self.m):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            np.add.at(a[i], self.col_idx[s:e], self.vals[s:e])
        return a

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """A @ x for input construction (row bounds from a generating point)."""
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        out = np.zeros(self.m)
        np.add.at(out, rows, self.vals * x[self.col_idx])
        return out


@dataclass
class Specs:
    """Per-LP override records, structure-of-arrays."""

    kind: np.ndarray  # int32
    var: np.ndarray  # int32
    lo: np.ndarray  # float64
    hi: np.ndarray  # float64
    sign: np.ndarray  # float64
    label: list = field(default_factory=list)

    def __len__(self) -> int:
        return int(self.kind.shape[0])

    def subset(self, idx) -> "Specs":
        idx = np.asarray(idx)
        return Specs(self.kind[idx].copy(), self.var[idx].copy(), self.lo[idx].copy(),
                     self.hi[idx].copy(), self.sign[idx].copy(),
                     [self.label[i] for i in idx] if self.label else [])


@dataclass
class Workload:
    lp: LPData
    specs: Specs
    precision: str  # "fp64" or "mixed"
    name: str


def make_specs(kind, var, lo=None, hi=None, sign=None, label=None) -> Specs:
    kind = np.asarray(kind, dtype=np.int32)
    k = kind.shape[0]
    var = np.asarray(var, dtype=np.int32)
    lo = np.full(k, -np.inf) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.full(k, np.inf) if hi is None else np.asarray(hi, dtype=np.float64)
    sign = np.ones(k) if sign is None else np.asarray(sign, dtype=np.float64)
    return Specs(kind, var, lo, hi, sign, list(label) if label is not None else [])


def base_specs(num: int) -> Specs:
    return make_specs(np.zeros(num), np.zeros(num))


def sb_specs(x_rel: np.ndarray, cand: np.ndarray) -> Specs:
    """Full strong branching on candidates ``cand`` (Sec. 5.1): LP i is the up
    child x_j >= ceil(x_rel_j); LP p+i is the down child x_j <= floor(x_rel_j)."""
    cand = np.asarray(cand, dtype=np.int32)
    p = cand.shape[0]
    up_lo = np.ceil(x_rel[cand])
    dn_hi = np.floor(x_rel[cand])
    kind = np.ones(2 * p, dtype=np.int32)
    var = np.concatenate([cand, cand])
    lo = np.concatenate([up_lo, np.full(p, -np.inf)])
    hi = np.concatenate([np.full(p, np.inf), dn_hi])
    label = [f"up{j}" for j in cand] + [f"down{j}" for j in cand]
    return make_specs(kind, var, lo, hi, None, label)


def obbt_specs(cand: np.ndarray) -> Specs:
    """Bound tightening (Sec. 5.2): objective matrix C = [I, -I] restricted to
    ``cand``: LP i minimises x_j, LP p+i maximises x_j (minimises -x_j)."""
    cand = np.asarray(cand, dtype=np.int32)
    p = cand.shape[0]
    kind = np.full(2 * p, KIND_OBJECTIVE, dtype=np.int32)
    var = np.concatenate([cand, cand])
    sign = np.concatenate([np.ones(p), -np.ones(p)])
    label = [f"min{j}" for j in cand] + [f"max{j}" for j in cand]
    return make_specs(kind, var, None, None, sign, label)


# ----------------------------------------------------------------------------
# matrix construction helpers
# ----------------------------------------------------------------------------

def _csr_from_rows(m: int, lengths: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), vals.astype(np.float64)


def _distinct_cols_per_row(rng, lengths: np.ndarray, ncols: int) -> np.ndarray:
    """For each row draw ``lengths[i]`` distinct column indices in [0, ncols),
    returned concatenated and sorted within each row."""
    lengths = np.asarray(lengths, dtype=np.int64)
    m = lengths.shape[0]
    nnz = int(lengths.sum())
    rows = np.repeat(np.arange(m, dtype=np.int64), lengths)
    cols = rng.integers(0, ncols, size=nnz, dtype=np.int64)
    for _ in range(100):
        key = rows * ncols + cols
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(nnz, dtype=bool)
        dup[order[1:]] = ks[1:] == ks[:-1]
        nd = int(dup.sum())
        if nd == 0:
            cols = (np.sort(key) - rows * ncols)
            return cols.astype(np.int32)
        cols[dup] = rng.integers(0, ncols, size=nd, dtype=np.int64)
    raise RuntimeError("could not draw distinct columns")


def _signed_uniform(rng, size, lo=0.1, hi=10.0):
    mag = rng.uniform(lo, hi, size=size)
    sgn = np.where(rng.random(size) < 0.5, -1.0, 1.0)
    return mag * sgn


def _rows_around(lp: LPData, x0: np.ndarray, rng) -> None:
    ax = lp.matvec(x0)
    lp.row_lo = ax - rng.uniform(0.0, 1.0, size=lp.m)
    lp.row_hi = ax + rng.uniform(0.0, 1.0, size=lp.m)


def _csc_to_csr(m: int, n: int, col_lengths: np.ndarray, row_idx: np.ndarray, vals: np.ndarray):
    cols = np.repeat(np.arange(n, dtype=np.int64), col_lengths)
    order = np.lexsort((cols, row_idx))
    r = row_idx[order]
    lengths = np.bincount(r, minlength=m)
    return _csr_from_rows(m, lengths, cols[order], vals[order])


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def sb_small(seed: int = 0) -> Workload:
    """m=200, n=400; each column has U{4..6} distinct random rows (nnz ~ 2000);
    values sign*U[0.1,10]; x0 ~ U[0,10]^n, box [0,10]; l, u = A x0 -/+ U[0,1];
    c ~ N(0,1); 16 strong-branching children = 8 random columns x {up, down}."""
    rng = np.random.default_rng(seed)
    m, n = 200, 400
    col_len = rng.integers(4, 7, size=n)
    row_idx = _distinct_cols_per_row(rng, col_len, m).astype(np.int64)
    vals = _signed_uniform(rng, row_idx.shape[0])
    row_ptr, col_idx, v = _csc_to_csr(m, n, col_len, row_idx, vals)
    x0 = rng.uniform(0.0, 10.0, size=n)
    lp = LPData(m, n, row_ptr, col_idx, v, rng.standard_normal(n), None, None,
                np.zeros(n), np.full(n, 10.0), x0, "sb_small")
    _rows_around(lp, x0, rng)
    cand = rng.choice(n, size=8, replace=False)
    return Workload(lp, sb_specs(x0, cand), "fp64", "sb_small m=200 n=400 B=16 fp64")


def powerlaw_lengths(rng, m: int, kmin: int = 2, kmax: int = 500, alpha: float = 1.839) -> np.ndarray:
    k = np.arange(kmin, kmax + 1)
    p = k.astype(np.float64) ** (-alpha)
    p /= p.sum()
    return rng.choice(k, size=m, p=p)


def sb_powerlaw_matrix(seed: int, m: int, n: int, name: str) -> LPData:
    rng = np.random.default_rng(seed)
    lengths = powerlaw_lengths(rng, m)
    lengths = np.minimum(lengths, n)
    cols = _distinct_cols_per_row(rng, lengths, n)
    vals = _signed_uniform(rng, cols.shape[0])
    row_ptr, col_idx, v = _csr_from_rows(m, lengths, cols, vals)
    x0 = rng.uniform(0.0, 10.0, size=n)
    lp = LPData(m, n, row_ptr, col_idx, v, rng.standard_normal(n), None, None,
                np.zeros(n), np.full(n, 10.0), x0, name)
    _rows_around(lp, x0, rng)
    return lp


def sb_powerlaw(seed: int = 0, m: int = 20000, n: int = 50000, children: int = 64) -> Workload:
    """m=20k, n=50k; row lengths P(k) ~ k^-1.839 on [2,500] (mean 12.5,
    nnz ~ 250k) with distinct random columns; values, x0, box, row bounds and
    c as in ``sb_small``; B = 64 = 32 random columns x {up, down}."""
    lp = sb_powerlaw_matrix(seed, m, n, "sb_powerlaw")
    rng = np.random.default_rng(seed + 1000)
    cand = rng.choice(n, size=children // 2, replace=False)
    return Workload(lp, sb_specs(lp.x0, cand), "mixed",
                    f"sb_powerlaw m={m} n={n} B={children} fp32-iterates/double-float-checks")


def obbt_square(seed: int = 0, m: int = 100000, n: int = 100000, lps: int = 1024,
                row_nnz: int = 10) -> Workload:
    """m=n=100k, 10 nnz per row at uniform random columns (nnz = 1M), values
    sign*U[0.1,10]; 90% of variables get the box [min, max] of two U[-100,100]
    draws, 10% are free; x0 uniform in each box (N(0,10) for free variables);
    l, u = A x0 -/+ U[0,1]; base c = 0; ``lps`` OBBT LPs = lps/2 random
    variables x {min, max}."""
    rng = np.random.default_rng(seed)
    lengths = np.full(m, row_nnz, dtype=np.int64)
    cols = _distinct_cols_per_row(rng, lengths, n)
    vals = _signed_uniform(rng, cols.shape[0])
    row_ptr, col_idx, v = _csr_from_rows(m, lengths, cols, vals)
    a = rng.uniform(-100.0, 100.0, size=n)
    b = rng.uniform(-100.0, 100.0, size=n)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    free = rng.random(n) < 0.10
    x_box = np.clip(rng.uniform(0.0, 1.0, size=n) * (hi - lo) + lo, lo, hi)
    x0 = np.where(free, rng.normal(0.0, 10.0, size=n), x_box)
    lo[free], hi[free] = -np.inf, np.inf
    lp = LPData(m, n, row_ptr, col_idx, v, np.zeros(n), None, None, lo, hi, x0, "obbt_square")
    _rows_around(lp, x0, rng)
    cand = rng.choice(n, size=lps // 2, replace=False)
    return Workload(lp, obbt_specs(cand), "mixed",
                    f"obbt_square m={m} n={n} B={lps} fp32-iterates/double-float-checks")


def sb_large(seed: int = 0, m: int = 1000000, n: int = 2000000, dense_rows: int = 500,
             dense_len: int = 10000, children: int = 128) -> Workload:
    """m=1M, n=2M; bimodal rows: U{3..8} nnz, plus ``dense_rows`` rows of
    ``dense_len`` nnz (nnz ~ 10.5M); values, box [0,10], x0, row bounds and c
    as in ``sb_small``; 128 strong-branching children."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(3, 9, size=m).astype(np.int64)
    dense = rng.choice(m, size=dense_rows, replace=False)
    lengths[dense] = min(dense_len, n)
    cols = _distinct_cols_per_row(rng, lengths, n)
    vals = _signed_uniform(rng, cols.shape[0])
    row_ptr, col_idx, v = _csr_from_rows(m, lengths, cols, vals)
    x0 = rng.uniform(0.0, 10.0, size=n)
    lp = LPData(m, n, row_ptr, col_idx, v, rng.standard_normal(n), None, None,
                np.zeros(n), np.full(n, 10.0), x0, "sb_large")
    _rows_around(lp, x0, rng)
    cand = rng.choice(n, size=children // 2, replace=False)
    return Workload(lp, sb_specs(x0, cand), "mixed",
                    f"sb_large m={m} n={n} B={children} fp32-iterates/double-float-checks")


def sb_dense_cols(seed: int = 0, m: int = 3000, n: int = 2000, dense_cols: int = 12, children: int = 16) -> Workload:
    """m=3000, n=2000: columns of U{3..8} distinct rows, plus ``dense_cols``
    columns of 40 .. 1500 rows (evenly spaced), so that rows of A^T exceed the
    32-entry long-row threshold and the longest spans several 256-entry
    segments; values sign*U[0.1,10]; x0 ~ U[0,10]^n, box [0,10]; l, u =
    A x0 -/+ U[0,1]; c ~ N(0,1); 16 strong-branching children on 8 columns,
    two of them dense."""
    rng = np.random.default_rng(seed)
    col_len = rng.integers(3, 9, size=n).astype(np.int64)
    dense = rng.choice(n, size=dense_cols, replace=False)
    col_len[dense] = np.linspace(40, 1500, dense_cols).astype(np.int64)
    row_idx = _distinct_cols_per_row(rng, col_len, m).astype(np.int64)
    vals = _signed_uniform(rng, row_idx.shape[0])
    row_ptr, col_idx, v = _csc_to_csr(m, n, col_len, row_idx, vals)
    x0 = rng.uniform(0.0, 10.0, size=n)
    lp = LPData(m, n, row_ptr, col_idx, v, rng.standard_normal(n), None, None,
                np.zeros(n), np.full(n, 10.0), x0, "sb_dense_cols")
    _rows_around(lp, x0, rng)
    others = np.setdiff1d(np.arange(n), dense)
    cand = np.concatenate([dense[-2:], rng.choice(others, size=children // 2 - 2, replace=False)])
    return Workload(lp, sb_specs(x0, cand), "mixed",
                    f"sb_dense_cols m={m} n={n} B={children} ({dense_cols} columns of 40-1500 rows)")


def covering_large_bounds(seed: int = 0, m: int = 300, n: int = 500, big: float = 1e10) -> Workload:
    """Covering LP whose variable boxes are mostly far larger than any
    optimum reaches, the case the reduced cost robust to large bounds is for:
    each column has U{3..5} distinct rows with values U[0.5, 3]; rows
    A x >= b with b = U[0.3, 0.9] * (A x_f), x_f ~ U[0.5, 1] (so every LP
    before branching is feasible); c ~ U[0.5, 2]; x in [0, big] for 80% of
    the variables and [0, U[1, 3]] for the rest.  16 strong-branching
    children = 8 random columns x {up, down} around x_rel ~ U[0.2, 2.8]."""
    rng = np.random.default_rng(seed)
    col_len = rng.integers(3, 6, size=n)
    row_idx = _distinct_cols_per_row(rng, col_len, m).astype(np.int64)
    vals = rng.uniform(0.5, 3.0, size=row_idx.shape[0])
    row_ptr, col_idx, v = _csc_to_csr(m, n, col_len, row_idx, vals)
    hi = np.where(rng.random(n) < 0.8, big, rng.uniform(1.0, 3.0, size=n))
    x_rel = rng.uniform(0.2, 2.8, size=n)
    lp = LPData(m, n, row_ptr, col_idx, v, rng.uniform(0.5, 2.0, size=n), None, np.full(m, np.inf),
                np.zeros(n), hi, x_rel, f"covering_large_bounds{seed}")
    lp.row_lo = rng.uniform(0.3, 0.9, size=m) * lp.matvec(rng.uniform(0.5, 1.0, size=n))
    cand = rng.choice(n, size=8, replace=False)
    return Workload(lp, sb_specs(x_rel, cand), "mixed", f"covering m={m} n={n} B=16, bounds {big:g}")


def random_lp(seed: int, m: int, n: int, density: float = 0.3, mixed_bounds: bool = True,
              feasible: bool = True, int_values: bool = False) -> LPData:
    """Small random LP with every bound type (free, one-sided and two-sided
    variables; equality, one-sided and ranged rows), feasible by construction
    when ``feasible``.  For unit tests and brute-force pins."""
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    for i in range(m):  # at least one entry per row
        if not mask[i].any():
            mask[i, rng.integers(n)] = True
    dense = np.where(mask, np.round(rng.uniform(-3, 3, size=(m, n)), 1 if not int_values else 0), 0.0)
    dense[mask & (dense == 0)] = 1.0
    x0 = rng.uniform(-2.0, 2.0, size=n)
    lo = np.full(n, -np.inf)
    hi = np.full(n, np.inf)
    kinds = rng.integers(0, 5 if mixed_bounds else 1, size=n)
    for j in range(n):
        k = kinds[j]
        if k == 0:  # two-sided
            lo[j] = x0[j] - rng.uniform(0.5, 3.0)
            hi[j] = x0[j] + rng.uniform(0.5, 3.0)
        elif k == 1:
            lo[j] = x0[j] - rng.uniform(0.0, 2.0)
        elif k == 2:
            hi[j] = x0[j] + rng.uniform(0.0, 2.0)
        elif k == 3:  # free
            pass
        else:  # fixed
            lo[j] = hi[j] = x0[j]
    ax = dense @ x0
    rl = np.full(m, -np.inf)
    ru = np.full(m, np.inf)
    rk = rng.integers(0, 4 if mixed_bounds else 1, size=m)
    for i in range(m):
        k = rk[i]
        if k == 0:
            rl[i] = ax[i] - rng.uniform(0.0, 1.0)
            ru[i] = ax[i] + rng.uniform(0.0, 1.0)
        elif k == 1:
            rl[i] = ax[i] - rng.uniform(0.0, 1.0)
        elif k == 2:
            ru[i] = ax[i] + rng.uniform(0.0, 1.0)
        else:
            rl[i] = ru[i] = ax[i]
    if not feasible:
        # contradict: a ranged row pushed away from the reachable range
        rl[0] = ru[0] = np.abs(dense[0]) @ np.maximum(np.abs(lo), np.abs(hi)).clip(max=1e3) + 1e4
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(m):
        nz = np.nonzero(dense[i])[0]
        cols.append(nz)
        vals.append(dense[i, nz])
        row_ptr[i + 1] = row_ptr[i] + nz.shape[0]
    c = np.round(rng.normal(size=n), 2)
    # keep the LP bounded: give unbounded-direction variables a cost pointing inward
    for j in range(n):
        if np.isinf(lo[j]) and not np.isinf(hi[j]):
            c[j] = -abs(c[j]) - 0.1
        elif np.isinf(hi[j]) and not np.isinf(lo[j]):
            c[j] = abs(c[j]) + 0.1
    return LPData(m, n, row_ptr, np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32),
                  np.concatenate(vals) if vals else np.zeros(0), c, rl, ru, lo, hi, x0, f"random{seed}")


def from_dense(a: np.ndarray, c, row_lo, row_hi, var_lo, var_hi, name: str = "") -> LPData:
    a = np.asarray(a, dtype=np.float64)
    m, n = a.shape
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(m):
        nz = np.nonzero(a[i])[0]
        cols.append(nz)
        vals.append(a[i, nz])
        row_ptr[i + 1] = row_ptr[i] + nz.shape[0]
    ci = np.concatenate(cols).astype(np.int32) if m else np.zeros(0, np.int32)
    vv = np.concatenate(vals) if m else np.zeros(0)
    f = lambda v: np.asarray(v, dtype=np.float64)
    return LPData(m, n, row_ptr, ci, vv, f(c), f(row_lo), f(row_hi), f(var_lo), f(var_hi), None, name)


# rows of the five serving matrices: geometric from 1k to 200k
SERVING_ROWS = (1000, 3760, 14100, 53200, 200000)


def serving_matrices(seed0: int = 0, rows=SERVING_ROWS):
    """The serving set: matrices built like ``sb_powerlaw`` with m rows and
    n = 2m columns (power-law row lengths on [2, 500], mean 12.5), seeds
    seed0 .. seed0+4."""
    return [sb_powerlaw_matrix(seed0 + k, m, 2 * m, f"serve{k}_m{m}") for k, m in enumerate(rows)]


def serving_stream(mats, seed: int = 100, count: int = 200, max_children: int = 256):
    """A seeded request stream over ``mats``: unit-rate exponential
    inter-arrival gaps (scale them by 1/rate), a uniformly drawn matrix and
    U{1..max_children} strong-branching children (random columns x {up,
    down}) per request.  Returns [(gap, matrix index, Specs)]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        gap = float(rng.exponential(1.0))
        k = int(rng.integers(len(mats)))
        b = int(rng.integers(1, max_children + 1))
        lp = mats[k]
        cand = rng.choice(lp.n, size=(b + 1) // 2, replace=False)
        out.append((gap, k, sb_specs(lp.x0, cand).subset(range(b))))
    return out


WORKLOADS = {
    "sb_small": sb_small,
    "sb_powerlaw": sb_powerlaw,
    "obbt_square": obbt_square,
    "sb_large": sb_large,
}
