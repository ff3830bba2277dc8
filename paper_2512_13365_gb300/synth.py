"""Seeded synthetic ternary expression sets shaped like fast-matmul schemes.

This module is the ONLY code shared by the oracle side and the CUDA side of
the tests and the benchmark.  It produces inputs (ternary coefficient
matrices and search parameters) and holds none of the method's arithmetic:
no pair counting, no selection, no substitution.

Shapes follow the split of a scheme (m, n, p : r) into three expression sets
(Section 3.2): E_U has r rows over m*n variables, E_V has r rows over n*p
variables and E_W has m*p rows over r variables (the rows of W transposed).
The paper's 149 real schemes are not available, so rows are drawn at random
with the sizes and densities of those workloads (Section 4.1 ranks, Tables 1-6
naive counts), plus "planted" signed pairs that give the search repeated
subexpressions to find.

Randomness: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), seeded from (config seed, scheme, matrix).
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 stream (Steele et al. 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Integer in [0, n) by the multiply-high map of the top 32 bits."""
        return ((self.next() >> 32) * n) >> 32

    def uniform(self) -> float:
        """Float in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def sign(self) -> int:
        return 1 if (self.next() >> 63) else -1


def stream(config_seed: int, scheme: int, matrix: int) -> SplitMix64:
    """Independent stream for one matrix of one scheme of one configuration."""
    s = SplitMix64((config_seed * 0x100000001B3) ^ (scheme << 20) ^ (matrix << 8) ^ 0x5EED)
    s.next()
    return s


def _positions(rng: SplitMix64, n: int, k: int) -> List[int]:
    """k distinct positions of range(n), uniform (partial Fisher-Yates)."""
    idx = list(range(n))
    for a in range(k):
        b = a + rng.below(n - a)
        idx[a], idx[b] = idx[b], idx[a]
    return idx[:k]


def rows_by_nnz(rng: SplitMix64, rows: int, cols: int, lo: int, hi: int) -> np.ndarray:
    """Each row draws k ~ U[lo, hi] (clamped to cols), then k distinct
    positions and independent +/-1 signs."""
    m = np.zeros((rows, cols), dtype=np.int8)
    for r in range(rows):
        k = min(cols, lo + rng.below(hi - lo + 1))
        for v in _positions(rng, cols, k):
            m[r, v] = rng.sign()
    return m


def rows_by_density(rng: SplitMix64, rows: int, cols: int, d: float) -> np.ndarray:
    """Each entry is nonzero with probability d; a row with fewer than two
    nonzeros is drawn again."""
    m = np.zeros((rows, cols), dtype=np.int8)
    for r in range(rows):
        while True:
            row = np.zeros(cols, dtype=np.int8)
            for v in range(cols):
                if rng.uniform() < d:
                    row[v] = rng.sign()
            if np.count_nonzero(row) >= 2:
                break
        m[r] = row
    return m


def plant_pairs(rng: SplitMix64, m: np.ndarray, n_pairs: int, frac_lo: float, frac_hi: float) -> None:
    """Insert n_pairs signed pairs (i, j, s): each picks i != j, s = +/-1 and a
    fraction f ~ U[frac_lo, frac_hi] of the rows (without replacement); in
    each chosen row it writes alpha_i = sigma, alpha_j = sigma*s for a random
    sigma (overwriting)."""
    rows, cols = m.shape
    if cols < 2:
        return
    for _ in range(n_pairs):
        i = rng.below(cols)
        j = rng.below(cols - 1)
        if j >= i:
            j += 1
        s = rng.sign()
        f = frac_lo + (frac_hi - frac_lo) * rng.uniform()
        n_rows = max(2, int(round(f * rows))) if rows >= 2 else rows
        for r in _positions(rng, rows, min(rows, n_rows)):
            sigma = rng.sign()
            m[r, i] = sigma
            m[r, j] = sigma * s


def scheme_shapes(m: int, n: int, p: int, r: int) -> List[Tuple[int, int]]:
    """(rows, cols) of E_U, E_V, E_W for a scheme (m, n, p : r) (Section 3.2)."""
    return [(r, m * n), (r, n * p), (m * p, r)]


@dataclasses.dataclass
class Search:
    """One search problem: matrices plus the parameters of the search."""

    name: str
    mats: List[np.ndarray]
    weights: Tuple[int, ...]  # gi, ga, gr, wr, mix, g[, gp] (x100 of the paper's); missing gp = 0
    n_proc: int
    seed: int
    budget: int
    interval: int
    permille: int
    cap: int

    def process_steps(self) -> int:
        return len(self.mats) * self.n_proc * self.budget


# The default strategy weights of Section 3.5.1 (x100): gi 8, ga 4, gr 2,
# wr 1, mix 0.1, gp 0.01; and the same without Greedy-Potential.
PAPER_WEIGHTS = (800, 400, 200, 100, 10, 0, 1)
PAPER_WEIGHTS_NO_GP = (800, 400, 200, 100, 10, 0)
GI_ONLY = (1, 0, 0, 0, 0, 0)
GP_ONLY = (0, 0, 0, 0, 0, 0, 1)


def config1(n_proc: int = 64, budget: int = 200) -> Search:
    """U side of a (2,2,2:7)-shaped scheme, 7 rows x 4 variables, row nnz
    U[2,4], plus its 4 x 7 W^T companion; Greedy-Intersections only."""
    a = rows_by_nnz(stream(1, 0, 0), 7, 4, 2, 4)
    b = rows_by_nnz(stream(1, 0, 1), 4, 7, 2, 4)
    return Search("tern-2x2x2r7-U+Wt", [a, b], GI_ONLY, n_proc, 0, budget, 32, 400, 32)


def config2(n_proc: int = 4096, budget: int = 1024) -> Search:
    """(3,3,3:23)-shaped scheme: E_U, E_V 23 x 9 and E_W 9 x 23, row nnz
    U[2,5], plus 12 planted signed pairs each in 30% of the rows."""
    mats = []
    for k, (rows, cols) in enumerate(scheme_shapes(3, 3, 3, 23)):
        rng = stream(2, 0, k)
        mat = rows_by_nnz(rng, rows, cols, 2, 5)
        plant_pairs(rng, mat, 12, 0.3, 0.3)
        mats.append(mat)
    return Search("tern-3x3x3r23", mats, PAPER_WEIGHTS, n_proc, 0, budget, 32, 400, 128)


def density_scheme(config_seed: int, scheme: int, fmt: Tuple[int, int, int, int],
                   d: float, n_planted: int) -> List[np.ndarray]:
    """Scheme-shaped matrices in density mode with planted pairs (f ~ U[0.1, 0.4])."""
    mats = []
    for k, (rows, cols) in enumerate(scheme_shapes(*fmt)):
        rng = stream(config_seed, scheme, k)
        mat = rows_by_density(rng, rows, cols, d)
        plant_pairs(rng, mat, n_planted, 0.1, 0.4)
        mats.append(mat)
    return mats


def config3_formats(n_schemes: int = 32) -> List[Tuple[int, int, int, int, float, int]]:
    """Formats of the batched workload: (2,3,4:20) and (4,4,4:49) plus random
    formats from {2,3,4}^3 with 24 <= mnp <= 64 and r = round(0.8 mnp);
    density U[0.25, 0.4] and 8-24 planted pairs each."""
    rng = stream(3, 0xFFFF, 0)
    fixed = [(2, 3, 4), (4, 4, 4)]
    fmts = []
    for i in range(n_schemes):
        if i < len(fixed):
            m, n, p = fixed[i]
        else:
            while True:
                m, n, p = 2 + rng.below(3), 2 + rng.below(3), 2 + rng.below(3)
                if 24 <= m * n * p <= 64:
                    break
        r = {(2, 3, 4): 20, (4, 4, 4): 49}.get((m, n, p), int(round(0.8 * m * n * p)))
        d = 0.25 + 0.15 * rng.uniform()
        planted = 8 + rng.below(17)
        fmts.append((m, n, p, r, d, planted))
    return fmts


def config3(n_schemes: int = 32, n_proc: int = 1024, budget: int = 512, interval: int = 32) -> List[Search]:
    out = []
    for s, (m, n, p, r, d, planted) in enumerate(config3_formats(n_schemes)):
        mats = density_scheme(3, s, (m, n, p, r), d, planted)
        out.append(Search(f"tern-{m}x{n}x{p}r{r}", mats, PAPER_WEIGHTS, n_proc, s, budget, interval, 400, 256))
    return out


def config4(n_proc: int = 65536, budget: int = 2000) -> Search:
    """(6,6,6:153)-shaped scheme: E_U, E_V 153 x 36, E_W 36 x 153, row nnz
    U[3,12], 64 planted pairs in 10-40% of rows; variables grow to 512."""
    mats = []
    for k, (rows, cols) in enumerate(scheme_shapes(6, 6, 6, 153)):
        rng = stream(4, 0, k)
        mat = rows_by_nnz(rng, rows, cols, 3, 12)
        plant_pairs(rng, mat, 64, 0.1, 0.4)
        mats.append(mat)
    return Search("tern-6x6x6r153", mats, PAPER_WEIGHTS, n_proc, 0, budget, 32, 400, 512)


def serving_requests(n_req: int = 2000, rate_hz: float = 50.0, n_proc: int = 2048,
                     budget: int = 256) -> List[Tuple[float, Search]]:
    """Poisson arrivals (mean rate_hz) of requests with formats uniform in
    {2..6}^3, r = round(0.85 mnp), matrices generated as in the batched
    workload from a per-request seed."""
    arr = stream(5, 0xFFFF, 0)
    t = 0.0
    out = []
    for q in range(n_req):
        t += -np.log(1.0 - arr.uniform()) / rate_hz
        rng = stream(5, q, 0xFF)
        m, n, p = 2 + rng.below(5), 2 + rng.below(5), 2 + rng.below(5)
        r = int(round(0.85 * m * n * p))
        d = 0.25 + 0.15 * rng.uniform()
        planted = 8 + rng.below(17)
        mats = density_scheme(5, q, (m, n, p, r), d, planted)
        out.append((t, Search(f"req{q}-{m}x{n}x{p}r{r}", mats, PAPER_WEIGHTS, n_proc, q, budget, 32, 400, 512)))
    return out


def random_matrix(seed: int, rows: int, cols: int, lo: int = 2, hi: int = 4,
                  n_planted: int = 0, frac: Tuple[float, float] = (0.2, 0.4)) -> np.ndarray:
    """Small random ternary matrix for tests."""
    rng = stream(1000 + seed, rows, cols)
    m = rows_by_nnz(rng, rows, cols, lo, hi)
    if n_planted:
        plant_pairs(rng, m, n_planted, frac[0], frac[1])
    return m


def strassen_uvw() -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Strassen's (2,2,2:7) scheme from its textbook definition:
    M1=(A11+A22)(B11+B22), M2=(A21+A22)B11, M3=A11(B12-B22), M4=A22(B21-B11),
    M5=(A11+A12)B22, M6=(A21-A11)(B11+B12), M7=(A12-A22)(B21+B22);
    C11=M1+M4-M5+M7, C12=M3+M5, C21=M2+M4, C22=M1-M2+M3+M6.
    Variables in row-major order (a11, a12, a21, a22)."""
    U = np.array([[1, 0, 0, 1], [0, 0, 1, 1], [1, 0, 0, 0], [0, 0, 0, 1],
                  [1, 1, 0, 0], [-1, 0, 1, 0], [0, 1, 0, -1]], dtype=np.int8)
    V = np.array([[1, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, -1], [-1, 0, 1, 0],
                  [0, 0, 0, 1], [1, 1, 0, 0], [0, 0, 1, 1]], dtype=np.int8)
    # W[l, (i,j)] : coefficient of M_l in C_ij
    W = np.zeros((7, 4), dtype=np.int8)
    for l, c in [(0, 1), (3, 1), (4, -1), (6, 1)]:
        W[l, 0] = c
    for l, c in [(2, 1), (4, 1)]:
        W[l, 1] = c
    for l, c in [(1, 1), (3, 1)]:
        W[l, 2] = c
    for l, c in [(0, 1), (1, -1), (2, 1), (5, 1)]:
        W[l, 3] = c
    return U, V, W


def standard_uvw(m: int, n: int, p: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """The schoolbook scheme (m,n,p:mnp): one product a_ij b_jk per (i, j, k),
    added into c_ik.  Rows of U, V, W in the layout of strassen_uvw."""
    r = m * n * p
    U = np.zeros((r, m * n), np.int8)
    V = np.zeros((r, n * p), np.int8)
    W = np.zeros((r, m * p), np.int8)
    for l, (i, j, k) in enumerate((i, j, k) for i in range(m) for j in range(n) for k in range(p)):
        U[l, i * n + j] = 1
        V[l, j * p + k] = 1
        W[l, i * p + k] = 1
    return U, V, W


def scheme_sides(U: np.ndarray, V: np.ndarray, W: np.ndarray) -> List[np.ndarray]:
    """E_U = U (r x mn), E_V = V (r x np), E_W = W^T (mp x r) (Section 3.2)."""
    return [np.ascontiguousarray(U, dtype=np.int8), np.ascontiguousarray(V, dtype=np.int8),
            np.ascontiguousarray(W.T, dtype=np.int8)]
