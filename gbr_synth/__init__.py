"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the ranking / H·v / Lanczos method: only
the counter-based generator (splitmix64), the distributions drawn from it, and
the model definitions (hopping matrices, interaction arrays) of the workloads.
Both the CPU oracle and the CUDA path take their inputs from here.

Generator: ``u(seed, i) = splitmix64(seed XOR (i * 0x9E3779B97F4A7C15))`` where
splitmix64 is Steele, Lea and Flood's published mixer (add the golden gamma,
then two xor-shift-multiply rounds and a final xor-shift).  Derived values:

* uniform[a, b):  ``a + (b - a) * ((u >> 11) * 2**-53)`` (exact in binary64
  for [-1, 1): ``2 * ((u >> 11) * 2**-53) - 1``),
* bounded integer in [0, n): ``(u * n) >> 64`` (the high word of the 128-bit
  product).

Seeds: 1 = Lanczos start vectors, 2 = fixed-popcount rank queries,
3 = trie member set, 4 = impurity models, 5 = trie queries.

A GPU twin of the same generator (``gpu`` submodule, a small CUDA library of
its own) produces the full-size inputs directly in device memory; tests check
that both produce identical bits.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK32 = np.uint64(0xFFFFFFFF)

SEED_START = 1
SEED_COMB_QUERIES = 2
SEED_TRIE_SET = 3
SEED_MODELS = 4
SEED_TRIE_QUERIES = 5


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 output for state ``x`` (uint64 array), wrapping arithmetic."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def u64(seed: int, idx) -> np.ndarray:
    """Counter-mode draw ``u(seed, i)`` for an array (or range) of indices."""
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64(np.uint64(seed) ^ (i * GOLDEN))


def mulhi64(a: np.ndarray, b: int) -> np.ndarray:
    """High 64 bits of the 128-bit product a*b (a uint64 array, 0 <= b < 2**64)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.uint64(b)
    a_lo, a_hi = a & MASK32, a >> np.uint64(32)
    b_lo, b_hi = b & MASK32, b >> np.uint64(32)
    with np.errstate(over="ignore"):
        ll = a_lo * b_lo
        lh = a_lo * b_hi
        hl = a_hi * b_lo
        hh = a_hi * b_hi
        mid = (ll >> np.uint64(32)) + (lh & MASK32) + (hl & MASK32)
        return hh + (lh >> np.uint64(32)) + (hl >> np.uint64(32)) + (mid >> np.uint64(32))


def bounded(seed: int, idx, n: int) -> np.ndarray:
    """Integers in [0, n) as ``(u * n) >> 64``."""
    return mulhi64(u64(seed, idx), n)


def uniform(seed: int, idx, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """binary64 draws in [lo, hi); for [-1, 1) exactly ``2*((u>>11)*2**-53)-1``."""
    f = (u64(seed, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    if lo == -1.0 and hi == 1.0:
        return 2.0 * f - 1.0
    return lo + (hi - lo) * f


def start_vector(n: int, seed: int = SEED_START, offset: int = 0) -> np.ndarray:
    """Un-normalised Lanczos start vector s_i = uniform[-1,1)(seed, offset+i)."""
    return uniform(seed, np.arange(offset, offset + n, dtype=np.uint64))


# ---------------------------------------------------------------------------
# Model definitions (one-body matrix h = -t and on-site U) for the workloads.
# Hopping matrices are built by summing over bonds, so coincident bonds add.
# ---------------------------------------------------------------------------

def chain(L: int, t: float = 1.0, pbc: bool = True) -> np.ndarray:
    """1D chain, h[i, i+1] = h[i+1, i] = -t, plus the wrap bond (0, L-1) if pbc."""
    h = np.zeros((L, L))
    bonds = [(i, i + 1) for i in range(L - 1)]
    if pbc and L > 1:
        bonds.append((L - 1, 0))
    for a, b in bonds:
        h[a, b] += -t
        h[b, a] += -t
    return h


def square(Lx: int, Ly: int, t: float = 1.0, tp: float = 0.0) -> np.ndarray:
    """Lx x Ly torus, site = y*Lx + x; H = -t sum_nn - t' sum_nnn (h = -t, -t')."""
    n = Lx * Ly
    h = np.zeros((n, n))

    def s(x, y):
        return (y % Ly) * Lx + (x % Lx)

    for y in range(Ly):
        for x in range(Lx):
            i = s(x, y)
            for (dx, dy, amp) in ((1, 0, -t), (0, 1, -t), (1, 1, -tp), (1, -1, -tp)):
                if amp == 0.0:
                    continue
                j = s(x + dx, y + dy)
                if j == i:
                    continue
                h[i, j] += amp
                h[j, i] += amp
    return h


def uniform_U(L: int, U: float) -> np.ndarray:
    return np.full(L, float(U))


def siam(model: int, U: float = 4.0, seed: int = SEED_MODELS):
    """Single-impurity Anderson model number ``model``.

    Site 0 is the impurity (eps_d = -U/2, U on site 0 only), sites 1..n_bath
    the bath with eps_k ~ U[-2, 2) and hybridisations V_k ~ U[0, 1).
    n_bath = 5 + bounded(u, 3).  Draw indices: model*64 + 0 for n_bath,
    model*64 + 1 + k for eps_k, model*64 + 32 + k for V_k.
    Returns (h, Uarr).
    """
    base = model * 64
    nb = 5 + int(bounded(seed, [base], 3)[0])
    L = 1 + nb
    k = np.arange(nb, dtype=np.uint64)
    eps = uniform(seed, base + 1 + k, -2.0, 2.0)
    V = uniform(seed, base + 32 + k, 0.0, 1.0)
    h = np.zeros((L, L))
    h[0, 0] = -U / 2.0
    for j in range(nb):
        h[1 + j, 1 + j] = eps[j]
        h[0, 1 + j] = V[j]
        h[1 + j, 0] = V[j]
    Uarr = np.zeros(L)
    Uarr[0] = U
    return h, Uarr


# ---------------------------------------------------------------------------
# Query generators for the ranking workloads.
# ---------------------------------------------------------------------------

def comb_query_ranks(n: int, dim: int, seed: int = SEED_COMB_QUERIES, offset: int = 0) -> np.ndarray:
    """Target ranks u_q = bounded(seed, q, dim); the query pattern is unrank(u_q)."""
    return bounded(seed, np.arange(offset, offset + n, dtype=np.uint64), dim)


def trie_member_set(n: int, bits: int, seed: int = SEED_TRIE_SET) -> np.ndarray:
    """``n`` distinct ``bits``-bit patterns, sorted ascending.

    Draws u(seed, i) & (2**bits - 1) for i = 0, 1, 2, ... and keeps the first
    ``n`` distinct values (in draw order), then sorts them.
    """
    mask = np.uint64((1 << bits) - 1)
    extra = max(1024, n // 64)
    while True:
        draws = u64(seed, np.arange(n + extra, dtype=np.uint64)) & mask
        vals, first = np.unique(draws, return_index=True)
        if vals.size >= n:
            keep = np.sort(first)[:n]
            return np.sort(draws[keep])
        extra *= 2


def trie_query_members(n: int, nset: int, seed: int = SEED_TRIE_QUERIES, offset: int = 0) -> np.ndarray:
    """Member indices j_q = bounded(seed, q, nset); the query is set[j_q]."""
    return bounded(seed, np.arange(offset, offset + n, dtype=np.uint64), nset)


# ---------------------------------------------------------------------------
# State sets (inputs of the trie-ranked and set Hamiltonians and of the
# ranking benchmarks): every pattern of a fixed popcount, listed in
# increasing order by splitting the word into a high and a low half.
# ---------------------------------------------------------------------------

_POP8 = np.array([bin(i).count("1") for i in range(256)], dtype=np.int64)


def _popcount(v: np.ndarray) -> np.ndarray:
    """Set bits of each value below 2**24 (a byte table)."""
    v = v.astype(np.int64)
    return _POP8[v & 255] + _POP8[(v >> 8) & 255] + _POP8[(v >> 16) & 255]


def popcount_states(M: int, N: int) -> np.ndarray:
    """All M-bit patterns with N set bits (M <= 64), in increasing order."""
    if N < 0 or N > M:
        return np.empty(0, dtype=np.uint64)
    if M > 44:
        raise ValueError("popcount_states enumerates words of at most 44 bits")   # halves below 2**24
    lo = M // 2
    hi = M - lo
    low = np.arange(1 << lo, dtype=np.uint64)
    high = np.arange(1 << hi, dtype=np.uint64)
    pl = _popcount(low)
    ph = _popcount(high)
    by_pop = [low[pl == k] for k in range(lo + 1)]
    blocks = []
    for u in high:                       # increasing high half, then increasing low half
        k = N - int(ph[int(u)])
        if 0 <= k <= lo and by_pop[k].size:
            blocks.append((u << np.uint64(lo)) | by_pop[k])
    return np.concatenate(blocks) if blocks else np.empty(0, dtype=np.uint64)


def fixed_N_states(L: int, N: int) -> np.ndarray:
    """All 2L-bit states with N particles in total (every S_z), sorted."""
    return popcount_states(2 * L, N)


def sector_states(L: int, Nup: int, Ndn: int) -> np.ndarray:
    """The (N_up, N_dn) sector as 2L-bit patterns (spin down in the low L
    bits), sorted: spin-up pattern major, spin-down pattern minor."""
    up = popcount_states(L, Nup)
    dn = popcount_states(L, Ndn)
    return ((up[:, None] << np.uint64(L)) | dn[None, :]).ravel()


# ---------------------------------------------------------------------------
# Momentum-basis Hubbard ring (operator-product form of the Hamiltonian).
# Orbitals: momentum k_m = 2 pi m / L, m = 0..L-1; spin down m -> bit m,
# spin up m -> bit L + m.  Operator code = 2 * orbital + 1 for a creator,
# 2 * orbital for an annihilator; a term is (coefficient, [codes left to right]).
# ---------------------------------------------------------------------------

def momentum_ring_terms(L: int, t: float = 1.0, U: float = 4.0):
    """H = sum_{m,s} -2t cos(k_m) n_{m s}
         + (U/L) sum_{m,m',q} c^dag_{m+q,up} c^dag_{m'-q,dn} c_{m',dn} c_{m,up}
    (momenta mod L): the Fourier transform of the periodic ring with on-site U."""
    terms = []
    for m in range(L):
        e = -2.0 * t * np.cos(2.0 * np.pi * m / L)
        for off in (0, L):
            terms.append((float(e), [2 * (off + m) + 1, 2 * (off + m)]))
    for m in range(L):
        for mp in range(L):
            for q in range(L):
                a = L + (m + q) % L          # up, created
                b = (mp - q) % L             # down, created
                terms.append((U / L, [2 * a + 1, 2 * b + 1, 2 * mp, 2 * (L + m)]))
    return terms


def two_orbital_impurity_terms(n_bath: int = 4, U: float = 4.0, J: float = 0.6, seed: int = SEED_MODELS,
                               model: int = 0):
    """Operator-product term list of a two-orbital Anderson impurity with the
    Kanamori interaction (a multi-orbital model whose U_ijkl goes beyond
    density-density terms), as (coefficient, [operator codes]) with code
    2 * orbital + 1 for a creator and 2 * orbital for an annihilator.

    Sites 0 and 1 are the impurity orbitals a, b; sites 2 .. 1 + n_bath the
    bath; spin-orbital p is (site p, down), L + p is (site p, up), L = 2 + n_bath.
    One-body: eps_a = -U/2 - 0.1, eps_b = -U/2 + 0.1 on the orbitals, bath
    energies eps_k ~ U[-2, 2), hybridisations V_mk ~ U[0, 1) between each
    orbital and each bath site (draw indices model*64 + 1 + k for eps_k,
    model*64 + 16 + m*8 + k for V_mk).  Interaction (U' = U - 2J):
        U sum_m n_m,up n_m,dn + U' sum_{s,s'} n_a,s n_b,s' - J sum_s n_a,s n_b,s
        - J (c+_a,up c_a,dn c+_b,dn c_b,up + h.c.)      (spin flip)
        + J (c+_a,up c+_a,dn c_b,dn c_b,up + h.c.)      (pair hopping).
    Every term comes with its adjoint, so the operator is symmetric; it
    conserves N_up and N_dn."""
    L = 2 + n_bath
    base = model * 64
    k = np.arange(n_bath, dtype=np.uint64)
    eps = uniform(seed, base + 1 + k, -2.0, 2.0)
    terms = []

    def cr(site, spin):
        return 2 * (site + (L if spin else 0)) + 1

    def an(site, spin):
        return 2 * (site + (L if spin else 0))

    for spin in (0, 1):
        terms.append((-U / 2 - 0.1, [cr(0, spin), an(0, spin)]))
        terms.append((-U / 2 + 0.1, [cr(1, spin), an(1, spin)]))
        for j in range(n_bath):
            terms.append((float(eps[j]), [cr(2 + j, spin), an(2 + j, spin)]))
    for m in (0, 1):
        V = uniform(seed, base + 16 + m * 8 + k, 0.0, 1.0)
        for j in range(n_bath):
            for spin in (0, 1):
                terms.append((float(V[j]), [cr(m, spin), an(2 + j, spin)]))
                terms.append((float(V[j]), [cr(2 + j, spin), an(m, spin)]))
    Up = U - 2 * J
    for m in (0, 1):
        terms.append((U, [cr(m, 1), an(m, 1), cr(m, 0), an(m, 0)]))
    for s in (0, 1):
        for sp in (0, 1):
            terms.append((Up - (J if s == sp else 0.0), [cr(0, s), an(0, s), cr(1, sp), an(1, sp)]))
    terms.append((-J, [cr(0, 1), an(0, 0), cr(1, 0), an(1, 1)]))
    terms.append((-J, [cr(1, 1), an(1, 0), cr(0, 0), an(0, 1)]))
    terms.append((J, [cr(0, 1), cr(0, 0), an(1, 0), an(1, 1)]))
    terms.append((J, [cr(1, 1), cr(1, 0), an(0, 0), an(0, 1)]))
    return L, terms


def momentum_sector_states(L: int, Nup: int, Ndn: int, K: int) -> np.ndarray:
    """Sorted 2L-bit states with N_up, N_dn particles and total momentum
    sum of m over occupied orbitals = K (mod L)."""
    import itertools
    out = []
    for up in itertools.combinations(range(L), Nup):
        for dn in itertools.combinations(range(L), Ndn):
            if (sum(up) + sum(dn)) % L == K % L:
                out.append(sum(1 << d for d in dn) | (sum(1 << u for u in up) << L))
    return np.array(sorted(out), dtype=np.uint64)
