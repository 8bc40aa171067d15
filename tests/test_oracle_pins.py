"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign, an off-by-one index, a transposed operand) fails at least one of
them: paper-printed examples, brute-force enumeration, closed forms of
textbook limits, spectral invariances, and dense diagonalisation.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import gbr_synth as S
import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def alpha_of(comb):
    return sum(1 << c for c in comb)


# ---------------------------------------------------------------- paper values

def test_full_space_rank_example():
    g = GOLD["full_space_rank"]
    everything = np.sort(np.concatenate([oracle.enumerate_sector(6, n) for n in range(7)]))
    assert oracle.rank_bisect(everything, int(g["bits"], 2)) == g["rank"]


def test_C43_example():
    g = GOLD["comb_C43"]
    lst = oracle.enumerate_sector(g["M"], g["N"])
    assert [int(a) for a in lst] == [alpha_of(c) for c in g["combinations"]]
    for comb, r in zip(g["combinations"], g["ranks"]):
        a = alpha_of(comb)
        assert oracle.rank_count(g["M"], a) == r
        assert oracle.rank_bisect(lst, a) == r
        assert oracle.unrank(g["M"], g["N"], r) == a


def test_cns_and_alpha_examples():
    assert oracle.rank_count(4, alpha_of(GOLD["cns_310"]["combination"])) == GOLD["cns_310"]["rank"]
    assert alpha_of(GOLD["alpha_310"]["combination"]) == GOLD["alpha_310"]["alpha"]


def test_binomial_table_size_and_pascal():
    # binomials for 0 <= c < 64 and 1 < k <= 64, 8 bytes each: 64*63*8 B < 32 KiB = 64*64*8 B
    assert 64 * 64 * 8 == GOLD["binom_table_kib"]["KiB"] * 1024
    for n in range(1, 65):
        for k in range(0, n + 1):
            assert oracle.binom(n, k) == oracle.binom(n - 1, k - 1) + oracle.binom(n - 1, k) if k else oracle.binom(n, 0) == 1
    assert oracle.binom(64, 32) == math.comb(64, 32)
    assert oracle.binom(5, 7) == 0


def test_trie_worked_example():
    g = GOLD["trie_walk"]
    lst = oracle.enumerate_sector(g["M"], g["N"])
    size, t = oracle.trie_build(lst, g["M"], g["R"])
    for idx, val in g["t"].items():
        assert t[int(idx)] == val, idx
    # node 0100 is reached through t_5 = 8 although its data starts at 9: its smallest child is r = 01
    assert t[5] + 1 == g["node_0100_start"]
    assert oracle.trie_rank(t, g["M"], g["R"], int(g["alpha"], 2)) == g["rank"]
    assert size / lst.size == g["f_approx"]
    for i, a in enumerate(lst):
        assert oracle.trie_rank(t, g["M"], g["R"], int(a)) == i


@pytest.mark.slow
def test_trie_overhead_factors_match_paper():
    g = GOLD["trie_overhead"]
    M = g["M"]
    lists = {}
    for row in g["rows"]:
        N = row["N"]
        if N not in lists:
            lists[N] = oracle.enumerate_sector(M, N)
        size, _ = oracle.trie_build(lists[N], M, row["R"], with_table=False)
        f = size / lists[N].size
        assert round(f, 2) == row["f"], (row, f)


# ------------------------------------------------------------- brute force

@pytest.mark.parametrize("M", list(range(1, 15)))
def test_rank_unrank_brute_force(M):
    for N in range(0, M + 1):
        lst = oracle.enumerate_sector(M, N)
        assert lst.size == math.comb(M, N)
        assert np.all(np.diff(lst.astype(np.int64)) > 0)
        for i, a in enumerate(lst):
            assert oracle.rank_count(M, int(a)) == i
            assert oracle.unrank(M, N, i) == int(a)
        # members found by bisection, non-members reported as -1
        for a in range(1 << M):
            r = oracle.rank_bisect(lst, a)
            if bin(a).count("1") == N:
                assert r >= 0 and int(lst[r]) == a
            else:
                assert r == oracle.NOT_FOUND


def test_rank_unrank_large_sectors():
    # M = 32 and 64: the extremes of the sector and random round trips
    for M, N in ((32, 16), (40, 20), (64, 32), (64, 5)):
        D = math.comb(M, N)
        lo = (1 << N) - 1
        hi = lo << (M - N)
        assert oracle.rank_count(M, lo) == 0
        assert oracle.rank_count(M, hi) == D - 1
        assert oracle.unrank(M, N, 0) == lo and oracle.unrank(M, N, D - 1) == hi
        for u in S.bounded(7, np.arange(200, dtype=np.uint64), D):
            a = oracle.unrank(M, N, int(u))
            assert bin(a).count("1") == N and a < (1 << M)
            assert oracle.rank_count(M, a) == int(u)


@pytest.mark.parametrize("M,R", [(7, 3), (9, 4), (10, 4), (12, 5), (13, 8), (16, 8), (11, 12)])
def test_trie_random_sets_brute_force(M, R):
    rng = np.random.default_rng(M * 100 + R)
    for trial in range(4):
        k = int(rng.integers(1, min(200, 1 << M)))
        members = np.sort(rng.choice(1 << M, size=k, replace=False).astype(np.uint64))
        size, t = oracle.trie_build(members, M, R)
        assert size >= members.size
        for i, a in enumerate(members):
            assert oracle.trie_rank(t, M, R, int(a)) == i


# ------------------------------------------------------------ sector index

@pytest.mark.parametrize("L,Nup,Ndn", [(3, 1, 2), (4, 2, 2), (4, 1, 3), (5, 2, 3), (6, 3, 3)])
def test_sector_index_is_lexicographic_position(L, Nup, Ndn):
    states = oracle.sector_states(L, Nup, Ndn)
    full = [a for a in range(1 << (2 * L))
            if bin(a & ((1 << L) - 1)).count("1") == Ndn and bin(a >> L).count("1") == Nup]
    assert [int(s) for s in states] == full
    for i, a in enumerate(full):
        assert oracle.sector_rank(L, Nup, Ndn, a) == i


# --------------------------------------------------------------------- H

def ham(L, U, kind="chain", **kw):
    if kind == "chain":
        h = S.chain(L, pbc=kw.get("pbc", True))
    else:
        h = S.square(kw["Lx"], kw["Ly"], 1.0, kw.get("tp", 0.0))
    return h, S.uniform_U(h.shape[0], U)


def test_two_site_hubbard_closed_form():
    for U in (0.0, 1.0, 4.0, 8.0):
        h = S.chain(2, t=1.0, pbc=False)
        E0 = oracle.dense_E0(2, h, S.uniform_U(2, U), 1, 1)
        assert abs(E0 - (U - math.sqrt(U * U + 16.0)) / 2.0) < 1e-12


def test_atomic_limit_diagonal():
    L = 4
    Uarr = np.array([1.0, 2.0, 3.5, -0.5])
    H = oracle.dense(L, np.zeros((L, L)), Uarr, 2, 2)
    states = oracle.sector_states(L, 2, 2)
    assert np.count_nonzero(H - np.diag(np.diag(H))) == 0
    for i, a in enumerate(states):
        d = int(a) & 0xF
        u = int(a) >> 4
        assert H[i, i] == sum(Uarr[p] for p in range(L) if (d >> p) & 1 and (u >> p) & 1)


@pytest.mark.parametrize("L,N", [(4, 2), (5, 2), (5, 3), (6, 3)])
def test_free_fermion_many_body_spectrum(L, N):
    # at U = 0 every many-body level is a sum of N_up plus N_dn distinct one-body levels
    h, U = ham(L, 0.0)
    e = np.linalg.eigvalsh(h)
    sums = sorted(sum(e[list(a)]) + sum(e[list(b)])
                  for a in itertools.combinations(range(L), N) for b in itertools.combinations(range(L), N))
    ev = np.linalg.eigvalsh(oracle.dense(L, h, U, N, N))
    assert np.allclose(ev, sums, atol=1e-11)


def test_free_ground_state_closed_forms():
    h = S.chain(8)
    assert abs(oracle.dense_E0(8, h, None, 4, 4) - (-4.0 - 4.0 * math.sqrt(2.0))) < 1e-11
    assert abs(oracle.free_E0(h, 4, 4) - (-4.0 - 4.0 * math.sqrt(2.0))) < 1e-12
    # 2x3 torus with diagonal hopping
    h2 = S.square(3, 2, 1.0, -0.3)
    assert abs(oracle.dense_E0(6, h2, None, 2, 3) - oracle.free_E0(h2, 2, 3)) < 1e-11


@pytest.mark.parametrize("Nup,Ndn", [(2, 2), (1, 3), (3, 2)])
def test_noninteracting_kronecker_identity(Nup, Ndn):
    # H = H_up (x) 1 + 1 (x) H_dn at U = 0: the Jordan-Wigner strings of the other spin cancel
    L = 5
    h = S.square(5, 1, 1.0, 0.0) + np.diag(np.arange(L) * 0.125)
    Hup = oracle.dense(L, h, None, Nup, 0)
    Hdn = oracle.dense(L, h, None, 0, Ndn)
    H = oracle.dense(L, h, None, Nup, Ndn)
    K = np.kron(Hup, np.eye(Hdn.shape[0])) + np.kron(np.eye(Hup.shape[0]), Hdn)
    assert np.array_equal(H, K)


def test_site_relabelling_invariance():
    # the spectrum does not depend on how sites are numbered, although every
    # Jordan-Wigner sign changes with the numbering
    h, U = ham(6, 3.0, kind="square", Lx=3, Ly=2, tp=-0.3)
    perm = np.array([4, 0, 5, 2, 1, 3])
    hp = h[np.ix_(perm, perm)]
    e1 = np.linalg.eigvalsh(oracle.dense(6, h, U, 3, 2))
    e2 = np.linalg.eigvalsh(oracle.dense(6, hp, U, 3, 2))
    assert np.allclose(e1, e2, atol=1e-11)


def test_spin_flip_symmetry():
    h, U = ham(6, 4.0)
    assert abs(oracle.dense_E0(6, h, U, 2, 4) - oracle.dense_E0(6, h, U, 4, 2)) < 1e-11


def test_hv_forms_agree_and_matrix_is_symmetric():
    L = 6
    h, U = ham(L, 2.5, kind="square", Lx=3, Ly=2, tp=-0.3)
    Hm = oracle.dense(L, h, U, 3, 2)
    assert np.array_equal(Hm, Hm.T)
    x = S.start_vector(Hm.shape[0])
    y = oracle.hv(L, h, U, 3, 2, x)
    assert np.allclose(y, Hm @ x, rtol=0, atol=1e-12)
    rows = np.arange(0, Hm.shape[0], 7)
    assert np.allclose(oracle.hv_rows(L, h, U, 3, 2, x, rows), y[rows], rtol=0, atol=1e-12)


def element_closed_form(h, L, Nup, Ndn):
    directed = int(np.count_nonzero(h - np.diag(np.diag(h))))
    Dup, Ddn = math.comb(L, Nup), math.comb(L, Ndn)
    per = lambda N: math.comb(L - 2, N - 1) if N >= 1 else 0
    return Dup * Ddn + directed * per(Nup) * Ddn + directed * per(Ndn) * Dup


@pytest.mark.parametrize("kind,L,Nup,Ndn", [("chain", 8, 4, 4), ("chain", 7, 2, 5), ("square", 6, 3, 3), ("square", 8, 4, 3)])
def test_element_count_closed_form(kind, L, Nup, Ndn):
    h = S.chain(L) if kind == "chain" else S.square(L // 2, 2, 1.0, -0.3)
    assert oracle.count_elements(L, h, Nup, Ndn) == element_closed_form(h, L, Nup, Ndn)


# ------------------------------------------------------------------ Lanczos

def test_tridiagonal_bisection_matches_eigvalsh():
    rng = np.random.default_rng(3)
    for k in (1, 2, 5, 40, 200):
        a = rng.normal(size=k)
        b = rng.uniform(0.1, 2.0, size=max(k - 1, 0))
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        assert abs(oracle.tridiag_lowest(a, b) - np.linalg.eigvalsh(T)[0]) < 1e-13 * max(1.0, abs(np.linalg.eigvalsh(T)[0]))


def test_lanczos_matches_dense_ring8():
    h, U = ham(8, 4.0)
    s = S.start_vector(4900)
    r = oracle.lanczos(8, h, U, 4, 4, s, 100, True)
    E_dense = oracle.dense_E0(8, h, U, 4, 4)
    assert r["k"] == 100
    assert abs(r["E0"] - E_dense) <= 1e-10 * abs(E_dense)


def test_lanczos_breakdown_on_tiny_sector():
    # a 2x2 sector is exhausted after two steps
    h, U = ham(2, 1.0, pbc=False)
    r = oracle.lanczos(2, h, U, 1, 0, np.array([0.3, -0.8]), 10, False)
    assert r["k"] == 2
    assert abs(r["E0"] - np.linalg.eigvalsh(oracle.dense(2, h, U, 1, 0))[0]) < 1e-13


def test_seeded_rows_equal_rows_of_the_seeded_vector():
    h, U = ham(6, 2.0, kind="square", Lx=3, Ly=2, tp=-0.3)
    D = oracle.sector_dim(6, 3, 2)
    x = S.start_vector(D)
    rows = np.arange(0, D, 5)
    assert np.array_equal(oracle.hv_rows_seeded(6, h, U, 3, 2, S.SEED_START, rows), oracle.hv_rows(6, h, U, 3, 2, x, rows))


def test_set_hv_equals_sector_hv_and_union_of_sectors():
    # on a sector the set form equals the sector form; on all S_z at fixed N it
    # is block diagonal with the sector blocks
    L = 5
    h, U = ham(L, 3.0, kind="square", Lx=5, Ly=1)
    st = oracle.sector_states(L, 2, 3)
    x = S.start_vector(st.size)
    y, drop = oracle.hv_set(L, h, U, st, x)
    assert drop == 0 and np.allclose(y, oracle.hv(L, h, U, 2, 3, x), rtol=0, atol=1e-13)
    allN = oracle.fixed_N_states(L, 5)
    xa = S.start_vector(allN.size, 9)
    ya, drop = oracle.hv_set(L, h, U, allN, xa)
    assert drop == 0
    for nu in range(0, 6):
        sec = oracle.sector_states(L, nu, 5 - nu)
        idx = np.searchsorted(allN, sec)
        assert np.array_equal(allN[idx], sec)
        assert np.allclose(ya[idx], oracle.hv(L, h, U, nu, 5 - nu, xa[idx]), rtol=0, atol=1e-13)


def test_set_hv_projects_onto_open_sets():
    # a random subset is not closed under H: the dropped terms are exactly the
    # entries of the full product outside the subset
    L = 4
    h, U = ham(L, 2.0)
    full = oracle.sector_states(L, 2, 2)
    rng = np.random.default_rng(5)
    keep = np.sort(rng.choice(full.size, size=20, replace=False))
    sub = full[keep]
    Hm = oracle.dense(L, h, U, 2, 2)
    x = S.start_vector(sub.size)
    y, drop = oracle.hv_set(L, h, U, sub, x)
    assert np.allclose(y, Hm[np.ix_(keep, keep)] @ x, rtol=0, atol=1e-13)
    assert drop > 0


def test_momentum_ring_spectrum_equals_real_space_ring():
    # the momentum-basis Hamiltonian is the real-space periodic ring in another
    # basis: the union of its K_tot sectors has the ring's sector spectrum
    for L, N, U in ((4, 2, 4.0), (5, 2, 3.0), (6, 3, 4.0)):
        terms = S.momentum_ring_terms(L, 1.0, U)
        ev = []
        for K in range(L):
            st = S.momentum_sector_states(L, N, N, K)
            Hm = oracle.dense_ops(terms, st)
            assert np.allclose(Hm, Hm.T, atol=1e-12)
            ev.extend(np.linalg.eigvalsh(Hm))
            _, drop = oracle.hv_ops(terms, st, np.ones(st.size))
            assert drop == 0                         # K_tot is conserved
        ref = np.linalg.eigvalsh(oracle.dense(L, S.chain(L), S.uniform_U(L, U), N, N))
        assert np.allclose(np.sort(ev), ref, atol=1e-10)


def test_operator_products_match_the_one_body_form():
    # the hopping and U terms written as operator products give the same H·v
    L = 5
    h, U = S.square(5, 1, 1.0, 0.0) + np.diag(np.arange(5) * 0.25), np.array([1.0, 0.0, 2.0, 0.5, 0.0])
    terms = []
    for sp in (0, L):
        for p in range(L):
            for q in range(L):
                if h[p, q] != 0.0:
                    terms.append((h[p, q], [2 * (sp + p) + 1, 2 * (sp + q)]))
    for p in range(L):
        if U[p]:
            terms.append((U[p], [2 * (L + p) + 1, 2 * p + 1, 2 * p, 2 * (L + p)]))
    st = oracle.sector_states(L, 2, 3)
    x = S.start_vector(st.size)
    y, drop = oracle.hv_ops(terms, st, x)
    assert drop == 0 and np.allclose(y, oracle.hv(L, h, U, 2, 3, x), rtol=0, atol=1e-13)


@pytest.mark.parametrize("L,N,U", [(4, 2, 4.0), (6, 1, 4.0), (6, 3, 2.0), (6, 3, 4.0), (6, 3, 8.0), (8, 3, 4.0),
                                   (8, 4, 4.0), (8, 4, 1.0)])
def test_bethe_ansatz_matches_dense_diagonalisation(L, N, U):
    """The Lieb-Wu energy of the periodic ring (the independent reference for
    the 18-site ring at U = 4) equals dense diagonalisation of the oracle's
    sector matrix, at closed-shell (N = 4n + 2 electrons) and open-shell
    (N = 4n, both shifts of the quantum numbers) fillings."""
    E_dense = oracle.dense_E0(L, S.chain(L), S.uniform_U(L, U), N, N)
    for shift in (0, 1):
        E_ba = oracle.bethe_ansatz_E0(L, N, N, U, shift=shift)[0]
        assert abs(E_ba - E_dense) <= 1e-12 * abs(E_dense), (shift, E_ba, E_dense)


@pytest.mark.slow
def test_bethe_ansatz_matches_lanczos_ring10():
    """L = 10, N_up = N_dn = 5 (63,504 states, beyond dense): Bethe ansatz
    against the oracle's FP64 Lanczos."""
    L, N, U = 10, 5, 4.0
    D = oracle.sector_dim(L, N, N)
    o = oracle.lanczos(L, S.chain(L), S.uniform_U(L, U), N, N, S.start_vector(D), 120, False)
    E_ba = oracle.bethe_ansatz_E0(L, N, N, U)[0]
    assert abs(E_ba - o["E0"]) <= 1e-12 * abs(E_ba)


def test_bethe_ansatz_weak_coupling_approaches_free_fermions():
    """As U -> 0 the Bethe-ansatz energy of the 18-site ring tends to the
    U = 0 closed form plus the first-order (Hartree) shift U N_up N_dn / L of
    the uniform free ground state; what remains is second order in U (the
    remainder quarters when U halves).  A wrong first-order term would leave
    a remainder linear in U (ratio 2)."""
    L, N = 18, 9
    E_free = oracle.free_E0(S.chain(L), N, N)
    d = {U: oracle.bethe_ansatz_E0(L, N, N, U)[0] - (E_free + U * N * N / L) for U in (0.025, 0.05)}
    assert abs(d[0.025]) < 1e-3
    assert 3.9 <= d[0.05] / d[0.025] <= 4.1


def test_two_orbital_kanamori_terms_are_spin_rotation_invariant():
    """The Kanamori interaction with U' = U - 2J is SU(2) symmetric: every
    level of the (N_up, N_dn) = (2, 4) sector (S >= 1) reappears in the
    (3, 3) sector.  A wrong sign of the spin-flip or pair-hop terms breaks
    it.  The term list is symmetric and conserves N_up and N_dn."""
    L, terms = S.two_orbital_impurity_terms(3)
    ev = {}
    for nu, nd in ((3, 3), (2, 4)):
        st = oracle.sector_states(L, nu, nd)
        Hm = oracle.dense_ops(terms, st)
        assert np.array_equal(Hm, Hm.T)
        _, drop = oracle.hv_ops(terms, st, np.ones(st.size))
        assert drop == 0
        ev[(nu, nd)] = np.linalg.eigvalsh(Hm)
    for e in ev[(2, 4)]:
        assert np.min(np.abs(ev[(3, 3)] - e)) <= 1e-10
