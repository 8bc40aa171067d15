"""Parity of the GPU rank / unrank kernels with the oracle: bit-exact."""
import math

import numpy as np
import pytest

import gbr_synth as S
import oracle
from gpu_common import as_u32, as_u64, lib, to_dev_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return lib()


def rank_both(G, c, pats_dev, check=0):
    import torch
    n = pats_dev.numel()
    r32 = torch.empty(n, dtype=torch.int32, device="cuda")
    r64 = torch.empty(n, dtype=torch.int64, device="cuda")
    G.gbr_comb_rank(c, pats_dev, r64, check=check)
    dim, _ = G.gbr_comb_info(c)
    if dim <= 2**32:
        G.gbr_comb_rank(c, pats_dev, r32, check=check)
        return as_u32(r32).astype(np.uint64), as_u64(r64)
    return None, as_u64(r64)


@pytest.mark.parametrize("R", [3, 8])
def test_comb_exhaustive_small_sectors(G, R):
    import torch
    for M in range(1, 17):
        for N in range(0, M + 1):
            lst = oracle.enumerate_sector(M, N)
            c = G.gbr_comb_create(M, N, R)
            r32, r64 = rank_both(G, c, to_dev_u64(lst), check=1)
            want = np.arange(lst.size, dtype=np.uint64)
            assert np.array_equal(r64, want), (M, N)
            assert np.array_equal(r32, want), (M, N)
            pats = torch.empty(lst.size, dtype=torch.int64, device="cuda")
            G.gbr_comb_unrank(c, torch.arange(lst.size, dtype=torch.int64, device="cuda"), pats)
            assert np.array_equal(as_u64(pats), lst), (M, N)


def test_comb_check_mode_flags_non_members(G):
    M, N = 20, 10
    c = G.gbr_comb_create(M, N, 8)
    rng = np.random.default_rng(1)
    q = rng.integers(0, 1 << 22, size=5000, dtype=np.uint64)       # many have bits >= M or popcount != N
    _, r64 = rank_both(G, c, to_dev_u64(q), check=1)
    for a, r in zip(q, r64):
        a = int(a)
        if a < (1 << M) and bin(a).count("1") == N:
            assert int(r) == oracle.rank_count(M, a)
        else:
            assert int(r) == 0xFFFFFFFFFFFFFFFF
    # without the check every access stays inside the table: members still right
    lst = oracle.enumerate_sector(M, N)[::37]
    _, r64 = rank_both(G, c, to_dev_u64(lst), check=0)
    assert np.array_equal(r64, np.arange(0, math.comb(M, N), 37, dtype=np.uint64))


@pytest.mark.parametrize("M,N,R", [(64, 32, 8), (64, 5, 8), (64, 59, 4), (48, 24, 12), (33, 16, 8)])
def test_comb_large_sectors_against_oracle(G, M, N, R):
    import torch
    D = math.comb(M, N)
    u = S.bounded(11, np.arange(4000, dtype=np.uint64), D)
    u = np.concatenate([u, np.array([0, D - 1], dtype=np.uint64)])
    c = G.gbr_comb_create(M, N, R)
    pats = torch.empty(u.size, dtype=torch.int64, device="cuda")
    G.gbr_comb_unrank(c, to_dev_u64(u), pats)
    p = as_u64(pats)
    for ui, a in zip(u[::40], p[::40]):
        assert int(a) == oracle.unrank(M, N, int(ui))
    _, r64 = rank_both(G, c, pats, check=1)
    assert np.array_equal(r64, u)
    # out-of-range ranks unrank to the not-found pattern
    G.gbr_comb_unrank(c, to_dev_u64(np.array([D, D + 5], dtype=np.uint64)), pats[:2])
    assert np.all(as_u64(pats[:2]) == np.uint64(0xFFFFFFFFFFFFFFFF))


@pytest.mark.parametrize("n", [0, 1, 7, 1023, 1024, 1025, 4097, 100003])
def test_comb_ragged_lengths(G, n):
    import torch
    M, N = 32, 16
    D = math.comb(M, N)
    c = G.gbr_comb_create(M, N, 8)
    u = S.bounded(12, np.arange(n, dtype=np.uint64), D)
    pats = torch.empty(n, dtype=torch.int64, device="cuda")
    r = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    if n:
        G.gbr_comb_unrank(c, to_dev_u64(u), pats)
    G.gbr_comb_rank(c, pats, r, check=1)
    assert np.array_equal(as_u32(r).astype(np.uint64), u)


def test_comb_full_size_2pow28(G):
    """Ranking workload: 2^28 seeded queries over the M=32, N=16 sector."""
    import torch
    import gbr_synth.gpu as SG
    M, N, n = 32, 16, 1 << 28
    D = math.comb(M, N)
    c = G.gbr_comb_create(M, N, 8)
    u = SG.bounded(S.SEED_COMB_QUERIES, n, D)
    pats = torch.empty(n, dtype=torch.int64, device="cuda")
    G.gbr_comb_unrank(c, u, pats)
    r = torch.empty(n, dtype=torch.int32, device="cuda")
    G.gbr_comb_rank(c, pats, r)
    assert torch.equal(r.to(torch.int64) & 0xFFFFFFFF, u)          # rank(unrank(u)) = u at full size
    idx = np.unique(S.bounded(13, np.arange(3000, dtype=np.uint64), n)).astype(np.int64)
    us = S.bounded(S.SEED_COMB_QUERIES, idx.astype(np.uint64), D)
    ps = as_u64(pats[torch.from_numpy(idx).cuda()])
    assert np.array_equal(as_u64(u[torch.from_numpy(idx).cuda()]), us)   # the GPU generator is the numpy one
    for ui, a in zip(us[:600], ps[:600]):
        assert int(a) == oracle.unrank(M, N, int(ui))
        assert oracle.rank_count(M, int(a)) == int(ui)


# ------------------------------------------------------------------- tries

@pytest.mark.parametrize("msb_first", [False, True])
@pytest.mark.parametrize("M,R", [(7, 3), (10, 4), (12, 5), (16, 8), (20, 8), (24, 8), (13, 16)])
def test_trie_random_sets(G, M, R, msb_first):
    """Both dispatch orders: the paper's (sizes equal to the oracle's) and
    most significant chunk first; ranks, unranks, non-member flags and the
    bisection baseline identical."""
    import torch
    rng = np.random.default_rng(100 * M + R)
    k = min(5000, (1 << M) // 3)
    members = np.sort(rng.choice(1 << M, size=k, replace=False).astype(np.uint64))
    t = G.gbr_trie_create(members, M, R, msb_first=msb_first)
    info = G.gbr_trie_info(t)
    osize, _ = oracle.trie_build(members, M, R, with_table=False)
    assert info["n_members"] == k
    if not msb_first:
        assert info["n_elements"] == osize
    r = torch.empty(k, dtype=torch.int32, device="cuda")
    G.gbr_trie_rank(t, to_dev_u64(members), r, check=1)
    assert np.array_equal(as_u32(r), np.arange(k, dtype=np.uint32))
    back = torch.empty(k, dtype=torch.int64, device="cuda")
    G.gbr_trie_unrank(t, r, back)
    assert np.array_equal(as_u64(back), members)
    # non-members, including patterns wider than M: flagged with check, in bounds without
    q = rng.integers(0, 1 << (M + 2), size=4000, dtype=np.uint64)
    r2 = torch.empty(q.size, dtype=torch.int64, device="cuda")
    G.gbr_trie_rank(t, to_dev_u64(q), r2, check=1)
    want = oracle.rank_bisect_many(members, q)
    got = as_u64(r2)
    for w, g in zip(want, got):
        assert (w >= 0 and int(g) == w) or (w < 0 and g == np.uint64(0xFFFFFFFFFFFFFFFF))
    G.gbr_trie_rank(t, to_dev_u64(q), r2, check=0)
    # the bisection baseline over the same member list agrees bit for bit
    r3 = torch.empty(q.size, dtype=torch.int64, device="cuda")
    G.gbr_trie_rank_bisect(t, to_dev_u64(q), r3, check=1)
    assert np.array_equal(as_u64(r3), got)
    r4 = torch.empty(k, dtype=torch.int32, device="cuda")
    G.gbr_trie_rank_bisect(t, to_dev_u64(members), r4, check=1)
    assert np.array_equal(as_u32(r4), np.arange(k, dtype=np.uint32))
    torch.cuda.synchronize()


def test_trie_paper_sector_M28_N5(G):
    import torch
    lst = oracle.enumerate_sector(28, 5)
    t = G.gbr_trie_create(lst, 28, 8)
    assert round(G.gbr_trie_info(t)["n_elements"] / lst.size, 2) == 10.45
    r = torch.empty(lst.size, dtype=torch.int32, device="cuda")
    G.gbr_trie_rank(t, to_dev_u64(lst), r, check=1)
    assert np.array_equal(as_u32(r), np.arange(lst.size, dtype=np.uint32))


@pytest.mark.parametrize("msb_first", [False, True])
def test_trie_full_size_40bit(G, msb_first):
    """Trie workload: 2^24 distinct 40-bit patterns, 2^28 member queries."""
    import torch
    import gbr_synth.gpu as SG
    nset, n = 1 << 24, 1 << 28
    members = S.trie_member_set(nset, 40)
    t = G.gbr_trie_create(members, 40, 8, msb_first=msb_first)
    mdev = to_dev_u64(members)
    j = SG.bounded(S.SEED_TRIE_QUERIES, n, nset)
    pats = mdev[j]
    r = torch.empty(n, dtype=torch.int32, device="cuda")
    G.gbr_trie_rank(t, pats, r, check=1)
    assert torch.equal(r.to(torch.int64), j)
    rb = torch.empty(n, dtype=torch.int32, device="cuda")
    G.gbr_trie_rank_bisect(t, pats, rb, check=1)
    assert torch.equal(rb, r)
    sel = np.unique(S.bounded(14, np.arange(2000, dtype=np.uint64), n)).astype(np.int64)
    ps = as_u64(pats[torch.from_numpy(sel).cuda()])
    assert np.array_equal(oracle.rank_bisect_many(members, ps), as_u32(r[torch.from_numpy(sel).cuda()]).astype(np.int64))
    # random 40-bit patterns (about 1.5 % members): the non-members walk to
    # arbitrary entries, also through the compressed copies of the large
    # levels, and the check flags every one of them
    q = SG.bounded(15, 1 << 16, 1 << 40)
    q[::7] = mdev[SG.bounded(16, q[::7].numel(), nset)]
    rq = torch.empty(q.numel(), dtype=torch.int32, device="cuda")
    G.gbr_trie_rank(t, q, rq, check=1)
    exp = oracle.rank_bisect_many(members, as_u64(q))
    got = as_u32(rq).astype(np.int64)
    got[got == 0xFFFFFFFF] = -1
    assert np.array_equal(got, exp) and (exp >= 0).sum() >= q.numel() // 7


def test_comb_unaligned_views_use_the_scalar_kernel(G):
    """Views that start 8 bytes into a buffer are not 16-byte aligned: the
    per-element kernel handles them with the same results."""
    import torch
    M, N = 30, 13
    D = math.comb(M, N)
    c = G.gbr_comb_create(M, N, 8)
    u = S.bounded(15, np.arange(10001, dtype=np.uint64), D)
    pats = torch.empty(u.size + 1, dtype=torch.int64, device="cuda")
    G.gbr_comb_unrank(c, to_dev_u64(u), pats[1:])
    r = torch.empty(u.size + 1, dtype=torch.int32, device="cuda")
    G.gbr_comb_rank(c, pats[1:], r[1:], check=1)
    assert np.array_equal(as_u32(r[1:]).astype(np.uint64), u)
    r64 = torch.empty(u.size + 1, dtype=torch.int64, device="cuda")
    G.gbr_comb_rank(c, pats[1:], r64[1:])
    assert np.array_equal(as_u64(r64[1:]), u)


def test_trie_edge_cases(G):
    """One member; 64-bit patterns; empty query batches."""
    import torch
    one = np.array([0b1011], dtype=np.uint64)
    t = G.gbr_trie_create(one, 4, 3)
    r = torch.empty(3, dtype=torch.int64, device="cuda")
    G.gbr_trie_rank(t, to_dev_u64(np.array([0b1011, 0b0011, 0], dtype=np.uint64)), r, check=1)
    assert list(as_u64(r)) == [0, 2**64 - 1, 2**64 - 1]
    G.gbr_trie_rank(t, torch.empty(0, dtype=torch.int64, device="cuda"), torch.empty(0, dtype=torch.int64, device="cuda"))
    rng = np.random.default_rng(64)
    wide = np.unique(rng.integers(0, 2**63, size=3000, dtype=np.uint64) * np.uint64(2) + np.uint64(1))
    t64 = G.gbr_trie_create(wide, 64, 8)
    r64 = torch.empty(wide.size, dtype=torch.int64, device="cuda")
    G.gbr_trie_rank(t64, to_dev_u64(wide), r64, check=1)
    assert np.array_equal(as_u64(r64), np.arange(wide.size, dtype=np.uint64))
    G.gbr_trie_rank_bisect(t64, to_dev_u64(wide), r64, check=1)
    assert np.array_equal(as_u64(r64), np.arange(wide.size, dtype=np.uint64))
