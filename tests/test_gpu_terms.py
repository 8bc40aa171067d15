"""On-the-fly H·v for general operator-product terms (tuples built by the
product rule of Fig. mul) over trie-ranked sets, against the oracle's
literal application of the same products."""
import numpy as np
import pytest

import gbr_synth as S
import oracle
from gpu_common import lib, rel_inf

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


@pytest.fixture(scope="module")
def G():
    return lib()


def tuples(G, terms):
    return [G.gbr_term_product(ops, coef) for coef, ops in terms]


def run(G, M, terms, states, check=1, fp=64, R=8, seed=3):
    import torch
    T = G.gbr_termham_create(M, tuples(G, terms), states, R)
    x = torch.from_numpy(S.start_vector(states.size, seed)).cuda()
    if fp == 32:
        x = x.float()
    y = torch.full_like(x, float("nan"))
    G.gbr_termham_hv(T, x, y, check=check)
    return y.double().cpu().numpy(), x.double().cpu().numpy(), G.gbr_termham_info(T)


@pytest.mark.parametrize("L,N", [(4, 2), (6, 3), (7, 3)])
def test_momentum_ring_every_K_sector(G, L, N):
    terms = S.momentum_ring_terms(L, 1.0, 4.0)
    for K in range(L):
        st = S.momentum_sector_states(L, N, N, K)
        for fp in (64, 32):
            y, x, info = run(G, 2 * L, terms, st, fp=fp)
            y_ref, drop = oracle.hv_ops(terms, st, x)
            assert drop == 0
            assert rel_inf(y, y_ref) <= (TOL64 if fp == 64 else TOL32), (L, K, fp)
    # bisection ranking (the baseline) gives the same product
    import torch
    st = S.momentum_sector_states(L, N, N, 0)
    T = G.gbr_termham_create(2 * L, tuples(G, terms), st, 8)
    x = torch.from_numpy(S.start_vector(st.size, 3)).cuda()
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    G.gbr_termham_hv(T, x, y1)
    G.gbr_termham_set_bisect(T, True)
    G.gbr_termham_hv(T, x, y2)
    assert torch.equal(y1, y2)


def test_real_space_terms_match_the_factored_hv(G):
    import torch
    L = 6
    h, U = S.square(3, 2, 1.0, -0.3), S.uniform_U(6, 4.0)
    terms = [(h[p, q], [2 * (sp + p) + 1, 2 * (sp + q)]) for sp in (0, L) for p in range(L) for q in range(L)
             if h[p, q] != 0.0]
    terms += [(U[p], [2 * (L + p) + 1, 2 * p + 1, 2 * p, 2 * (L + p)]) for p in range(L)]
    st = oracle.sector_states(L, 3, 3)
    y, x, info = run(G, 2 * L, terms, st, check=0)
    H = G.gbr_ham_create(L, h, U, 3, 3)
    G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
    yy = torch.empty(st.size, dtype=torch.float64, device="cuda")
    G.gbr_hv(H, torch.from_numpy(x).cuda(), yy)
    assert rel_inf(y, yy.cpu().numpy()) <= TOL64
    # elements: every hop whose left demand holds plus every doubly occupied site's U term
    hops = oracle.count_elements(L, h, 3, 3) - st.size
    doubles = sum(bin(int(a) & (int(a) >> L) & ((1 << L) - 1)).count("1") for a in st)
    assert info["elements"] == hops + doubles


def test_non_hermitian_term_list_gives_the_row_action(G):
    # a lone c^dag_3 c_1 (no conjugate) and a lone pair hop: y = H x exactly
    M = 8
    terms = [(0.7, [2 * 3 + 1, 2 * 1]), (-1.3, [2 * 5 + 1, 2 * 6 + 1, 2 * 2, 2 * 0])]
    st = oracle.enumerate_sector(M, 3)
    y, x, _ = run(G, M, terms, st)
    y_ref, _ = oracle.hv_ops(terms, st, x)
    assert rel_inf(y, y_ref) <= TOL64


def test_open_set_projection_and_radices(G):
    L = 5
    terms = S.momentum_ring_terms(L, 1.0, 2.0)
    full = np.concatenate([S.momentum_sector_states(L, 2, 2, K) for K in range(L)])
    full.sort()
    rng = np.random.default_rng(4)
    sub = np.sort(rng.choice(full, size=40, replace=False))
    for R in (3, 8, 11):
        y, x, _ = run(G, 2 * L, terms, sub, R=R)
        y_ref, drop = oracle.hv_ops(terms, sub, x)
        assert drop > 0 and rel_inf(y, y_ref) <= TOL64
