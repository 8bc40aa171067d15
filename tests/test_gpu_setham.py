"""Trie-ranked on-the-fly H·v over arbitrary state sets against the
oracle's literal operator application on the same sets."""
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


def run(G, L, h, U, states, R, check, fp):
    import torch
    Sh = G.gbr_setham_create(L, h, U, states, R)
    info = G.gbr_setham_info(Sh)
    assert info["dim"] == states.size
    x = torch.from_numpy(S.start_vector(states.size, 3)).cuda()
    if fp == 32:
        x = x.float()
    y = torch.full_like(x, float("nan"))
    G.gbr_setham_hv(Sh, x, y, check=check)
    return y.double().cpu().numpy(), x.double().cpu().numpy(), info


@pytest.mark.parametrize("fp", [64, 32])
@pytest.mark.parametrize("R", [4, 8, 5])
def test_sector_set_matches_oracle_and_factored_hv(G, fp, R):
    import torch
    L = 6
    h, U = S.square(3, 2, 1.0, -0.3), S.uniform_U(6, 4.0)
    st = oracle.sector_states(L, 3, 2)
    for check in (1, 0):
        y, x, info = run(G, L, h, U, st, R, check, fp)
        y_ref = oracle.hv(L, h, U, 3, 2, x)
        assert rel_inf(y, y_ref) <= (TOL64 if fp == 64 else TOL32), (check, R)
    assert info["elements"] == oracle.count_elements(L, h, 3, 2)


@pytest.mark.parametrize("L,N", [(5, 5), (6, 6), (8, 7)])
def test_fixed_total_N_every_Sz(G, L, N):
    h, U = S.chain(L), S.uniform_U(L, 2.5)
    st = oracle.fixed_N_states(L, N)
    for fp in (64, 32):
        y, x, _ = run(G, L, h, U, st, 8, 1, fp)
        y_ref, drop = oracle.hv_set(L, h, U, st, x)
        assert drop == 0
        assert rel_inf(y, y_ref) <= (TOL64 if fp == 64 else TOL32)


def test_open_subset_is_projected(G):
    L = 7
    h, U = S.chain(L, pbc=False) + np.diag(np.linspace(-0.5, 0.5, 7)), np.array([0, 1, 2, 3, 2, 1, 0.5])
    full = oracle.sector_states(L, 3, 3)
    rng = np.random.default_rng(11)
    sub = np.sort(full[rng.choice(full.size, size=500, replace=False)])
    y, x, _ = run(G, L, h, U, sub, 8, 1, 64)
    y_ref, drop = oracle.hv_set(L, h, U, sub, x)
    assert drop > 0
    assert rel_inf(y, y_ref) <= TOL64


def test_large_fixed_N_set_sampled(G):
    """Every S_z of the 10-site ring at 10 particles (184,756 states)."""
    L, N = 10, 10
    h, U = S.chain(L), S.uniform_U(L, 4.0)
    st = oracle.fixed_N_states(L, N)
    y, x, info = run(G, L, h, U, st, 8, 1, 64)
    y_ref, drop = oracle.hv_set(L, h, U, st, x)
    assert drop == 0 and rel_inf(y, y_ref) <= TOL64
    assert info["trie_elements"] >= st.size


@pytest.mark.parametrize("fp", [64, 32])
def test_bisection_ranking_gives_the_same_bits(G, fp):
    """Bisection in the member list (the baseline of Fig. eig-timings) and
    the trie walk rank every target identically, so the products agree bit
    for bit; on an open subset both drop the same targets."""
    import torch
    L = 7
    h, U = S.chain(L, pbc=False), S.uniform_U(L, 4.0)
    full = oracle.sector_states(L, 3, 3)
    rng = np.random.default_rng(5)
    for st in (full, np.sort(full[rng.choice(full.size, size=700, replace=False)])):
        Sh = G.gbr_setham_create(L, h, U, st, 8)
        x = torch.from_numpy(S.start_vector(st.size, 3)).cuda()
        if fp == 32:
            x = x.float()
        ya, yb = torch.full_like(x, float("nan")), torch.full_like(x, float("nan"))
        G.gbr_setham_hv(Sh, x, ya, check=1)
        G.gbr_setham_set_bisect(Sh, True)
        G.gbr_setham_hv(Sh, x, yb, check=0)
        assert torch.equal(ya, yb)
        y_ref, _ = oracle.hv_set(L, h, U, st, x.double().cpu().numpy())
        assert rel_inf(yb.double().cpu().numpy(), y_ref) <= (TOL64 if fp == 64 else TOL32)


@pytest.mark.parametrize("fp", [64, 32])
def test_both_trie_orders_give_the_same_bits(G, fp):
    """The set H·v ranks through a trie dispatched either from the least
    (the paper's order) or the most significant chunk; ranks are equal, so
    the products agree bit for bit, on a sector and on an open subset."""
    import torch
    L = 8
    h, U = S.square(4, 2, 1.0, -0.3), S.uniform_U(8, 4.0)
    full = oracle.sector_states(L, 3, 4)
    rng = np.random.default_rng(8)
    for st, check in ((full, 0), (np.sort(full[rng.choice(full.size, size=900, replace=False)]), 1)):
        x = torch.from_numpy(S.start_vector(st.size, 3)).cuda()
        if fp == 32:
            x = x.float()
        ys = []
        for msb in (False, True):
            Sh = G.gbr_setham_create(L, h, U, st, 8, msb_first=msb)
            y = torch.full_like(x, float("nan"))
            G.gbr_setham_hv(Sh, x, y, check=check)
            ys.append(y)
        assert torch.equal(ys[0], ys[1])
        y_ref, _ = oracle.hv_set(L, h, U, st, x.double().cpu().numpy())
        assert rel_inf(ys[1].double().cpu().numpy(), y_ref) <= (TOL64 if fp == 64 else TOL32)
