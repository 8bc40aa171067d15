"""Lanczos with the trie-ranked set and term H·v as the operator: the ground
state of state sets cut by further quantum numbers (Sec. IV), of the
momentum-basis ring in each total-momentum sector (Sec. V-C, Eqs. Hk and
Ktot) and of a two-orbital impurity with a Kanamori U_ijkl (Eq. H, built
by the product rule of Fig. mul), against dense diagonalisation by the
oracle.  FP64: E0 within 1e-10 relative; mixed precision with the FP64
Rayleigh-quotient refinement: within 1e-9."""
import numpy as np
import pytest

import gbr_synth as S
import oracle
from gpu_common import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return lib()


def _solve(G, fn, handle, n, iters, prec):
    import torch
    v0 = torch.from_numpy(S.start_vector(n)).cuda()
    return fn(handle, v0, min(iters, n), reorth=True, prec=prec, refine=True)


def _check(E, ref, prec):
    tol = 1e-10 if prec == 0 else 1e-9
    assert abs(E - ref) <= tol * abs(ref), (E, ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_set_lanczos_every_Sz_at_fixed_N(G, prec):
    """All S_z of the 8-site ring at 8 particles (12,870 states): the ground
    state is the lowest over the (N_up, N_dn) sectors."""
    L, N, U = 8, 8, 4.0
    h, Uv = S.chain(L), S.uniform_U(L, U)
    st = S.fixed_N_states(L, N)
    ref = min(oracle.dense_E0(L, h, Uv, a, N - a) for a in range(max(0, N - L), min(N, L) + 1)
              if oracle.sector_dim(L, a, N - a) <= 5000)
    Sh = G.gbr_setham_create(L, h, Uv, st, 8)
    r = _solve(G, G.gbr_setham_lanczos, Sh, st.size, 160, prec)
    _check(r["E0"], ref, prec)
    # the residual of a Ritz vector built from FP32 Lanczos vectors cannot go
    # below about |H| u_32 (|H| = 20.6 here, u_32 = 2^-24: 1.2e-6); FP64 vectors
    # reach the converged Ritz pair's own residual
    assert r["residual"] <= (1e-6 if prec == 0 else 1e-5)


def test_set_lanczos_open_subset_is_the_projected_operator(G):
    """A subset that H does not map into itself: the operator is P H P, whose
    dense form the oracle builds column by column from its set H·v."""
    L = 6
    h, Uv = S.chain(L, pbc=False) + np.diag(np.linspace(-0.4, 0.4, L)), S.uniform_U(L, 3.0)
    full = oracle.fixed_N_states(L, 5)
    rng = np.random.default_rng(11)
    sub = np.sort(rng.choice(full, size=300, replace=False))
    cols = []
    for j in range(sub.size):
        e = np.zeros(sub.size)
        e[j] = 1.0
        cols.append(oracle.hv_set(L, h, Uv, sub, e)[0])
    Hm = np.array(cols).T
    ref = float(np.linalg.eigvalsh(0.5 * (Hm + Hm.T))[0])
    assert np.allclose(Hm, Hm.T, atol=1e-14)
    Sh = G.gbr_setham_create(L, h, Uv, sub, 8)
    for prec in (0, 1):
        _check(_solve(G, G.gbr_setham_lanczos, Sh, sub.size, 300, prec)["E0"], ref, prec)


@pytest.mark.parametrize("L,N", [(6, 3), (8, 4)])
def test_term_lanczos_momentum_ring_every_K(G, L, N):
    """Every total-momentum sector of the momentum-basis ring (Eq. Hk): its
    ground state equals the sector's dense lowest eigenvalue and is a level
    of the real-space ring's dense spectrum; the lowest over K is the ring's
    ground state."""
    U = 4.0
    terms = S.momentum_ring_terms(L, 1.0, U)
    tup = [G.gbr_term_product(o, c) for c, o in terms]
    real = np.linalg.eigvalsh(oracle.dense(L, S.chain(L), S.uniform_U(L, U), N, N))
    best = []
    for K in range(L):
        st = S.momentum_sector_states(L, N, N, K)
        ref = float(np.linalg.eigvalsh(oracle.dense_ops(terms, st))[0])
        assert np.min(np.abs(real - ref)) <= 1e-10 * abs(ref)
        T = G.gbr_termham_create(2 * L, tup, st, 8)
        for prec in (0, 1):
            r = _solve(G, G.gbr_termham_lanczos, T, st.size, 200, prec)
            _check(r["E0"], ref, prec)
            if prec == 0:
                best.append(r["E0"])
    assert abs(min(best) - real[0]) <= 1e-10 * abs(real[0])


@pytest.mark.parametrize("nu,nd", [(3, 3), (2, 3)])
def test_term_lanczos_two_orbital_kanamori_impurity(G, nu, nd):
    """Two-orbital impurity with four bath sites and the Kanamori U_ijkl
    (spin flip and pair hopping included): Lanczos on the term H·v against
    dense diagonalisation of the literal operator products."""
    L, terms = S.two_orbital_impurity_terms(4)
    st = oracle.sector_states(L, nu, nd)
    ref = float(np.linalg.eigvalsh(oracle.dense_ops(terms, st))[0])
    T = G.gbr_termham_create(2 * L, [G.gbr_term_product(o, c) for c, o in terms], st, 8)
    for prec in (0, 1):
        _check(_solve(G, G.gbr_termham_lanczos, T, st.size, 200, prec)["E0"], ref, prec)


def test_set_lanczos_kept_head_and_ritz_tail(G):
    """The operator-generic recurrence (set H·v, no spin factorisation) with a
    kept head of the basis: every head size, with and without a cut Ritz
    tail, gives the energy of the stored-basis solve (the same vectors,
    summed from memory or rebuilt by the second run).  12,870 states: an
    FP32 vector is not a whole number of 16-byte packs, so FP32 keeps no
    head (its slots would not be aligned for the packed Ritz sum) and runs
    the plain second run; FP64 keeps one."""
    import torch
    L, N = 8, 8
    h, Uv = S.chain(L), S.uniform_U(L, 4.0)
    st = S.fixed_N_states(L, N)
    Sh = G.gbr_setham_create(L, h, Uv, st, 8)
    v0 = torch.from_numpy(S.start_vector(st.size)).cuda()
    for prec in (0, 1):
        for tail in (0.0, 1e-6):
            full = G.gbr_setham_lanczos(Sh, v0, 90, prec=prec, refine=True, store_basis=1, ritz_tail=tail)
            sec = G.gbr_setham_lanczos(Sh, v0, 90, prec=prec, refine=True, store_basis=0, ritz_tail=tail)
            for m in (2, 7, 40, 500):
                hd = G.gbr_setham_lanczos(Sh, v0, 90, prec=prec, refine=True, store_basis=-m, ritz_tail=tail)
                es = 8 if prec == 0 else 4
                kept = min(m, hd["ritz_terms"]) if (st.size * es) % 16 == 0 else 0
                assert hd["basis_head"] == kept, (prec, m, hd["basis_head"])
                # the same recurrence as the second-run solve (the head only adds
                # the slot writes); a stored basis whose slots are not 16-byte
                # aligned sums its dots element by element, so its alpha and
                # beta may differ from these in the last bits
                assert np.array_equal(hd["alpha"], sec["alpha"]) and np.array_equal(hd["beta"], sec["beta"]), (prec, m)
                assert hd["ritz_terms"] == sec["ritz_terms"]
                assert abs(hd["E0"] - sec["E0"]) <= 1e-13 * abs(sec["E0"]), (prec, tail, m)
                assert abs(hd["E0"] - full["E0"]) <= 1e-12 * abs(full["E0"]), (prec, tail, m)
