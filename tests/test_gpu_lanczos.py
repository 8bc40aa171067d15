"""Lanczos on the GPU against dense diagonalisation, the oracle's FP64
Lanczos and the non-interacting closed forms.

Bars: FP64 E0 within 1e-10 relative of the reference; mixed precision with
the FP64 Rayleigh-quotient refinement within 1e-9 relative."""
import math

import numpy as np
import pytest

import gbr_synth as S
import oracle
from gpu_common import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return lib()


def ring8(U=4.0):
    return 8, S.chain(8), S.uniform_U(8, U), 4, 4


def v0(D, seed=S.SEED_START):
    import torch
    return torch.from_numpy(S.start_vector(D, seed)).cuda()


def test_ring8_fp64_reorth_matches_dense_and_oracle(G):
    L, h, U, Nu, Nd = ring8()
    H = G.gbr_ham_create(L, h, U, Nu, Nd, G.GBR_RANK_CNS)
    r = G.gbr_lanczos(H, v0(4900), 100, reorth=True, prec=G.GBR_PREC_FP64, refine=True, want_ritz=True)
    E_dense = oracle.dense_E0(L, h, U, Nu, Nd)
    assert r["iters"] == 100
    assert abs(r["E_ritz"] - E_dense) <= 1e-10 * abs(E_dense)
    assert abs(r["E0"] - E_dense) <= 1e-10 * abs(E_dense)
    o = oracle.lanczos(L, h, U, Nu, Nd, S.start_vector(4900), 100, True)
    assert np.max(np.abs(r["alpha"] - o["alpha"])) <= 1e-9
    assert np.max(np.abs(r["beta"] - o["beta"])) <= 1e-9
    assert np.max(np.abs(r["ritz"] - o["ritz"])) <= 1e-9


def test_ring8_mixed_refined_meets_1e9(G):
    L, h, U, Nu, Nd = ring8()
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    E_dense = oracle.dense_E0(L, h, U, Nu, Nd)
    for reorth in (True, False):
        r = G.gbr_lanczos(H, v0(4900), 100, reorth=reorth, prec=G.GBR_PREC_MIXED, refine=True)
        assert abs(r["E0"] - E_dense) <= 1e-9 * abs(E_dense), (reorth, r["E0"], E_dense)
        assert r["residual"] < 1e-3


def test_graph_replay_and_second_pass_are_bit_identical(G):
    L, h, U, Nu, Nd = ring8()
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    for prec in (G.GBR_PREC_FP64, G.GBR_PREC_MIXED):
        a = G.gbr_lanczos(H, v0(4900), 60, prec=prec, refine=True, store_basis=1, use_graph=False)
        b = G.gbr_lanczos(H, v0(4900), 60, prec=prec, refine=True, store_basis=0, use_graph=True)
        assert np.array_equal(a["alpha"], b["alpha"]) and np.array_equal(a["beta"], b["beta"])
        assert a["stored_basis"] and not b["stored_basis"]
        assert abs(a["E0"] - b["E0"]) <= 1e-13 * abs(a["E0"])


def test_second_run_finishes_each_step_in_the_spin_up_pass(G):
    """Without a stored basis the Ritz vector comes from a second run of the
    recurrence with the stored scalars.  When the per-spin dimensions are
    whole 16-byte packs, the spin-up pass of that run finishes each step
    itself (u_{k+1} row-major and transposed for the next H·v): one launch
    fewer per step than the separate update, which the windowed passes keep.
    Both rebuild the first run's vectors, so E0 and the residual agree with
    the stored-basis solve, and eager and graph launches agree bit for bit."""
    # 4x3 torus with diagonal hopping, N_up = 5, N_dn = 6: 792 x 924 states,
    # both multiples of 4; the 924 columns end in a ragged column chunk, and
    # 16 rows per CTA in a ragged row block (792 = 49.5 x 16)
    L, h, U, Nu, Nd = 12, S.square(4, 3, 1.0, -0.3), S.uniform_U(12, 8.0), 5, 6
    D = oracle.sector_dim(L, Nu, Nd)
    assert D == 792 * 924
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
    for prec, fp in ((G.GBR_PREC_FP64, 64), (G.GBR_PREC_MIXED, 32)):
        for rows_lz in (4, 16):
            G.gbr_ham_set_shape(H, fp, 0, 8, 8, rows_lz)
            a = G.gbr_lanczos(H, v0(D), 60, prec=prec, refine=True, store_basis=1)
            n0 = G.gbr_launch_count()
            b = G.gbr_lanczos(H, v0(D), 60, prec=prec, refine=True, store_basis=0, use_graph=False)
            nb = G.gbr_launch_count() - n0
            c = G.gbr_lanczos(H, v0(D), 60, prec=prec, refine=True, store_basis=0, use_graph=True)
            assert a["stored_basis"] and not b["stored_basis"] and b["ritz_terms"] <= 60
            assert np.array_equal(a["alpha"], b["alpha"]) and np.array_equal(a["beta"], b["beta"])
            assert np.array_equal(b["alpha"], c["alpha"]) and np.array_equal(b["beta"], c["beta"])
            assert b["E0"] == c["E0"] and b["residual"] == c["residual"], (prec, rows_lz)
            assert abs(a["E0"] - b["E0"]) <= 1e-13 * abs(a["E0"]), (prec, rows_lz)
            # the two Ritz vectors differ only by the rounding of their sums
            assert abs(a["residual"] - b["residual"]) <= 1e-6 * a["residual"], (prec, rows_lz)
        G.gbr_ham_set_shape(H, fp, 1, 32, 32, 32)
        assert G.gbr_ham_get_shape(H, fp)["window"] == 1
        n0 = G.gbr_launch_count()
        w = G.gbr_lanczos(H, v0(D), 60, prec=prec, refine=True, store_basis=0, use_graph=False)
        nw = G.gbr_launch_count() - n0
        assert w["ritz_terms"] == b["ritz_terms"]
        assert nw - nb == w["ritz_terms"] - 1, (prec, nw, nb)
        assert abs(w["E0"] - a["E0"]) <= 1e-12 * abs(a["E0"])
        G.gbr_ham_set_shape(H, fp, 0)
    assert G.gbr_device_status() == 0


def test_free_fermion_closed_form_ring8(G):
    L, h, U, Nu, Nd = ring8(U=0.0)
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    r = G.gbr_lanczos(H, v0(4900), 100, prec=G.GBR_PREC_MIXED, refine=True)
    E = -4.0 - 4.0 * math.sqrt(2.0)
    assert abs(r["E0"] - E) <= 1e-9 * abs(E)


def test_breakdown_on_exhausted_sector(G):
    h = S.chain(3, pbc=False)
    H = G.gbr_ham_create(3, h, S.uniform_U(3, 1.0), 1, 0)
    r = G.gbr_lanczos(H, v0(3), 10, prec=G.GBR_PREC_FP64, refine=True)
    assert r["iters"] <= 3
    assert abs(r["E0"] - np.linalg.eigvalsh(oracle.dense(3, h, S.uniform_U(3, 1.0), 1, 0))[0]) < 1e-12


def test_single_impurity_sector(G):
    h, U = S.siam(7)
    L = h.shape[0]
    Nu, Nd = L // 2, L // 2
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    D, _ = G.gbr_ham_info(H)
    E_dense = oracle.dense_E0(L, h, U, Nu, Nd)
    r = G.gbr_lanczos(H, v0(D), min(150, D), prec=G.GBR_PREC_MIXED, refine=True)
    assert abs(r["E0"] - E_dense) <= 1e-9 * abs(E_dense)


def test_hubbard_4x4_mixed_vs_fp64_and_free_limit(G):
    """The 4x4 t' Hubbard sector (1.31e8 states): mixed precision with FP64
    refinement agrees with the all-FP64 GPU path to 1e-9; at U = 0 it meets
    the closed form -26.4."""
    import gbr_synth.gpu as SG
    L = 16
    h = S.square(4, 4, 1.0, -0.3)
    H = G.gbr_ham_create(L, h, S.uniform_U(L, 8.0), 7, 7)
    D, _ = G.gbr_ham_info(H)
    s = SG.uniform(S.SEED_START, D)
    rm = G.gbr_lanczos(H, s, 200, prec=G.GBR_PREC_MIXED, refine=True, store_basis=1)
    rd = G.gbr_lanczos(H, s, 200, prec=G.GBR_PREC_FP64, refine=False, store_basis=0)
    assert abs(rm["E0"] - rd["E0"]) <= 1e-9 * abs(rd["E0"]), (rm["E0"], rd["E0"])
    H0 = G.gbr_ham_create(L, h, S.uniform_U(L, 0.0), 7, 7)
    r0 = G.gbr_lanczos(H0, s, 200, prec=G.GBR_PREC_MIXED, refine=True, store_basis=1)
    E_free = oracle.free_E0(h, 7, 7)
    assert abs(E_free - (-26.4)) < 1e-12
    assert abs(r0["E0"] - E_free) <= 1e-9 * abs(E_free), r0["E0"]


def test_tolerance_stop_meets_the_bar_earlier(G):
    """With tol the recurrence stops once the lowest Ritz pair has converged;
    the refined mixed-precision energy still meets 1e-9."""
    L, h, U, Nu, Nd = ring8()
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    E_dense = oracle.dense_E0(L, h, U, Nu, Nd)
    r = G.gbr_lanczos(H, v0(4900), 300, prec=G.GBR_PREC_MIXED, refine=True, tol=1e-6)
    assert r["converged"] and r["iters"] < 300 and r["iters"] % 8 == 0
    assert abs(r["E0"] - E_dense) <= 1e-9 * abs(E_dense)
    r64 = G.gbr_lanczos(H, v0(4900), 300, prec=G.GBR_PREC_FP64, refine=False, tol=1e-6)
    assert r64["converged"] and abs(r64["E0"] - E_dense) <= 1e-9 * abs(E_dense)


def test_factored_path_fused_update_matches_oracle_and_is_reproducible(G):
    """The factored H·v carries the first Lanczos update in its epilogue; on a
    10-site ring (63,504 states) the FP64 run matches the oracle's Lanczos,
    graph replay equals eager launches bit for bit, and the second pass that
    rebuilds the Ritz vector reproduces the first."""
    L = 10
    h, U = S.chain(L), S.uniform_U(L, 4.0)
    H = G.gbr_ham_create(L, h, U, 5, 5)
    G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
    D, _ = G.gbr_ham_info(H)
    o = oracle.lanczos(L, h, U, 5, 5, S.start_vector(D), 60, False)
    r = G.gbr_lanczos(H, v0(D), 60, prec=G.GBR_PREC_FP64, refine=True, store_basis=1)
    # without re-orthogonalisation rounding differences grow once Ritz values
    # converge, so the recurrences are compared over their first 30 steps
    assert np.max(np.abs(r["alpha"][:30] - o["alpha"][:30])) <= 1e-9
    assert np.max(np.abs(r["beta"][:29] - o["beta"][:29])) <= 1e-9
    assert abs(r["E_ritz"] - o["E0"]) <= 1e-10 * abs(o["E0"])
    for prec in (G.GBR_PREC_FP64, G.GBR_PREC_MIXED):
        a = G.gbr_lanczos(H, v0(D), 50, prec=prec, refine=True, store_basis=1, use_graph=False)
        b = G.gbr_lanczos(H, v0(D), 50, prec=prec, refine=True, store_basis=0, use_graph=True)
        assert np.array_equal(a["alpha"], b["alpha"]) and np.array_equal(a["beta"], b["beta"])
        assert abs(a["E0"] - b["E0"]) <= 1e-13 * abs(a["E0"])


def test_kept_head_of_the_basis(G):
    """When the whole basis does not fit, the first run keeps its leading
    vectors (store_basis = -m asks for m of them; -1 keeps as many as fit):
    the Ritz sum takes those from memory and the second run of the
    recurrence starts after them, with fewer launches.  Energy and residual
    match the stored-basis solve, and the recurrence is the same."""
    L, h, U, Nu, Nd = 12, S.square(4, 3, 1.0, -0.3), S.uniform_U(12, 8.0), 5, 6
    D = oracle.sector_dim(L, Nu, Nd)
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
    for prec in (G.GBR_PREC_FP64, G.GBR_PREC_MIXED):
        full = G.gbr_lanczos(H, v0(D), 60, prec=prec, refine=True, store_basis=1)
        n0 = G.gbr_launch_count()
        sec = G.gbr_lanczos(H, v0(D), 60, prec=prec, refine=True, store_basis=0, use_graph=True)
        n_sec = G.gbr_launch_count() - n0
        assert sec["basis_head"] == 0
        # head sizes that leave each remainder of the groups of three
        for m in (2, 10, 11, 12, 1000):
            n0 = G.gbr_launch_count()
            hd = G.gbr_lanczos(H, v0(D), 60, prec=prec, refine=True, store_basis=-m, use_graph=True)
            n_hd = G.gbr_launch_count() - n0
            assert not hd["stored_basis"] and hd["ritz_terms"] == sec["ritz_terms"]
            assert hd["basis_head"] == min(m, hd["ritz_terms"]), (prec, m)
            assert np.array_equal(hd["alpha"], sec["alpha"]) and np.array_equal(hd["beta"], sec["beta"])
            assert abs(hd["E0"] - full["E0"]) <= 1e-13 * abs(full["E0"]), (prec, m)
            assert abs(hd["residual"] - full["residual"]) <= 1e-6 * full["residual"], (prec, m)
            if m >= 10:
                assert n_hd < n_sec, (prec, m, n_hd, n_sec)


def test_ritz_vector_of_the_converged_prefix(G):
    """A run far past convergence (300 steps on 4,900 states, no
    re-orthogonalisation) forms its Ritz vector from the shortest prefix whose
    lowest pair has converged to the vectors' roundoff, before the recurrence
    grows copies of that state: the same energy and residual, bit for bit, as
    a run stopped at that prefix, and the refined energy close to dense
    diagonalisation."""
    L, h, U, Nu, Nd = ring8()
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    E_dense = oracle.dense_E0(L, h, U, Nu, Nd)
    for prec, bar in ((G.GBR_PREC_MIXED, 1e-11), (G.GBR_PREC_FP64, 1e-13)):
        run = G.gbr_lanczos(H, v0(4900), 300, prec=prec, refine=True, store_basis=1)
        assert run["iters"] == 300
        assert abs(run["E0"] - E_dense) <= bar * abs(E_dense), (prec, run["E0"], E_dense)
        k = run["ritz_terms"]
        assert 8 <= k <= 300
        if prec == G.GBR_PREC_MIXED:
            assert k % 8 == 0 and k < 300
        if k < 300:
            short = G.gbr_lanczos(H, v0(4900), k, prec=prec, refine=True, store_basis=1)
            assert short["ritz_terms"] == k
            assert short["E0"] == run["E0"] and short["residual"] == run["residual"], prec


def test_ritz_tail_cut_keeps_the_bar_and_matches_between_basis_modes(G):
    """Dropping the trailing Ritz coefficients (norm <= ritz_tail) moves the
    refined energy by about ritz_tail^2 times the spectral spread: at 1e-6
    the mixed E0 still meets 1e-9 against dense diagonalisation, stays above
    it (a Rayleigh quotient), uses fewer terms than steps once converged, and
    the stored-basis and recomputed-basis sums agree."""
    import torch
    L, h, U, Nu, Nd = ring8()
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    E_dense = oracle.dense_E0(L, h, U, Nu, Nd)
    a = G.gbr_lanczos(H, v0(4900), 120, prec=G.GBR_PREC_MIXED, refine=True, store_basis=1, ritz_tail=1e-6)
    b = G.gbr_lanczos(H, v0(4900), 120, prec=G.GBR_PREC_MIXED, refine=True, store_basis=0, ritz_tail=1e-6)
    full = G.gbr_lanczos(H, v0(4900), 120, prec=G.GBR_PREC_MIXED, refine=True, store_basis=1)
    assert full["ritz_terms"] <= full["iters"]
    assert a["ritz_terms"] == b["ritz_terms"] <= full["ritz_terms"]
    for r in (a, b):
        assert abs(r["E0"] - E_dense) <= 1e-9 * abs(E_dense)
        assert r["E0"] >= E_dense - 1e-12 * abs(E_dense)
    assert abs(a["E0"] - b["E0"]) <= 1e-12 * abs(E_dense)
    with pytest.raises(G.GbrError):
        G.gbr_lanczos(H, v0(4900), 10, ritz_tail=-1.0)


def test_newton_reciprocal_of_the_eigensolvers_is_within_two_ulp(G):
    """The tridiagonal eigensolvers divide through a Newton-Raphson reciprocal
    seeded in single precision; against the IEEE division it stays within
    two units in the last place over 1e-29..1e29."""
    assert G.gbr_check_rcp64(1 << 22) <= 2 * 2.0 ** -52


def test_basis_cache_is_reused_and_released(G):
    """A stored-basis solve leaves its basis in the library's cache; a second
    solve on a new handle reuses it with the same result, and after
    gbr_release_cache a third still solves (allocating afresh)."""
    L, h, U, Nu, Nd = ring8()
    E = []
    for _ in range(2):
        H = G.gbr_ham_create(L, h, U, Nu, Nd)
        E.append(G.gbr_lanczos(H, v0(4900), 80, prec=G.GBR_PREC_MIXED, refine=True, store_basis=1)["E0"])
        H.close()
    G.gbr_release_cache()
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    E.append(G.gbr_lanczos(H, v0(4900), 80, prec=G.GBR_PREC_MIXED, refine=True, store_basis=1)["E0"])
    G.gbr_release_cache()
    assert E[0] == E[1] == E[2]


def _golden():
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "reference_energies.json")))


def test_square4x4_U8_reduced_filling_against_oracle_lanczos(G):
    """The 4x4 t' torus at U = 8 (the workload's geometry and couplings) at
    N_up = N_dn = 3 (313,600 states), where the oracle's FP64 Lanczos is in
    reach: FP64 within 1e-10, mixed with refinement within 1e-9."""
    import torch
    g = _golden()
    ref = g["square4x4_tp_U8_N3_3_lanczos_E0"]
    assert g["square4x4_tp_U8_N3_3_lanczos_change_last_50_steps"] <= 1e-12 * abs(ref)
    H = G.gbr_ham_create(16, S.square(4, 4, 1.0, -0.3), S.uniform_U(16, 8.0), 3, 3)
    D, _ = G.gbr_ham_info(H)
    x = v0(D)
    r64 = G.gbr_lanczos(H, x, 200, prec=G.GBR_PREC_FP64, refine=True)
    assert abs(r64["E0"] - ref) <= 1e-10 * abs(ref), (r64["E0"], ref)
    rm = G.gbr_lanczos(H, x, 200, prec=G.GBR_PREC_MIXED, refine=True)
    assert abs(rm["E0"] - ref) <= 1e-9 * abs(ref), (rm["E0"], ref)
    del x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("U", [0.0, 4.0])
def test_ring18_full_size_against_closed_form_and_bethe_ansatz(G, U):
    """The 18-site ring at full size (2.36e9 states), 150 mixed-precision
    steps with the Ritz vector recomputed and the FP64 refinement, as the
    benchmark runs it: U = 0 against the sum of the lowest one-body levels,
    U = 4 against the Lieb-Wu Bethe-ansatz energy."""
    import torch
    import gbr_synth.gpu as SG
    g = _golden()
    ref = g["chain18_U0_N9_9_free_E0"] if U == 0.0 else g["chain18_U4_N9_9_bethe_E0"]
    H = G.gbr_ham_create(18, S.chain(18), S.uniform_U(18, U), 9, 9)
    D, _ = G.gbr_ham_info(H)
    s = SG.uniform(S.SEED_START, D)
    r = G.gbr_lanczos(H, s, 150, prec=G.GBR_PREC_MIXED, refine=True, store_basis=0, use_graph=True)
    assert abs(r["E0"] - ref) <= 1e-9 * abs(ref), (r["E0"], ref)
    assert not r["stored_basis"]
    H.close()
    del s
    G.gbr_release_cache()
    torch.cuda.empty_cache()
