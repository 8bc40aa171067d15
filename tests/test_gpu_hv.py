"""Parity of the GPU H·v (both paths, both precisions, both rankings) with
the oracle's literal operator application.

Tolerances: FP64, max|y - y_ref| / max|y_ref| <= 1e-12 (the stated bar);
FP32, <= 1e-5 (each element sums at most ~70 terms of FP32 products with
unit-size coefficients: error ~ 70 * 2^-24 |x| ~ 4e-6 of the largest term).
"""
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


def model(kind):
    if kind == "ring8":
        return 8, S.chain(8), S.uniform_U(8, 4.0), 4, 4
    if kind == "ring6_unequal":
        return 6, S.chain(6), S.uniform_U(6, 2.5), 2, 4
    if kind == "ring10":
        return 10, S.chain(10), S.uniform_U(10, 4.0), 5, 5
    if kind == "sq3x3":
        h = S.square(3, 3, 1.0, -0.3)
        return 9, h, S.uniform_U(9, 8.0), 4, 3
    if kind == "sq4x4_dilute":
        h = S.square(4, 4, 1.0, -0.3)
        return 16, h, S.uniform_U(16, 8.0), 2, 3
    if kind == "siam":
        h, U = S.siam(3)
        L = h.shape[0]
        return L, h, U, L // 2, L // 2 + 1
    if kind == "nonuniformU":
        h = S.chain(7, pbc=False) + np.diag(np.linspace(-1, 1, 7))
        return 7, h, np.array([0.0, 1.0, 2.0, 1.0, 0.0, 3.0, 1.5]), 3, 3
    if kind == "one_site":
        return 1, np.array([[0.7]]), np.array([3.0]), 1, 1
    if kind == "empty_spin":
        return 6, S.chain(6), S.uniform_U(6, 4.0), 0, 3
    if kind == "full_spin":
        return 6, S.chain(6), S.uniform_U(6, 4.0), 6, 2
    raise KeyError(kind)


KINDS = ["ring8", "ring6_unequal", "ring10", "sq3x3", "sq4x4_dilute", "siam", "nonuniformU", "one_site",
         "empty_spin", "full_spin"]


@pytest.mark.parametrize("kind", KINDS)
def test_hv_small_sectors_all_paths(G, kind):
    import torch
    L, h, U, Nu, Nd = model(kind)
    x = S.start_vector(oracle.sector_dim(L, Nu, Nd))
    y_ref = oracle.hv(L, h, U, Nu, Nd, x)
    for method in (G.GBR_RANK_STAGGERED, G.GBR_RANK_CNS):
        H = G.gbr_ham_create(L, h, U, Nu, Nd, method)
        D, elems = G.gbr_ham_info(H)
        assert D == x.size
        assert elems == oracle.count_elements(L, h, Nu, Nd)
        for path in (G.GBR_HV_FUSED, G.GBR_HV_FACTORED):
            G.gbr_ham_set_path(H, path)
            x64 = torch.from_numpy(x).cuda()
            y64 = torch.full_like(x64, float("nan"))
            G.gbr_hv(H, x64, y64)
            assert rel_inf(y64.cpu().numpy(), y_ref) <= TOL64, (kind, method, path)
            x32 = x64.float()
            y32 = torch.full_like(x32, float("nan"))
            G.gbr_hv(H, x32, y32)
            y_ref32 = oracle.hv(L, h, U, Nu, Nd, x32.double().cpu().numpy())
            assert rel_inf(y32.cpu().numpy(), y_ref32) <= TOL32, (kind, method, path)


def test_hv_tuned_shapes_keep_parity(G):
    import torch
    L, h, U, Nu, Nd = model("ring10")
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    x = S.start_vector(oracle.sector_dim(L, Nu, Nd))
    y_ref = oracle.hv(L, h, U, Nu, Nd, x)
    assert G.gbr_ham_get_path(H) == G.GBR_HV_AUTO
    for fp in (32, 64):
        G.gbr_ham_tune(H, fp)
    assert G.gbr_ham_get_path(H) in (G.GBR_HV_FUSED, G.GBR_HV_FACTORED)
    x64 = torch.from_numpy(x).cuda()
    y64 = torch.empty_like(x64)
    G.gbr_hv(H, x64, y64)
    assert rel_inf(y64.cpu().numpy(), y_ref) <= TOL64
    # the tuned tile of the spin-up pass with the fused Lanczos update
    G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
    o = oracle.lanczos(L, h, U, Nu, Nd, x, 40, False)
    r = G.gbr_lanczos(H, x64, 40, prec=G.GBR_PREC_FP64, refine=False)
    assert np.max(np.abs(r["alpha"][:20] - o["alpha"][:20])) <= 1e-9
    assert abs(r["E_ritz"] - o["E0"]) <= 1e-10 * abs(o["E0"])


def test_hv_rejects_overlap_and_bad_dtype(G):
    import torch
    L, h, U, Nu, Nd = model("ring8")
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    x = torch.zeros(4900 * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GbrError):
        G.gbr_hv(H, x[:4900], x[100:5000])
    with pytest.raises(ValueError):
        G.gbr_hv(H, x[:4900].half(), x[4900:].half())


FULL = {
    "hubbard_4x4_tp": (16, lambda: S.square(4, 4, 1.0, -0.3), 8.0, 7, 7),
    "hubbard_chain_L18": (18, lambda: S.chain(18), 4.0, 9, 9),
}


@pytest.mark.parametrize("name", list(FULL))
@pytest.mark.parametrize("fp", [32, 64])
def test_hv_full_size_sampled_rows(G, name, fp):
    """Full-size sectors in the benchmark's launch configuration (factored
    path): sampled rows against the oracle, which reads x_j from the seeded
    generator on demand."""
    import torch
    import gbr_synth.gpu as SG
    L, hf, Uv, Nu, Nd = FULL[name]
    h, U = hf(), S.uniform_U(L, Uv)
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    D, _ = G.gbr_ham_info(H)
    x = SG.uniform(S.SEED_START, D)
    if fp == 32:
        x = x.float()
    y = torch.empty_like(x)
    G.gbr_hv(H, x, y)
    torch.cuda.synchronize()
    rows = np.unique(np.concatenate([[0, 1, D - 1, D - 2], S.bounded(21, np.arange(300, dtype=np.uint64), D)])).astype(np.int64)
    y_ref = oracle.hv_rows_seeded(L, h, U, Nu, Nd, S.SEED_START, rows)
    got = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    tol = TOL64 if fp == 64 else TOL32
    assert rel_inf(got, y_ref) <= tol, rel_inf(got, y_ref)
    del x, y
    torch.cuda.empty_cache()


def test_hv_full_size_hermitian_and_fused_agree(G):
    """<u, H v> = <H u, v> at full size (FP64), and the factored path agrees
    with the fused per-element path on the 4x4 sector."""
    import torch
    import gbr_synth.gpu as SG
    L, hf, Uv, Nu, Nd = FULL["hubbard_4x4_tp"]
    H = G.gbr_ham_create(L, hf(), S.uniform_U(L, Uv), Nu, Nd)
    D, _ = G.gbr_ham_info(H)
    u = SG.uniform(31, D)
    v = SG.uniform(32, D)
    Hu, Hv = torch.empty_like(u), torch.empty_like(v)
    G.gbr_hv(H, u, Hu)
    G.gbr_hv(H, v, Hv)
    a, b = torch.dot(u, Hv).item(), torch.dot(Hu, v).item()
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0) * 100
    G.gbr_ham_set_path(H, G.GBR_HV_FUSED)
    Hv2 = torch.empty_like(v)
    G.gbr_hv(H, v, Hv2)
    assert (Hv2 - Hv).abs().max().item() <= TOL64 * Hv.abs().max().item()


# Sectors whose per-spin dimensions are multiples of 4, so that both gather
# families run (the windowed one needs rows of whole 16-byte packs); each is
# ragged against the 32- and 64-row tiles and the 512-byte column slices.
WIN_KINDS = {
    "ring12": lambda: (12, S.chain(12), S.uniform_U(12, 4.0), 6, 6),                 # 924 x 924
    "ring12_unequal": lambda: (12, S.chain(12), S.uniform_U(12, 4.0), 5, 6),         # 792 x 924
    "sq4x4_N3": lambda: (16, S.square(4, 4, 1.0, -0.3), S.uniform_U(16, 8.0), 3, 3),  # 560 x 560
    "siam_bath7": lambda: (lambda h, U: (h.shape[0], h, U, 3, 3))(*S.siam(4)),            # 56 x 56, non-uniform hops
}


def _hv(G, H, x):
    import torch
    y = torch.full_like(x, float("nan"))
    G.gbr_hv(H, x, y)
    return y


@pytest.mark.parametrize("kind", list(WIN_KINDS))
@pytest.mark.parametrize("fp", [32, 64])
def test_windowed_gathers_equal_plain_gathers_and_oracle(G, kind, fp):
    """Every element sums its hops in the same order in both gather families
    and under every tile and CTA width, so every shape gives the plain H·v
    bit for bit; it matches the oracle."""
    import torch
    L, h, U, Nu, Nd = WIN_KINDS[kind]()
    D = oracle.sector_dim(L, Nu, Nd)
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
    x = torch.from_numpy(S.start_vector(D)).cuda()
    if fp == 32:
        x = x.float()
    G.gbr_ham_set_shape(H, fp, 0)
    assert G.gbr_ham_get_shape(H, fp)["window"] == 0
    y_plain = _hv(G, H, x)
    y_ref = oracle.hv(L, h, U, Nu, Nd, x.double().cpu().numpy())
    assert rel_inf(y_plain.cpu().numpy(), y_ref) <= (TOL64 if fp == 64 else TOL32)
    for nt in (64, 128):
        for rows in ((4, 16, 8), (16, 4, 4)):
            G.gbr_ham_set_shape(H, fp, 0, *rows, threads_dn=nt, threads_up=nt, threads_lz=nt)
            assert G.gbr_ham_get_shape(H, fp)["threads_up"] == nt
            assert torch.equal(_hv(G, H, x), y_plain), (kind, fp, nt, rows)
    for rows in ((32, 32, 32), (64, 64, 64), (64, 32, 64)):
        G.gbr_ham_set_shape(H, fp, 1, *rows)
        sh = G.gbr_ham_get_shape(H, fp)
        if D % 4 == 0 and oracle.sector_dim(L, Nu, 0) % 4 == 0 and oracle.sector_dim(L, 0, Nd) % 4 == 0:
            assert sh["window"] == 1 and (sh["rows_dn"], sh["rows_up"]) == rows[:2]
        y_win = _hv(G, H, x)
        assert torch.equal(y_win, y_plain), (kind, fp, rows)
    assert G.gbr_device_status() == 0


@pytest.mark.parametrize("fp", [32, 64])
def test_windowed_gathers_stages_and_unaligned_vectors(G, fp):
    """Stage-by-stage calls equal gbr_hv with the windowed family; vectors
    off a 16-byte boundary make the combine pass fall back to the plain
    kernel reading the row-major spin-down product, with identical results."""
    import torch
    L, h, U, Nu, Nd = WIN_KINDS["ring12"]()
    D = oracle.sector_dim(L, Nu, Nd)
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
    G.gbr_ham_set_shape(H, fp, 1, 64, 64, 64)
    dt = torch.float64 if fp == 64 else torch.float32
    x = torch.from_numpy(S.start_vector(D)).cuda().to(dt)
    y = _hv(G, H, x)
    ys = torch.full_like(x, float("nan"))
    for stage in (1, 2, 3, 4):
        G.gbr_hv_stage(H, x, ys, stage)
    assert torch.equal(ys, y)
    xb = torch.zeros(D + 1, dtype=dt, device="cuda")
    yb = torch.full((D + 1,), float("nan"), dtype=dt, device="cuda")
    xb[1:] = x
    G.gbr_hv(H, xb[1:], yb[1:])
    assert torch.equal(yb[1:], y)


@pytest.mark.parametrize("kind", ["ring10", "sq3x3", "siam", "nonuniformU", "one_site", "empty_spin"])
def test_chunk_width_and_threads_per_state_keep_parity(G, kind):
    """Every chunk width of the staggered tables (R = 8, 4) and every number
    of threads per state of the fused kernel (1, 2, 4) against the oracle;
    in the factored path R changes nothing (the ranks are the same)."""
    import torch
    L, h, U, Nu, Nd = model(kind)
    x64 = torch.from_numpy(S.start_vector(oracle.sector_dim(L, Nu, Nd))).cuda()
    y_ref = oracle.hv(L, h, U, Nu, Nd, x64.cpu().numpy())
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
    G.gbr_ham_set_shape(H, 64, 0, chunk_bits=8)
    y8 = _hv(G, H, x64)
    G.gbr_ham_set_shape(H, 64, 0, chunk_bits=4)
    assert G.gbr_ham_get_shape(H, 64)["chunk_bits"] == 4
    assert torch.equal(_hv(G, H, x64), y8)
    G.gbr_ham_set_path(H, G.GBR_HV_FUSED)
    for fp, x, tol in ((64, x64, TOL64), (32, x64.float(), TOL32)):
        yr = y_ref if fp == 64 else oracle.hv(L, h, U, Nu, Nd, x.double().cpu().numpy())
        for R in (8, 4):
            for tps in (1, 2, 4):
                G.gbr_ham_set_shape(H, fp, 0, chunk_bits=R, threads_per_state=tps)
                sh = G.gbr_ham_get_shape(H, fp)
                assert (sh["chunk_bits"], sh["threads_per_state"]) == (R, tps)
                assert rel_inf(_hv(G, H, x).double().cpu().numpy(), yr) <= tol, (kind, fp, R, tps)


@pytest.mark.parametrize("fp", [32, 64])
def test_quarter_filled_open_chain_sampled_rows(G, fp):
    """The quarter-filled open chain of Eq. Hring (L = 16, N_up = N_dn = 4,
    3.3 million states; the low-filling regime of Sec. V-B): sampled rows of
    both paths and both chunk widths against the oracle, which reads x_j from
    the seeded generator on demand."""
    import torch
    import gbr_synth.gpu as SG
    L, N = 16, 4
    h, U = S.chain(L, pbc=False), S.uniform_U(L, 4.0)
    H = G.gbr_ham_create(L, h, U, N, N)
    D, _ = G.gbr_ham_info(H)
    x = SG.uniform(S.SEED_START, D)
    if fp == 32:
        x = x.float()
    rows = np.unique(np.concatenate([[0, 1, D - 1], S.bounded(23, np.arange(400, dtype=np.uint64), D)])).astype(np.int64)
    y_ref = oracle.hv_rows_seeded(L, h, U, N, N, S.SEED_START, rows)
    idx = torch.from_numpy(rows).cuda()
    tol = TOL64 if fp == 64 else TOL32
    for path in (G.GBR_HV_FUSED, G.GBR_HV_FACTORED):
        G.gbr_ham_set_path(H, path)
        for R in (8, 4):
            G.gbr_ham_set_shape(H, fp, 0, chunk_bits=R)
            y = torch.empty_like(x)
            G.gbr_hv(H, x, y)
            assert rel_inf(y[idx].double().cpu().numpy(), y_ref) <= tol, (path, R)
