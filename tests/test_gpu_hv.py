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
