"""Failure detection that needs no GPU fault: a non-finite value in the
input propagates through the H·v exactly where the operator couples it and
stops the Lanczos recurrence with an error; a trie table that does not
belong to its member list is caught by the rank's membership check; the
device status word of the bounded waits stays clear."""
import numpy as np
import pytest

import gbr_synth as S
import oracle
from gpu_common import lib, to_dev_u64, as_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return lib()


@pytest.mark.parametrize("path", ["fused", "factored"])
@pytest.mark.parametrize("fp", [32, 64])
def test_nan_in_x_propagates_to_the_coupled_rows_only(G, path, fp):
    import torch
    L, Nu, Nd = 12, 6, 6                       # 924 x 924: both gather families possible
    h, U = S.chain(L), S.uniform_U(L, 4.0)
    D = oracle.sector_dim(L, Nu, Nd)
    x = S.start_vector(D)
    j = 123457
    x[j] = np.nan
    y_ref = oracle.hv(L, h, U, Nu, Nd, x)      # literal operator application, NaN included
    H = G.gbr_ham_create(L, h, U, Nu, Nd)
    G.gbr_ham_set_path(H, G.GBR_HV_FUSED if path == "fused" else G.GBR_HV_FACTORED)
    xd = torch.from_numpy(x).cuda()
    if fp == 32:
        xd = xd.float()
    for window in ((0, 1) if path == "factored" else (0,)):
        G.gbr_ham_set_shape(H, fp, window)
        y = torch.zeros_like(xd)
        G.gbr_hv(H, xd, y)
        yh = y.double().cpu().numpy()
        assert np.array_equal(np.isnan(yh), np.isnan(y_ref)), (path, fp, window)
        assert 1 < np.isnan(y_ref).sum() < 100
        ok = ~np.isnan(y_ref)
        tol = 1e-12 if fp == 64 else 1e-5
        assert np.max(np.abs(yh[ok] - y_ref[ok])) <= tol * np.max(np.abs(y_ref[ok]))


@pytest.mark.parametrize("prec", [0, 1])
def test_nan_start_vector_stops_lanczos_with_an_error(G, prec):
    import torch
    L, h, U = 8, S.chain(8), S.uniform_U(8, 4.0)
    H = G.gbr_ham_create(L, h, U, 4, 4)
    v = S.start_vector(4900)
    v[17] = np.nan
    with pytest.raises(G.GbrError) as e:
        G.gbr_lanczos(H, torch.from_numpy(v).cuda(), 50, prec=prec, refine=True)
    assert e.value.code == G.GBR_ENONFINITE
    # the handle stays usable
    r = G.gbr_lanczos(H, torch.from_numpy(S.start_vector(4900)).cuda(), 80, prec=prec, refine=True)
    assert abs(r["E0"] - oracle.dense_E0(L, h, U, 4, 4)) <= 1e-9 * 5


def test_corrupted_trie_table_is_caught_by_the_membership_check(G):
    import torch
    M, R = 20, 8
    members = np.unique(S.u64(9, np.arange(3000, dtype=np.uint64)) & np.uint64((1 << M) - 1))
    n = members.size
    size, table = G.gbr_trie_build_host(members, M, R)
    q = to_dev_u64(members)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    # the stored table as given: the same ranks as a trie built from the members
    t_ok = G.gbr_trie_create_from_table(members, M, R, table)
    G.gbr_trie_rank(t_ok, q, out, check=1)
    assert np.array_equal(as_u32(out), np.arange(n, dtype=np.uint32))
    # every entry holding the value n - 1 (the last member's leaf among them)
    # now holds 0: the check turns every misrouted query into NOT_FOUND
    bad = table.copy()
    hit = bad[:size] == n - 1
    assert hit.any()
    bad[:size][hit] = 0
    t_bad = G.gbr_trie_create_from_table(members, M, R, bad)
    G.gbr_trie_rank(t_bad, q, out, check=1)
    r = as_u32(out)
    assert r[n - 1] == G.NOT_FOUND_U32
    assert np.all((r == np.arange(n, dtype=np.uint32)) | (r == G.NOT_FOUND_U32))
    G.gbr_trie_rank(t_bad, q, out, check=0)
    assert as_u32(out)[n - 1] != n - 1           # without the check the error is silent
    with pytest.raises(G.GbrError):
        G.gbr_trie_create_from_table(members, M, R, table[:-1])
    assert G.gbr_device_status() == 0


def test_stage_calls_refuse_to_run_before_their_inputs_exist(G):
    """The gather stages of gbr_hv_stage read the hop lists (stage 1) and
    the scratch stage 2 allocates: on a fresh handle they return EINVAL
    instead of reading uninitialised lists; in order they equal gbr_hv."""
    import torch
    L, h, U = 10, S.chain(10), S.uniform_U(10, 4.0)
    H = G.gbr_ham_create(L, h, U, 5, 5)
    D, _ = G.gbr_ham_info(H)
    x = torch.from_numpy(S.start_vector(D)).cuda()
    y = torch.empty_like(x)
    for stage in (3, 4):
        with pytest.raises(G.GbrError) as e:
            G.gbr_hv_stage(H, x, y, stage)
        assert e.value.code == G.GBR_EINVAL and "stage 1" in str(e.value)
    G.gbr_hv_stage(H, x, y, 1)
    with pytest.raises(G.GbrError) as e:
        G.gbr_hv_stage(H, x, y, 3)
    assert "stage 2" in str(e.value)
    for stage in (2, 3, 4):
        G.gbr_hv_stage(H, x, y, stage)
    G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
    y2 = torch.empty_like(x)
    G.gbr_hv(H, x, y2)
    assert torch.equal(y, y2)
