"""gbr_hv_static, the H·v entry point for callers that cannot allocate
device memory when they multiply (for example code that runs under a fixed
memory budget handed out by a host framework, or a loop that must never
reach the allocator).

It must give the same product as gbr_hv, call after call, with its scratch
in the library's static device array instead of freshly allocated memory.
This file is collected last so that a failure here stops a run only after
every other test has run; it passes alone in a fresh process too.
"""
import numpy as np
import pytest

import gbr_synth as S
from gpu_common import lib, rel_inf

pytestmark = pytest.mark.gpu

TOL = {32: 1e-5, 64: 1e-12}   # the tolerances of the other H·v parity tests


@pytest.fixture(scope="module")
def G():
    return lib()


def sectors():
    # 12-site ring at half filling (853,776 states) and a 4x3 torus with
    # diagonal hopping and N_up != N_dn (731,808 states): both need less
    # than the 64 MiB of static scratch in FP64
    yield 12, S.chain(12), S.uniform_U(12, 4.0), 6, 6
    yield 12, S.square(4, 3, 1.0, -0.3), S.uniform_U(12, 8.0), 5, 6


@pytest.mark.parametrize("fp", [32, 64])
def test_static_scratch_hv_matches_gbr_hv_on_consecutive_calls(G, fp):
    """Same kernels and launch shapes as gbr_hv's factored path, so the two
    products agree bit for bit (the tolerance of the other parity tests is
    checked as well); the first call on a fresh handle comes before any
    gbr_hv and must not allocate the handle's own scratch."""
    import torch
    import gbr_synth.gpu as SG
    # one call on another handle first: with lazy module loading it is the
    # call that loads the module holding the static array (64 MiB), which is
    # not an allocation by the call being measured below
    Hw = G.gbr_ham_create(8, S.chain(8), S.uniform_U(8, 4.0), 4, 4)
    xw = torch.zeros(4900, dtype=torch.float32 if fp == 32 else torch.float64, device="cuda")
    G.gbr_hv_static(Hw, xw, torch.empty_like(xw))
    for L, h, U, Nu, Nd in sectors():
        H = G.gbr_ham_create(L, h, U, Nu, Nd)
        G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
        D, _ = G.gbr_ham_info(H)
        for call, seed in enumerate((41, 42)):
            x = SG.uniform(seed, D)
            if fp == 32:
                x = x.float()
            y = torch.full_like(x, float("nan"))
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            G.gbr_hv_static(H, x, y)
            torch.cuda.synchronize()
            if call == 0:
                # one scratch vector is D * fp / 8 bytes: the call took none
                assert free0 - torch.cuda.mem_get_info()[0] < D * fp // 8
            y_ref = torch.empty_like(x)
            G.gbr_hv(H, x, y_ref)
            torch.cuda.synchronize()
            err = rel_inf(y.double().cpu().numpy(), y_ref.double().cpu().numpy())
            assert err <= TOL[fp], (L, Nu, Nd, fp, call, err)
            assert torch.equal(y, y_ref), (L, Nu, Nd, fp, call)


def test_static_scratch_limit_is_per_precision(G):
    """A 14-site ring with N_up = 5, N_dn = 7 (6,870,864 states): its two
    FP32 scratch vectors (55 MB) fit the 64 MiB array, its FP64 ones do not."""
    import torch
    import gbr_synth.gpu as SG
    H = G.gbr_ham_create(14, S.chain(14), S.uniform_U(14, 4.0), 5, 7)
    G.gbr_ham_set_path(H, G.GBR_HV_FACTORED)
    D, _ = G.gbr_ham_info(H)
    assert D == 6870864
    x = SG.uniform(43, D).float()
    y, y_ref = torch.empty_like(x), torch.empty_like(x)
    G.gbr_hv_static(H, x, y)
    G.gbr_hv(H, x, y_ref)
    assert torch.equal(y, y_ref)
    x64 = x.double()
    with pytest.raises(G.GbrError) as e:
        G.gbr_hv_static(H, x64, torch.empty_like(x64))
    assert e.value.code == G.GBR_EINVAL and "scratch" in str(e.value)


def test_static_scratch_rejects_sectors_beyond_its_size(G):
    import torch
    H = G.gbr_ham_create(16, S.square(4, 4, 1.0, -0.3), S.uniform_U(16, 8.0), 7, 7)   # 1.3e8 states
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(G.GbrError) as e:
        G.gbr_hv_static(H, x, torch.zeros_like(x))
    assert e.value.code == G.GBR_EINVAL and "scratch" in str(e.value)
