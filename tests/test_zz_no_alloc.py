"""gbr_hv_static, the H·v entry point for callers that cannot allocate
device memory when they multiply (for example while a stream is being
captured into a CUDA graph, or under a fixed memory budget).

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
    import torch
    import gbr_synth.gpu as SG
    for L, h, U, Nu, Nd in sectors():
        H = G.gbr_ham_create(L, h, U, Nu, Nd)
        D, _ = G.gbr_ham_info(H)
        for call, seed in enumerate((41, 42)):
            x = SG.uniform(seed, D)
            if fp == 32:
                x = x.float()
            y_ref = torch.empty_like(x)
            G.gbr_hv(H, x, y_ref)
            y = torch.full_like(x, float("nan"))
            G.gbr_hv_static(H, x, y)
            torch.cuda.synchronize()
            err = rel_inf(y.double().cpu().numpy(), y_ref.double().cpu().numpy())
            assert err <= TOL[fp], (L, Nu, Nd, fp, call, err)


def test_static_scratch_rejects_sectors_beyond_its_size(G):
    import torch
    H = G.gbr_ham_create(16, S.square(4, 4, 1.0, -0.3), S.uniform_U(16, 8.0), 7, 7)   # 1.3e8 states
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(G.GbrError) as e:
        G.gbr_hv_static(H, x, torch.zeros_like(x))
    assert e.value.code == G.GBR_EINVAL and "scratch" in str(e.value)
