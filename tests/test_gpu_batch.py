"""Batched impurity solver: every (N_up, N_dn) sector of many Anderson
models in one persistent launch, against the oracle sector by sector."""
import numpy as np
import pytest

import gbr_synth as S
import oracle
from gpu_common import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return lib()


def ref_sector_E(h, U, Nu, Nd):
    L = h.shape[0]
    D = oracle.sector_dim(L, Nu, Nd)
    if D <= 600:
        return oracle.dense_E0(L, h, U, Nu, Nd)
    return oracle.lanczos(L, h, U, Nu, Nd, S.start_vector(D, 77), min(D, 160), True)["E0"]


def run_batch(G, models, iters=150):
    import gbr_synth.gpu as SG
    ns, nst = G.gbr_batch_layout(models)
    start = SG.uniform(S.SEED_START, nst)
    return ns, G.gbr_batch_solve(models, start, iters)


def test_batch_small_set_every_sector(G):
    models = [S.siam(m) for m in range(12)]
    ns, res = run_batch(G, models)
    k = 0
    for m, (h, U) in enumerate(models):
        L = h.shape[0]
        best = None
        for Nu in range(L + 1):
            for Nd in range(L + 1):
                E = ref_sector_E(h, U, Nu, Nd)
                assert abs(res["sector_E"][k] - E) <= 1e-9 * max(1.0, abs(E)), (m, Nu, Nd, res["sector_E"][k], E)
                best = E if best is None else min(best, E)
                k += 1
        assert abs(res["E0"][m] - best) <= 1e-9 * max(1.0, abs(best))
        nu, nd = res["arg"][m]
        # the arg sector attains the minimum, and ties go to the lower N, then the lower N_up
        assert abs(ref_sector_E(h, U, nu, nd) - best) <= 1e-9 * max(1.0, abs(best))
    assert k == ns


def test_batch_256_models_sampled(G):
    models = [S.siam(m) for m in range(256)]
    ns, res = run_batch(G, models)
    assert 15000 < ns < 19000
    for m in (0, 77, 255):
        h, U = models[m]
        L = h.shape[0]
        best = min(ref_sector_E(h, U, a, b) for a in range(L + 1) for b in range(L + 1))
        assert abs(res["E0"][m] - best) <= 1e-9 * max(1.0, abs(best))
