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


def test_batch_tuned_shapes_keep_parity(G):
    """The batch autotuner times every launch shape (CTA size x CTAs per SM)
    on a batch; the solve under every shape matches the oracle sector by
    sector, and the tuner's pick becomes the process-wide shape."""
    import gbr_synth.gpu as SG
    models = [S.siam(m) for m in (3, 40, 101)]
    ns, nst = G.gbr_batch_layout(models)
    start = SG.uniform(S.SEED_START, nst)
    ref = []
    for h, U in models:
        L = h.shape[0]
        ref.extend(ref_sector_E(h, U, a, b) for a in range(L + 1) for b in range(L + 1))
    ref = np.array(ref)
    keep = G.gbr_batch_get_shape()
    try:
        for threads in (128, 256, 512):
            for per_sm in (0, 2, 1):
                G.gbr_batch_set_shape(threads, per_sm)
                res = G.gbr_batch_solve(models, start, 150)
                err = np.abs(res["sector_E"] - ref) / np.maximum(1.0, np.abs(ref))
                assert err.max() <= 1e-9, (threads, per_sm, err.max())
        t = G.gbr_batch_tune(models, start, 150)
        assert (t["threads"], t["ctas_per_sm"]) in [(a, b) for a in (128, 256, 512) for b in (0, 2, 1)]
        assert len(t["candidate_ms"]) == 9 and min(t["candidate_ms"]) > 0
        assert G.gbr_batch_get_shape() == {"threads": t["threads"], "ctas_per_sm": t["ctas_per_sm"]}
    finally:
        G.gbr_batch_set_shape(keep["threads"], keep["ctas_per_sm"])
    with pytest.raises(G.GbrError):
        G.gbr_batch_set_shape(100, 0)
