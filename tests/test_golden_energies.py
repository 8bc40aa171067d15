"""The stored reference energies (tests/golden/reference_energies.json,
read by the benchmark's extra configurations) are the oracle's: rerunning
their generator reproduces them, and the U = 0 entries meet the closed
forms printed for the workloads (-26.4 for the 4x4 t' torus)."""
import importlib.util
import json
import os

import gbr_synth as S
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "reference_energies.json")


def _maker():
    spec = importlib.util.spec_from_file_location("make_reference_energies",
                                                  os.path.join(HERE, "golden", "make_reference_energies.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_energies_are_the_oracles():
    g = json.load(open(GOLDEN))
    assert abs(g["ring8_U4_N4_4_dense_E0"] - oracle.dense_E0(8, S.chain(8), S.uniform_U(8, 4.0), 4, 4)) <= 1e-12
    assert abs(g["chain18_U0_N9_9_free_E0"] - (-23.035081932575)) <= 1e-11
    assert abs(g["square4x4_tp_U0_N7_7_free_E0"] - (-26.4)) <= 1e-12
    mk = _maker()
    assert abs(g["siam_lowest_E0"]["0"] - mk.siam_E0(0)) <= 1e-12
    assert set(g["siam_lowest_E0"]) == {str(m) for m in mk.SIAM_MODELS}


def test_state_set_generators_match_the_oracle_enumeration():
    """The seeded-input module lists the state sets the benchmarks hand to the
    trie and set Hamiltonians; they equal the oracle's brute-force lists."""
    import numpy as np
    for M, N in ((1, 0), (1, 1), (7, 3), (16, 8), (20, 2), (24, 12)):
        assert np.array_equal(S.popcount_states(M, N), oracle.enumerate_sector(M, N)), (M, N)
    assert np.array_equal(S.sector_states(7, 3, 2), oracle.sector_states(7, 3, 2))
    assert np.array_equal(S.fixed_N_states(6, 6), oracle.fixed_N_states(6, 6))
