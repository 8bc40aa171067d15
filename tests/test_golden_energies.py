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
    # the 18-site ring at U = 4: the Bethe-ansatz energy (recomputed, seconds)
    E_ba = oracle.bethe_ansatz_E0(18, 9, 9, 4.0)[0]
    assert abs(g["chain18_U4_N9_9_bethe_E0"] - E_ba) <= 1e-12 * abs(E_ba)
    # the reduced 4x4 sector (minutes to recompute): converged, and below the
    # U = 0 closed form shifted by the Hartree energy U N_up N_dn / L (the
    # variational bound of the uniform free state)
    E_sq = g["square4x4_tp_U8_N3_3_lanczos_E0"]
    assert g["square4x4_tp_U8_N3_3_lanczos_change_last_50_steps"] <= 1e-12 * abs(E_sq)
    E_free = oracle.free_E0(S.square(4, 4, 1.0, -0.3), 3, 3)
    assert E_free < E_sq < E_free + 8.0 * 9 / 16
    assert set(g["siam_lowest_E0"]) == {str(m) for m in mk.SIAM_MODELS}


def test_state_set_generators_match_the_oracle_enumeration():
    """The seeded-input module lists the state sets the benchmarks hand to the
    trie and set Hamiltonians; they equal the oracle's brute-force lists."""
    import numpy as np
    for M, N in ((1, 0), (1, 1), (7, 3), (16, 8), (20, 2), (24, 12)):
        assert np.array_equal(S.popcount_states(M, N), oracle.enumerate_sector(M, N)), (M, N)
    assert np.array_equal(S.sector_states(7, 3, 2), oracle.sector_states(7, 3, 2))
    assert np.array_equal(S.fixed_N_states(6, 6), oracle.fixed_N_states(6, 6))
