"""Writes reference_energies.json: ground-state energies of the extra
configurations the benchmark reports, computed by the oracle alone.

* the L = 8 ring (t = 1, U = 4, N_up = N_dn = 4): dense diagonalisation;
* the U = 0 limits of the L = 18 ring and of the 4x4 t' torus: the closed
  form (sum of the lowest one-body levels);
* impurity models 0, 128 and 255 of the batched workload: the lowest energy
  over every (N_up, N_dn) sector, by dense diagonalisation up to 600 states
  and by the oracle's FP64 Lanczos with full re-orthogonalisation above;
* the L = 18 ring at U = 4 (N_up = N_dn = 9): the Lieb-Wu Bethe-ansatz
  equations (pinned against dense diagonalisation at L = 4, 6, 8 and the
  oracle's Lanczos at L = 10);
* the 4x4 t' torus at U = 8 with N_up = N_dn = 3 (313,600 states, the
  workload's geometry and couplings at a filling the oracle can solve):
  the oracle's FP64 Lanczos, 200 steps from the seed-1 start vector; the
  change of the lowest Ritz value over the last 50 steps is stored beside it
  as the convergence record (minutes of CPU time).

Run from the repository root: python tests/golden/make_reference_energies.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import gbr_synth as S  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "reference_energies.json")
SIAM_MODELS = (0, 128, 255)


def sector_E0(L, h, U, a, c):
    D = oracle.sector_dim(L, a, c)
    if D <= 600:
        return oracle.dense_E0(L, h, U, a, c)
    return oracle.lanczos(L, h, U, a, c, S.start_vector(D, 77), min(160, D), True)["E0"]


def siam_E0(m):
    h, U = S.siam(m)
    L = h.shape[0]
    return min(sector_E0(L, h, U, a, c) for a in range(L + 1) for c in range(L + 1))


def square_U8_N3_E0():
    h, U = S.square(4, 4, 1.0, -0.3), S.uniform_U(16, 8.0)
    D = oracle.sector_dim(16, 3, 3)
    o = oracle.lanczos(16, h, U, 3, 3, S.start_vector(D), 200, False)
    return o["E0"], float(abs(o["ritz"][-1] - o["ritz"][-51]))


def compute():
    E_sq, d_sq = square_U8_N3_E0()
    return {
        "chain18_U4_N9_9_bethe_E0": oracle.bethe_ansatz_E0(18, 9, 9, 4.0)[0],
        "square4x4_tp_U8_N3_3_lanczos_E0": E_sq,
        "square4x4_tp_U8_N3_3_lanczos_change_last_50_steps": d_sq,
        "ring8_U4_N4_4_dense_E0": oracle.dense_E0(8, S.chain(8), S.uniform_U(8, 4.0), 4, 4),
        "chain18_U0_N9_9_free_E0": oracle.free_E0(S.chain(18), 9, 9),
        "square4x4_tp_U0_N7_7_free_E0": oracle.free_E0(S.square(4, 4, 1.0, -0.3), 7, 7),
        "siam_lowest_E0": {str(m): siam_E0(m) for m in SIAM_MODELS},
    }


if __name__ == "__main__":
    data = {"_about": "written by make_reference_energies.py from the oracle only"}
    data.update(compute())
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)
    print(json.dumps(data, indent=1))
