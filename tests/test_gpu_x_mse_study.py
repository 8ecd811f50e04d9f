"""The MSE study of Sec. 3.5 replayed through the library on the GPU.

The same noisy harmonic pairs (N = 71, noise sd 5) go through the C ABI and
through the oracle: the library's mean squared errors of the rank-r
reconstruction and of the 24-term forecasts must equal the oracle's on the
same noise (1% -- the FP32 form's component error is far below the noise),
and both must match the printed Tables tab:mssa:an and tab:mssa:for within
the Monte-Carlo spread of 400 replications (12%).
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_5050_gb300 as pkg  # noqa: E402
from oracle import ssa_oracle as O  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))["mse_tables"]
N, SD, M = GOLD["N"], GOLD["noise_sd"], GOLD["M"]
REPS = 400
ORACLE_FC = {"recurrent": O.forecast_recurrent_column, "vector": O.forecast_vector_column,
             "recurrent_row": O.forecast_recurrent_row, "vector_row": O.forecast_vector_row}


def signals(ex, k):
    h1 = 30 * np.cos(2 * np.pi * k / 12)
    h2 = 20 * np.cos(2 * np.pi * k / 12 + np.pi / 4) if ex == "A" else 20 * np.cos(2 * np.pi * k / 8 + np.pi / 4)
    return h1, h2


def study(ex, L, multi, task, seed):
    """(library MSE, oracle MSE) over REPS replications of the same noise;
    the MSSA inputs are rounded to FP32 for both (the library stores them so)."""
    rng = np.random.default_rng(seed)
    k = np.arange(1, N + 1, dtype=float)
    h1, h2 = signals(ex, k)
    ref = signals(ex, np.arange(N + 1, N + M + 1, dtype=float)) if task != "rec" else (h1, h2)
    r = 2 if (not multi or ex == "A") else 4
    grp = list(range(r))
    tot_g = tot_o = 0.0
    for _ in range(REPS):
        xs = [h1 + SD * rng.normal(size=N), h2 + SD * rng.normal(size=N)]
        if multi:
            xs = [np.asarray(x, np.float32).astype(np.float64) for x in xs]
            runs = [(pkg.SSA.multi(xs, L), O.Problem.multi(xs, L))]
        else:
            runs = [(pkg.SSA.series(x, L), O.Problem.series(x, L)) for x in xs]
        got, exp = [], []
        for s, P in runs:
            s.decompose(r, "fp32")
            so, Uo, Vo = O.decompose(P, r)
            if task == "rec":
                g = s.reconstruct([grp])[0]
                got += g if isinstance(g, list) else [g]
                exp += [c[:, 0] for c in O.reconstruct(P, so, Uo, Vo, [grp])[0]]
            else:
                g = s.forecast(grp, M, method=task)
                got += g if isinstance(g, list) else [g]
                exp += ORACLE_FC[task](P, so, Uo, Vo, grp, M)
            s.close()
        tot_g += 0.5 * (np.mean((got[0] - ref[0]) ** 2) + np.mean((got[1] - ref[1]) ** 2))
        tot_o += 0.5 * (np.mean((exp[0] - ref[0]) ** 2) + np.mean((exp[1] - ref[1]) ** 2))
    return tot_g / REPS, tot_o / REPS


CASES = [
    ("rec", "A", 24, False, GOLD["reconstruction"]["SSA_ABC"][1]),
    ("rec", "A", 48, True, GOLD["reconstruction"]["MSSA_AB"][3]),
    ("recurrent", "A", 24, True, GOLD["forecast_recurrent"]["A"]["MSSA_column"][1]),
    ("vector", "A", 48, True, GOLD["forecast_vector"]["A"]["MSSA_column"][3]),
    ("vector_row", "A", 24, True, GOLD["forecast_vector"]["A"]["MSSA_row"][1]),
]


@pytest.mark.parametrize("task,ex,L,multi,paper", CASES,
                         ids=[f"{c[0]}_{c[1]}_L{c[2]}_{'mssa' if c[3] else 'ssa'}" for c in CASES])
def test_mse_study_on_the_gpu(task, ex, L, multi, paper):
    g, o = study(ex, L, multi, task, seed=31 + L)
    assert abs(g - o) <= 0.01 * o, (g, o)
    assert abs(g - paper) <= 0.12 * paper, (g, paper)
