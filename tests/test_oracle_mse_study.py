"""The MSE study of Sec. 3.5 (Numerical comparison) replayed with the oracle.

Two noisy harmonic series (N = 71, noise sd 5): the mean squared errors of
the rank-r reconstruction (SSA per series, MSSA of the pair) and of the
24-term recurrent and vector forecasts (column and row), averaged over
replications, against the
values printed in Tables tab:mssa:an and tab:mssa:for
(``tests/golden/paper_values.json``).  The paper used 10000 replications;
2000 here leave a Monte-Carlo spread of about 2% (reconstruction) and 4%
(forecast), so the tolerances are 5% and 8%.  A dropped term or wrong index
in the reconstruction or the recurrence moves these figures far more.
"""
import json
import os

import numpy as np
import pytest

from oracle import ssa_oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))["mse_tables"]
N, SD, M = GOLD["N"], GOLD["noise_sd"], GOLD["M"]
REPS = 2000
FORECAST = {"for": O.forecast_recurrent_column, "vec": O.forecast_vector_column,
            "for_row": O.forecast_recurrent_row, "vec_row": O.forecast_vector_row}


def signals(ex, k):
    h1 = 30 * np.cos(2 * np.pi * k / 12)
    h2 = 20 * np.cos(2 * np.pi * k / 12 + np.pi / 4) if ex == "A" else 20 * np.cos(2 * np.pi * k / 8 + np.pi / 4)
    return h1, h2


def mse(ex, L, method, task, seed):
    rng = np.random.default_rng(seed)
    k = np.arange(1, N + 1, dtype=float)
    h1, h2 = signals(ex, k)
    f1, f2 = signals(ex, np.arange(N + 1, N + M + 1, dtype=float))
    r = 2 if (method == "ssa" or ex == "A") else 4
    tot = 0.0
    for _ in range(REPS):
        xs = [h1 + SD * rng.normal(size=N), h2 + SD * rng.normal(size=N)]
        problems = [O.Problem.series(x, L) for x in xs] if method == "ssa" else [O.Problem.multi(xs, L)]
        outs = []
        for P in problems:
            s, U, V = O.decompose(P, r)
            if task == "rec":
                outs += [c[:, 0] for c in O.reconstruct(P, s, U, V, [list(range(r))])[0]]
            else:
                outs += FORECAST[task](P, s, U, V, list(range(r)), M)
        ref = (h1, h2) if task == "rec" else (f1, f2)
        tot += 0.5 * (np.mean((outs[0] - ref[0]) ** 2) + np.mean((outs[1] - ref[1]) ** 2))
    return tot / REPS


CASES = [
    ("rec", "A", 24, "ssa", GOLD["reconstruction"]["SSA_ABC"][1], 0.05),
    ("rec", "A", 48, "mssa", GOLD["reconstruction"]["MSSA_AB"][3], 0.05),
    ("rec", "C", 48, "mssa", GOLD["reconstruction"]["MSSA_C"][3], 0.05),
    ("for", "A", 24, "ssa", GOLD["forecast_recurrent"]["A"]["SSA"][1], 0.08),
    ("for", "A", 24, "mssa", GOLD["forecast_recurrent"]["A"]["MSSA_column"][1], 0.08),
    ("for", "C", 24, "mssa", GOLD["forecast_recurrent"]["C"]["MSSA_column"][1], 0.08),
    ("vec", "A", 24, "ssa", GOLD["forecast_vector"]["A"]["SSA"][1], 0.08),
    ("vec", "A", 48, "mssa", GOLD["forecast_vector"]["A"]["MSSA_column"][3], 0.08),
    ("vec", "C", 48, "mssa", GOLD["forecast_vector"]["C"]["MSSA_column"][3], 0.08),
    ("for_row", "A", 48, "mssa", GOLD["forecast_recurrent"]["A"]["MSSA_row"][3], 0.08),
    ("vec_row", "A", 24, "mssa", GOLD["forecast_vector"]["A"]["MSSA_row"][1], 0.08),
    ("vec_row", "C", 24, "mssa", GOLD["forecast_vector"]["C"]["MSSA_row"][1], 0.08),
]


@pytest.mark.parametrize("task,ex,L,method,paper,rtol", CASES,
                         ids=[f"{c[0]}_{c[1]}_L{c[2]}_{c[3]}" for c in CASES])
def test_mse_study_against_paper_tables(task, ex, L, method, paper, rtol):
    got = mse(ex, L, method, task, seed=11 + L + (0 if method == "ssa" else 1) + {"rec": 0, "for": 2, "vec": 4, "for_row": 6, "vec_row": 8}[task])
    assert abs(got - paper) <= rtol * paper, (got, paper)
