"""Per-step records of a population-annealing run as JSON lines.

One record per temperature step (Sec. 2 step 4 and Eq. 2 of arXiv:1704.01888):
beta, the step dbeta, the population size R_i, ln Q_i and ln Z_i, the energy
and magnetisation per site, the specific heat per site, the family entropy
and family count, the near-tie count of the step's copy numbers, and, where
the caller knows them, the adaptive schedule's overlap target and the run's
mean time per step.  Pure Python over the library's observables.
"""
from __future__ import annotations

import json


def step_records(obs, N: int, beta_prev: float, seconds_per_step: float | None = None,
                 overlap_target: float | None = None) -> list:
    """Records of consecutive steps from their observables (the dicts that
    Population.run returns); beta_prev is the inverse temperature before the
    first of them."""
    out = []
    b = float(beta_prev)
    for o in obs:
        rec = {"beta": o["beta"], "dbeta": o["beta"] - b, "R": int(o["R"]), "lnQ": o["lnQ"], "lnZ": o["lnZ"],
               "e": o["meanE"] / N, "C": o["C"], "m": o["meanM"] / N, "S_f": o["S_f"],
               "n_families": int(o["n_families"]), "n_near_ties": int(o["n_near_ties"])}
        if overlap_target is not None:
            rec["overlap_target"] = overlap_target
        if seconds_per_step is not None:
            rec["seconds_per_step"] = seconds_per_step
        out.append(rec)
        b = o["beta"]
    return out


def write_jsonl(dest, records) -> None:
    """Appends the records to dest (a path or an open text file), one JSON
    object per line."""
    if hasattr(dest, "write"):
        for r in records:
            dest.write(json.dumps(r) + "\n")
        return
    with open(dest, "a") as f:
        for r in records:
            f.write(json.dumps(r) + "\n")
