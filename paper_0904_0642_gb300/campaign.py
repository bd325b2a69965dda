"""The paper's verification runs on the GPU (Sec. 3): eq. act1, Tables 1-3.

Statistics as in the paper (Sec. 3.1.1): nequi = 2^12 equilibration
sweeps, then nrpt = 32 repetitions of nmeas = 2^12 measurements taken
every nsw = 2 sweeps; the 32 repetitions are the bins of the error bar.
The FHKP heatbath runs with nhit = 1 (the paper's mc.par).  `scale`
multiplies nequi and nmeas (the tests use a fraction of the paper's
statistics).

Undivided lattices run together in one ensemble (one fused launch per
tick).  Rows of Tables 1 and 3 with np > 1 (mpifactor 2, ndmpi 1..3) run
as divided lattices (sublattice boxes with halo exchange) with their own
seeds: like the paper's lsd2mpi = true runs they are statistically
independent repetitions, compared by Gaussian difference tests with the
row above and with the paper's reference row.

Usage: python -m paper_0904_0642_gb300.campaign [--scale S] [--json FILE]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import analysis
from . import (SU3_DLT, SU3_FP32_12, SU3_PBC, SU3_START_COLD, SU3_START_HOT, Ensemble, Lattice, make_config)

# Reference values printed in the paper: value, error, citation.
PAPER = {
    "act1_mpi": (0.53811, 0.00019, "Sec. 3.1.1, eq. act1MPI"),
    "act1_single": (0.53770, 0.00018, "Sec. 3.1.1, eq. act1noMPI"),
    "tab1_nonmpi": (0.538547, 0.000070, "Table 1, first row"),
    "tab2_space_Bo96": (0.537638, 0.000017, "Table 2, row B"),
    "tab2_time_Bo96": (0.537692, 0.000019, "Table 2, row B"),
    "tab2_space_nonmpi": (0.537650, 0.000015, "Table 2, second row"),
    "tab2_time_nonmpi": (0.537711, 0.000014, "Table 2, second row"),
    "tab3_np2": (0.510608, 0.000033, "Table 3, first row"),
}
TAU_INT_ACT1 = (49.5, 3.4, "Sec. 3.1.1")

NRPT, NSW = 32, 2


def _stats(scale: float):
    """(nequi, nmeas): nmeas scales; equilibration keeps at least 1024 sweeps."""
    nmeas = max(8, int(round(4096 * scale)))
    nequi = int(round(4096 * max(scale, 0.25))) // NSW * NSW
    return nequi, nmeas


# name, dims, boundary, beta, start, the paper's reference keys, observables
UNDIVIDED = [
    ("act1", [4, 4, 4, 4], SU3_PBC, 5.6, SU3_START_COLD, ["act1_single", "act1_mpi"], "total"),
    ("tab1", [8, 8, 8, 4], SU3_PBC, 5.65, SU3_START_COLD, ["tab1_nonmpi"], "total"),
    ("tab2", [16, 16, 16, 4], SU3_PBC, 5.65, SU3_START_COLD,
     ["tab2_space_Bo96", "tab2_space_nonmpi", "tab2_time_Bo96", "tab2_time_nonmpi"], "space+time"),
    ("tab3", [8, 8, 8, 4], SU3_DLT, 5.55, SU3_START_HOT, ["tab3_np2"], "total"),
]
# (table, dims, boundary, beta, start, ndiv, np as the paper counts processes)
DIVIDED = [
    ("tab1", [8, 8, 8, 4], SU3_PBC, 5.65, SU3_START_COLD, [2, 1, 1, 1], 2),
    ("tab1", [8, 8, 8, 4], SU3_PBC, 5.65, SU3_START_COLD, [2, 2, 1, 1], 4),
    ("tab1", [8, 8, 8, 4], SU3_PBC, 5.65, SU3_START_COLD, [2, 2, 2, 1], 8),
    ("tab3", [8, 8, 8, 4], SU3_DLT, 5.55, SU3_START_HOT, [2, 1, 1, 1], 4),
    ("tab3", [8, 8, 8, 4], SU3_DLT, 5.55, SU3_START_HOT, [2, 2, 1, 1], 8),
    ("tab3", [8, 8, 8, 4], SU3_DLT, 5.55, SU3_START_HOT, [2, 2, 2, 1], 16),
]


def _observables(m: np.ndarray, nlayers: int, skip: int) -> dict:
    """Series of the whole-lattice plaquette averages after equilibration:
    m[k, slot, (total, space, time, poly_re, poly_im)], slot nlayers = all."""
    w = m[skip:, nlayers, :]
    return {"total": w[:, 0], "space": w[:, 1], "time": w[:, 2]}


def _analyse(series: np.ndarray) -> dict:
    mean, err = analysis.binned_mean_error(series, NRPT)
    tau, window = analysis.tau_int_window(series)
    return {"mean": mean, "err": err, "tau_int": tau, "tau_window": window, "n": int(len(series)),
            "text": analysis.format_value(mean, err)}


def run(scale: float = 1.0, seed: int = 20090406, divided: bool = True, log=print) -> dict:
    nequi, nmeas = _stats(scale)
    total = nequi + NRPT * nmeas * NSW
    skip = nequi // NSW
    cap = total // NSW + 8
    out = {"scale": scale, "nequi": nequi, "nmeas": nmeas, "nrpt": NRPT, "nsw": NSW, "sweeps": total, "rows": []}
    kw = dict(storage=SU3_FP32_12, hits=1, reunit_every=10, measure_every=NSW, measure_capacity=cap)

    cfgs = [make_config(d, boundary=b, beta=beta, seed=seed + i, start=st, **kw)
            for i, (_, d, b, beta, st, _, _) in enumerate(UNDIVIDED)]
    t0 = time.time()
    ens = Ensemble(cfgs)
    ens.sweep(total)
    out["ensemble_seconds"] = time.time() - t0
    log(f"ensemble of {len(cfgs)} undivided runs: {total} sweeps each in {out['ensemble_seconds']:.1f} s")
    results = {}
    for i, (name, dims, b, beta, st, refs, obs) in enumerate(UNDIVIDED):
        nl = 2 if b == SU3_DLT else 1
        series = _observables(ens.measurements(i, max_entries=cap), nl, skip)
        keys = ["space", "time"] if obs == "space+time" else ["total"]
        for k in keys:
            r = _analyse(series[k])
            r.update(run=name, observable=k, lattice="x".join(map(str, dims)) + (" DLT" if nl == 2 else ""),
                     beta=beta, np="-")
            for ref in refs:
                if obs == "space+time" and k not in ref:
                    continue
                v, e, cite = PAPER[ref]
                r.setdefault("q", {})[ref] = analysis.gaussian_difference_q(r["mean"], r["err"], v, e)
            results[(name, k)] = r
            out["rows"].append(r)
    ens.close()

    if divided:
        above = {"tab1": results[("tab1", "total")], "tab3": results[("tab3", "total")]}
        for j, (table, dims, b, beta, st, ndiv, np_) in enumerate(DIVIDED):
            lat = Lattice(dims, boundary=b, beta=beta, seed=seed + 100 + j, start=st, ndiv=ndiv, **kw)
            t0 = time.time()
            lat.sweep(total)
            secs = time.time() - t0
            nl = 2 if b == SU3_DLT else 1
            r = _analyse(_observables(lat.measurements(max_entries=cap), nl, skip)["total"])
            lat.close()
            ref = "tab1_nonmpi" if table == "tab1" else "tab3_np2"
            v, e, _ = PAPER[ref]
            prev = above[table]
            r.update(run=table, observable="total", lattice="x".join(map(str, dims)) + (" DLT" if nl == 2 else ""),
                     beta=beta, np=np_, ndiv=ndiv, seconds=secs,
                     q={ref: analysis.gaussian_difference_q(r["mean"], r["err"], v, e),
                        "row_above": analysis.gaussian_difference_q(r["mean"], r["err"], prev["mean"], prev["err"])})
            above[table] = r
            out["rows"].append(r)
            log(f"{table} np={np_} ndiv={ndiv}: {r['text']} in {secs:.1f} s")
    return out


def report(out: dict) -> str:
    lines = [f"statistics: nequi={out['nequi']}, {out['nrpt']} x nmeas={out['nmeas']} measurements every "
             f"{out['nsw']} sweeps ({out['sweeps']} sweeps per run), error bars from {out['nrpt']} bins",
             f"{'run':6s}{'lattice':16s}{'beta':>6s}{'np':>4s}{'obs':>7s}{'value':>18s}{'tau_int':>9s}  Q"]
    for r in out["rows"]:
        qs = ", ".join(f"{k} {v:.2f}" for k, v in r.get("q", {}).items())
        lines.append(f"{r['run']:6s}{r['lattice']:16s}{r['beta']:6.2f}{str(r['np']):>4s}{r['observable']:>7s}"
                     f"{r['text']:>18s}{r['tau_int']:9.1f}  {qs}")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the paper's statistics")
    ap.add_argument("--seed", type=int, default=20090406)
    ap.add_argument("--no-divided", action="store_true", help="skip the divided-lattice rows")
    ap.add_argument("--json", default=None, help="write the results here")
    a = ap.parse_args(argv)
    out = run(a.scale, a.seed, divided=not a.no_divided)
    print(report(out))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(out, f, indent=1, default=float)


if __name__ == "__main__":
    main()
