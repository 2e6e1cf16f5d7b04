"""Cycle counts of the oracle under the protocol of the paper's Sec. 6, for each reading of
Sec. 5.2's subdomains and local pressure spaces, beside the counts the paper prints.

TEST INFRASTRUCTURE ONLY (part of the oracle).  Run on the host:

    python -m oracle.paper_tables [--max-nl2d 5] [--max-nl3d 2] [--procs 8]

Protocol (Sec. 6 preamble): V(1,2) cycles, coarsest mesh one element, fine mesh 2^n_l
elements per direction, random divergence-free initial guess, convergence when the initial
residual is reduced by 1e6, C_I = 4(p-1), manufactured forcing (Sec. 6.1 / Sec. 6.3 solution
fields), nu = 1 and sigma = Da.  Additive smoother with eta = 0.5 (Table 2).
"""
import argparse
import itertools
import multiprocessing as mp
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

READINGS = [("interior", "border"), ("all", "border"), ("interior", "pin"), ("interior", "lstsq")]


def _paper(name):
    rows, cur = {}, None
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_tables.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha():
            cur = line
            rows[cur] = []
            continue
        rows[cur].append([float(x) for x in line.split()])
    return rows[name]


def cycles_2d(p, nl, da, smoother="mult", eta=0.5, patch_set="interior", local_pressure="border",
              seed=None, max_cycles=60):
    from paper_1705_09282_gb300 import inputs

    from . import stokes2d as o2
    n = 2 ** nl
    H = o2.Hierarchy(p, n, nl + 1, float(da), 1.0, smoother=smoother, eta=eta, nu1=1, nu2=2,
                     patch_set=patch_set, local_pressure=local_pressure)
    S = H.fine
    psi, pr = inputs.random_divfree_guess(p, n, seed=nl if seed is None else seed)
    U = S.curl(psi)
    U[S.n_u: S.n_u + S.n_p] = pr
    F = S.load_vector(inputs.manufactured_forcing(p, n, float(da), 1.0))
    k, hist = H.solve(U, F, 1e-6, max_cycles)
    if hist[-1] > 1e-6 * hist[0]:
        return None                      # no convergence within max_cycles
    return k


def cycles_3d(p, nl, da, patch_set="interior", local_pressure="border", seed=None, max_cycles=40):
    from paper_1705_09282_gb300 import inputs

    from . import stokes3d as o3
    n = 2 ** nl
    H = o3.Hierarchy3D(p, n, nl + 1, float(da), 1.0, nu1=1, nu2=2, patch_set=patch_set,
                       local_pressure=local_pressure)
    S = H.fine
    psi, pr = inputs.random_divfree_guess_3d(p, n, seed=nl if seed is None else seed)
    U = S.curl(psi)
    U[S.n_u: S.n_u + S.n_p] = pr
    F = S.load_vector(inputs.manufactured_forcing_3d(p, n, float(da), 1.0))
    k, hist = H.solve(U, F, 1e-6, max_cycles)
    if hist[-1] > 1e-6 * hist[0]:
        return None
    return k


def _job(args):
    kind, kw = args
    try:
        return kind, kw, (cycles_2d(**kw) if kind == "2d" else cycles_3d(**kw))
    except Exception as e:  # a reading whose local systems are singular
        return kind, kw, f"error: {type(e).__name__}"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--max-nl2d", type=int, default=5)
    ap.add_argument("--max-nl3d", type=int, default=2)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 4)
    a = ap.parse_args()
    jobs = []
    for (ps, lp), p, nl, da in itertools.product(READINGS, (2, 3), range(1, a.max_nl2d + 1), (1, 1000)):
        jobs.append(("2d", dict(p=p, nl=nl, da=da, patch_set=ps, local_pressure=lp)))
    for (ps, lp), nl, da in itertools.product(READINGS, range(1, a.max_nl2d + 1), (1, 1000)):
        jobs.append(("2d", dict(p=2, nl=nl, da=da, smoother="add", eta=0.5, patch_set=ps, local_pressure=lp)))
    for (ps, lp), p, nl, da in itertools.product(READINGS, (2, 3), range(1, a.max_nl3d + 1), (1, 1000)):
        jobs.append(("3d", dict(p=p, nl=nl, da=da, patch_set=ps, local_pressure=lp)))
    with mp.get_context("spawn").Pool(a.procs) as pool:
        res = pool.map(_job, jobs)
    out = {}
    for kind, kw, k in res:
        key = (kind, kw.get("smoother", "mult"), kw["p"], kw["da"], kw["patch_set"], kw["local_pressure"])
        out.setdefault(key, {})[kw["nl"]] = k
    t1, t2, t4 = _paper("table1"), _paper("table2"), _paper("table4")
    print("| table | smoother | p | Da | reading | " + " | ".join(f"n_l={i}" for i in range(1, a.max_nl2d + 1)) + " |")
    for key in sorted(out, key=str):
        kind, sm, p, da, ps, lp = key
        cnt = out[key]
        cells = [("—" if cnt.get(i) is None else str(cnt.get(i))) for i in range(1, max(cnt) + 1)]
        tab = "4" if kind == "3d" else ("2" if sm == "add" else "1")
        print(f"| {tab} | {sm} | {p} | {da} | {ps}/{lp} | " + " | ".join(cells) + " |")
    col = {1: 2, 1000: 3}
    for p, off in ((2, 0), (3, 3)):
        for da in (1, 1000):
            print(f"| 1 (paper) | mult | {p} | {da} | printed | " +
                  " | ".join(str(int(r[col[da] + off])) for r in t1[: a.max_nl2d]) + " |")
            print(f"| 4 (paper) | mult | {p} | {da} | printed | " +
                  " | ".join(str(int(r[col[da] + off])) for r in t4[: a.max_nl3d]) + " |")
    for da in (1, 1000):
        print(f"| 2 (paper) | add | 2 | {da} | printed | " +
              " | ".join(str(int(r[col[da]])) for r in t2[: a.max_nl2d]) + " |")


if __name__ == "__main__":
    main()
