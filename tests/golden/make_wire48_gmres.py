"""Write tests/golden/wire48_gmres.json: oracle values for the 48 x 48 x 160 wire.

The direct oracle cannot factor this operator (its dense Eq. 8 end blocks alone
are (4 * 2304)^2 per end), so every open incident channel of the sampled
energies is solved by the iterative FP64 oracle (oracle/iterative.py:
preconditioned restarted GMRES with refinement on the true residual of the
matrix-free Eq. 7 operator, to ||b - A psi|| / ||b|| <= 1e-12), projected with
the explicit Eq. 19 sums (Eq. 6) and reduced to T, R and G (Sec. III).

Sampled energies (indices into the 32 of linspace(E_F - 2 eV, E_F + 0.5 eV)):
13, 14, 15 -- just below the opening of four new channels, the slowest energies
of the mixed-precision solver -- and 31 (E_F + 0.5 eV, the most open channels).

Only oracle/ and the seeded input generator are called.  Channels run in
worker processes (spawn start method, one BLAS thread each).

    python tests/golden/make_wire48_gmres.py [--workers N]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "wire48_gmres.json")
ENERGY_INDICES = (13, 14, 15, 31)
TOL = 1e-12


def _one(job):
    e_idx, chan = job
    sys.path.insert(0, ROOT)
    import iobm_synth as S
    from oracle import iterative
    jn = S.wire48()
    E = float(jn.energies[e_idx])
    t0 = time.perf_counter()
    sol = iterative.solve_gmres(jn, E, side="L", channels=[chan], tol=TOL)
    return {"e_idx": e_idx, "chan": chan, "t": [[c.real, c.imag] for c in sol.t[:, 0]],
            "r": [[c.real, c.imag] for c in sol.r[:, 0]],
            "T": sol.T[:, 0].tolist(), "R": sol.R[:, 0].tolist(),
            "residual": float(sol.residuals[0]), "gmres_matvecs": int(sol.gmres_iterations[0]),
            "seconds": time.perf_counter() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    args = ap.parse_args()
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    sys.path.insert(0, ROOT)
    import iobm_synth as S
    from oracle import modes
    jn = S.wire48()
    energies = {}
    jobs = []
    for i in ENERGY_INDICES:
        E = float(jn.energies[i])
        md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, jn.nf, E)
        opens = md.open_modes
        energies[i] = {"E": E, "n_open": int(len(opens)),
                       "nu": [[int(a) for a in md.nu[m]] for m in opens],
                       "vel": [float(md.vel[m]) for m in opens]}
        jobs += [(i, c) for c in range(len(opens))]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(args.workers) as pool:
        done = pool.map(_one, jobs, chunksize=1)
    out = {"workload": "wire48 (48x48x160, h=0.35, 6 Gaussian wells + s/p KB, r_s=3.28, seed 1000), "
                       "left incidence",
           "oracle": "oracle.iterative.solve_gmres (FP64 preconditioned GMRES + refinement, "
                     "matrix-free Eq. 7 operator, explicit Eq. 19 projection)",
           "tol": TOL, "energies": []}
    for i in ENERGY_INDICES:
        rows = sorted((d for d in done if d["e_idx"] == i), key=lambda d: d["chan"])
        ent = dict(energies[i])
        ent["index"] = i
        ent["channels"] = rows
        ent["G"] = float(sum(sum(d["T"]) for d in rows))
        out["energies"].append(ent)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {OUT}: {len(jobs)} channel solves in {time.perf_counter() - t0:.0f} s; "
          f"max residual {max(d['residual'] for d in done):.2e}")


if __name__ == "__main__":
    main()
