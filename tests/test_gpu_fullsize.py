"""Oracle parity on the 48x48x160 wire (the benchmark workload) in the launch
configuration the benchmark times: mixed precision (complex FP32 COCG, FP64
residual replacement and projection), free-propagator Fourier preconditioner,
implicit operator form, every open channel of several energies in one batch.

Expected values: tests/golden/wire48_gmres.json, written by
tests/golden/make_wire48_gmres.py, which calls only the oracle (FP64
preconditioned GMRES on the matrix-free Eq. 7 operator to a relative residual of
1e-12, explicit Eq. 19 projection, Eq. 6, Sec. III Landauer sum).  The sampled
energies are the three just below the opening of four new channels (the slowest
for the mixed solver) and the top of the window.

Bars (the accuracy the method is held to): conductance within 1e-6 G_0 of the oracle
per energy, every T and R entry within 1e-6, and for EVERY returned wave the oracle's
own matrix-free FP64 operator gives ||b - A psi|| / ||b|| <= 1e-8."""
import json
import os

import numpy as np
import pytest

import iobm_synth as S
from oracle import modes, operator, transport

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "wire48_gmres.json")
G_TOL = 1e-6
TR_TOL = 1e-6


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def wire():
    from paper_1009_5300_gb300 import build_library
    build_library()
    jn = S.wire48()
    gd = golden()
    idx = [e["index"] for e in gd["energies"]]
    assert np.allclose(jn.energies[idx], [e["E"] for e in gd["energies"]], rtol=0, atol=1e-15)
    return jn, gd, jn.energies[idx]


def _compare(res, gd):
    errs = {"G": 0.0, "T": 0.0, "R": 0.0}
    for e, ent in enumerate(gd["energies"]):
        assert res.n_open[e] == ent["n_open"]
        errs["G"] = max(errs["G"], abs(res.G[e] - ent["G"]))
        rows = np.nonzero(res.energy_index == e)[0]
        assert len(rows) == ent["n_open"]
        n = ent["n_open"]
        for k, ch in zip(rows, ent["channels"]):
            assert res.channel[k] == ch["chan"]
            errs["T"] = max(errs["T"], float(np.max(np.abs(res.T[k, :n] - np.array(ch["T"])))))
            errs["R"] = max(errs["R"], float(np.max(np.abs(res.R[k, :n] - np.array(ch["R"])))))
    return errs


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_conductance_matches_gmres_oracle(wire, precision):
    from paper_1009_5300_gb300 import IOBMSolver
    jn, gd, E = wire
    sol = IOBMSolver.from_junction(jn, precision=precision)
    res = sol.solve(E)
    assert res.converged, res.status
    assert np.all(res.residual <= 1e-8)
    errs = _compare(res, gd)
    print(f"{precision}: max |dG| {errs['G']:.2e} G0, |dT| {errs['T']:.2e}, |dR| {errs['R']:.2e}; "
          f"iterations mean {res.iterations.mean():.1f} max {res.iterations.max()}")
    assert errs["G"] < G_TOL
    assert errs["T"] < TR_TOL
    assert errs["R"] < TR_TOL
    sol.close()


def test_every_wave_has_oracle_residual_below_1e8(wire):
    from paper_1009_5300_gb300 import IOBMSolver
    jn, gd, E = wire
    sol = IOBMSolver.from_junction(jn, precision="mixed")
    res = sol.solve(E)
    assert res.nrhs == sum(e["n_open"] for e in gd["energies"])
    worst = 0.0
    for e, Ee in enumerate(E):
        md = modes.mode_data(jn.nx, jn.ny, jn.hx, jn.hy, jn.hz, jn.nf, float(Ee))
        for k in np.nonzero(res.energy_index == e)[0]:
            m = md.open_modes[int(res.channel[k])]
            psi = sol.solution(int(k)).cpu().numpy()
            b = transport.source_vector(jn, md, m, "L", matrix_free=True)
            r = b - operator.apply_A(jn, float(Ee), md, psi)
            rel = np.linalg.norm(r) / np.linalg.norm(b)
            worst = max(worst, rel)
            assert rel <= 1e-8, (e, int(k), rel)
    print(f"max oracle-operator residual over {res.nrhs} waves: {worst:.2e}")
    sol.close()
