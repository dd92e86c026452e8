"""Preconditioner study (Sec. II preconditioner, Table I trend) on a synthetic junction.

FP64 COCG (so the counts reflect the method, not FP32 rounding) on one junction at
E_F, every open channel: without preconditioning, with Eq. 10 at alpha = 3.0, 2.4,
1.8, and with the lateral-Fourier free propagator.  The paper's Table I (sodium
wires, CPU) reports about 1.3x, 1.7x and 2.2x fewer iterations for alpha = 3.0, 2.4,
1.8 than without preconditioning.  Bar: every variant reaches the oracle's
conductance within 1e-6 G_0, the mean iteration count falls monotonically from no
preconditioning through alpha = 3.0, 2.4, 1.8, and the free propagator needs fewer
iterations than all of them.  The ratios are printed (pytest -s)."""
import numpy as np
import pytest

import iobm_synth as S
from oracle import transport

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1009_5300_gb300 import build_library
    build_library()


def test_iteration_trend():
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.small_wire(nx=16, ny=16, nz=40, h=0.45, natom=3, spacing=3.0, depth=0.7, width=1.0,
                      rs=2.0, kb_kinds=S.SP, nf=4, seed=21)
    E = jn.e_fermi
    G_ref = transport.conductance(jn, E)
    runs = [("none", dict(use_precond="none")),
            ("alpha=3.0", dict(use_precond="eq10", alpha=3.0)),
            ("alpha=2.4", dict(use_precond="eq10", alpha=2.4)),
            ("alpha=1.8", dict(use_precond="eq10", alpha=1.8)),
            ("free propagator", dict(use_precond="fourier"))]
    means = {}
    for name, kw in runs:
        sol = IOBMSolver.from_junction(jn, precision="fp64", **kw)
        res = sol.solve([E])
        assert res.converged, (name, res.status)
        assert abs(res.G[0] - G_ref) < 1e-6, name
        means[name] = float(res.iterations.mean())
        sol.close()
    base = means["none"]
    print("\nmean COCG iterations per channel:",
          {k: round(v, 1) for k, v in means.items()},
          "\nreduction vs none:", {k: round(base / v, 2) for k, v in means.items()})
    seq = [means[k] for k in ("none", "alpha=3.0", "alpha=2.4", "alpha=1.8")]
    assert all(a > b for a, b in zip(seq, seq[1:]))
    assert means["free propagator"] < seq[-1]
