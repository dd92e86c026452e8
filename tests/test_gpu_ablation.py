"""Solver ablation of Sec. III on the GPU: solver (b), the end-plane self-energy of
Eq. 7 applied as the dense N_f N_xy square matrix of each energy (O((N_f N_xy)^2)
per RHS), against solver (c), the same operator through the lateral FFT of Eq. 19,
both without preconditioning.  The two are the same operator up to rounding, so the
operator outputs agree with each other and with the oracle's explicit Eq. 19 sums,
and the solves give the oracle's transmission in the same number of iterations."""
import numpy as np
import pytest
import torch

import iobm_synth as S
from oracle import modes, operator, transport

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1009_5300_gb300 import build_library
    build_library()


def make(nx, ny, nz, nf, kb, seed=3):
    return S.small_wire(nx=nx, ny=ny, nz=nz, h=0.45, natom=1 if nz < 30 else 2, spacing=3.0,
                        depth=0.7, width=1.0, rs=2.0, kb_kinds=S.SP if kb else None, nf=nf,
                        seed=seed)


@pytest.mark.parametrize("nx,ny,nz,nf,kb", [(12, 12, 20, 4, True), (16, 16, 24, 1, False),
                                             (20, 12, 30, 4, True), (6, 5, 11, 2, False),
                                             (48, 48, 12, 4, False)])
def test_dense_sigma_operator_matches_fft_and_oracle(nx, ny, nz, nf, kb):
    # square and non-square planes, ragged 64-row tiles (6 x 5 x 2 = 60 rows), N_f 1, 2, 4
    from paper_1009_5300_gb300 import IOBMSolver
    jn = make(nx, ny, nz, nf, kb)
    E = jn.e_fermi + 0.009
    md = modes.mode_data(nx, ny, jn.hx, jn.hy, jn.hz, nf, E)
    x = np.stack([S.random_field((nz, ny, nx), 300 + i) for i in range(3)])
    ref = np.stack([operator.apply_A(jn, E, md, xi) for xi in x])
    scale = np.max(np.abs(ref))
    xd = torch.from_numpy(x).cuda()
    out = {}
    for form in ("fft", "dense"):
        sol = IOBMSolver.from_junction(jn, precision="fp64", sigma_form=form)
        out[form] = (sol.apply(E, xd).cpu().numpy(),
                     sol.apply(E, xd.to(torch.complex64)).cpu().numpy())
        sol.close()
    assert np.max(np.abs(out["dense"][0] - out["fft"][0])) < 1e-13 * scale
    assert np.max(np.abs(out["dense"][0] - ref)) < 1e-12 * scale
    assert np.max(np.abs(out["dense"][1] - ref)) < 2e-5 * scale


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dense_sigma_solve_matches_oracle(precision):
    # solvers (b) and (c): unpreconditioned COCG with the explicit operator
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.small_wire(nx=12, ny=12, nz=26, h=0.5, natom=2, spacing=3.4, depth=0.7, width=0.9,
                      rs=1.6, kb_kinds=S.SP, nf=4, seed=77)
    E = jn.e_fermi
    ref = transport.solve(jn, E)
    res = {}
    for form in ("dense", "fft"):
        sol = IOBMSolver.from_junction(jn, precision=precision, use_precond="none",
                                       op_form="explicit", sigma_form=form, max_iter_mixed=20000)
        r = sol.solve([E])
        assert r.converged, (form, r.status)
        assert np.all(r.residual <= 1e-8)
        assert abs(r.G[0] - ref.G) < 1e-6, (form, r.G[0], ref.G)
        n = ref.n_open
        for k in range(r.nrhs):
            c = int(r.channel[k])
            assert np.max(np.abs(r.T[k, :n] - ref.T[:, c])) < 1e-6
            assert np.max(np.abs(r.R[k, :n] - ref.R[:, c])) < 1e-6
        res[form] = r
        sol.close()
    it_d = res["dense"].iterations.astype(float)
    it_f = res["fft"].iterations.astype(float)
    print(f"{precision}: iterations dense {it_d.tolist()} fft {it_f.tolist()}")
    # the same operator: the same iteration counts up to rounding, which unpreconditioned
    # COCG amplifies over hundreds of iterations (measured: within 2 % in FP64, 6.3 % with
    # FP32 inner iterations)
    bound = 0.05 if precision == "fp64" else 0.10
    assert np.all(np.abs(it_d - it_f) <= np.maximum(2.0, bound * it_f))


def test_dense_sigma_rejections():
    from paper_1009_5300_gb300 import IOBMSolver, solve_batch
    from paper_1009_5300_gb300._lib import IOBM_E_UNSUPPORTED, IOBMError
    jn = make(12, 12, 20, 4, False)
    sol = IOBMSolver.from_junction(jn, precision="mixed", sigma_form="dense")
    with pytest.raises(IOBMError) as err:
        sol.set_bloch((0.1, 0.0))
    assert err.value.code == IOBM_E_UNSUPPORTED
    with pytest.raises(IOBMError) as err:
        solve_batch([sol], [[jn.e_fermi]])
    assert err.value.code == IOBM_E_UNSUPPORTED
    sol.close()
