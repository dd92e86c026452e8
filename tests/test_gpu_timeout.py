"""The bounded-wait error path of the bulk-copy stencil, exercised without any GPU
fault: iobm_set_wait_limit makes every CTA of the kernel also wait on an mbarrier
that no copy completes, with a limit of about 0.1 ms of SM clock.  The wait gives
up, the CTA waits for its own copies still in flight and returns, and the call
reports IOBM_E_TIMEOUT; the context stays usable, and with the default limit the
same call gives the same result as before, bit for bit."""
import numpy as np
import pytest
import torch

import iobm_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    from paper_1009_5300_gb300 import IOBMSolver, build_library
    build_library()
    jn = S.small_wire(nx=16, ny=16, nz=40, h=0.45, natom=2, spacing=3.0, depth=0.6, width=1.0,
                      rs=2.0, nf=4, seed=8)
    sol = IOBMSolver.from_junction(jn, precision="mixed", use_precond="eq10")
    yield jn, sol
    sol.close()


def test_operator_wait_gives_up_with_timeout_status(solver):
    from paper_1009_5300_gb300._lib import IOBM_E_TIMEOUT, IOBMError
    jn, sol = solver
    E = jn.e_fermi
    x = torch.from_numpy(np.stack([S.random_field((jn.nz, jn.ny, jn.nx), 40 + i)
                                   for i in range(3)]).astype(np.complex64)).cuda()
    ref = sol.apply(E, x)
    sol.set_wait_limit(200000, inject_stall=True)
    with pytest.raises(IOBMError) as err:
        sol.apply(E, x)
    assert err.value.code == IOBM_E_TIMEOUT
    # a bounded wait that gives up leaves the context usable
    sol.set_wait_limit(0, inject_stall=False)
    torch.cuda.synchronize()
    again = sol.apply(E, x)
    assert torch.equal(again, ref)


def test_preconditioner_wait_gives_up_with_timeout_status(solver):
    from paper_1009_5300_gb300._lib import IOBM_E_TIMEOUT, IOBMError
    jn, sol = solver
    r = torch.from_numpy(S.random_field((1, jn.nz, jn.ny, jn.nx), 77).astype(np.complex64)).cuda()
    ref = sol.apply_precond(r)
    sol.set_wait_limit(200000, inject_stall=True)
    with pytest.raises(IOBMError) as err:
        sol.apply_precond(r)
    assert err.value.code == IOBM_E_TIMEOUT
    sol.set_wait_limit(0, inject_stall=False)
    assert torch.equal(sol.apply_precond(r), ref)


def test_ring_stencil_wait_gives_up_with_timeout_status():
    # the same error path in the plane-ring kernel (stencil variant 4)
    from paper_1009_5300_gb300 import IOBMSolver
    from paper_1009_5300_gb300._lib import IOBM_E_TIMEOUT, IOBMError
    jn = S.small_wire(nx=16, ny=16, nz=40, h=0.45, natom=2, spacing=3.0, depth=0.6, width=1.0,
                      rs=2.0, nf=4, seed=8)
    sol = IOBMSolver.from_junction(jn, precision="mixed", use_precond="eq10")
    sol.set_tiling(16, 4)
    E = jn.e_fermi
    x = torch.from_numpy(np.stack([S.random_field((jn.nz, jn.ny, jn.nx), 60 + i)
                                   for i in range(2)]).astype(np.complex64)).cuda()
    ref = sol.apply(E, x)
    sol.set_wait_limit(200000, inject_stall=True)
    with pytest.raises(IOBMError) as err:
        sol.apply(E, x)
    assert err.value.code == IOBM_E_TIMEOUT
    sol.set_wait_limit(0, inject_stall=False)
    torch.cuda.synchronize()
    assert torch.equal(sol.apply(E, x), ref)
    sol.close()


def test_wait_limit_arguments(solver):
    from paper_1009_5300_gb300._lib import IOBM_E_ARG, IOBMError
    _, sol = solver
    with pytest.raises(IOBMError) as err:
        sol.set_wait_limit(-1)
    assert err.value.code == IOBM_E_ARG
    sol.set_wait_limit(0, inject_stall=False)
