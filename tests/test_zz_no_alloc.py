"""The allocation-free preconditioner entry point against the regular one.

iobm_precond_dots_noalloc serves callers that cannot allocate device memory
(an application pool that owns the GPU, latency-critical loops, stream
capture): its partial sums live in a fixed device array inside the library.
Two calls in a row with different inputs must both agree with
iobm_apply_precond (Eq. 10, FP64) and with the dot products of its result.
This file is collected last so that a stop-at-first-failure run has already
run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

import iobm_synth as S

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point():
    from paper_1009_5300_gb300 import IOBMSolver, build_library
    from paper_1009_5300_gb300 import _lib
    build_library()
    lib = _lib.load()
    jn = S.small_wire(nx=40, ny=12, nz=70, h=0.45, natom=2, spacing=3.0, depth=0.7, width=1.0,
                      rs=2.0, nf=4, seed=3)
    alpha = 1.8
    regular = IOBMSolver.from_junction(jn, precision="fp64", alpha=alpha, use_precond="eq10")
    grid = _lib.Grid(jn.nx, jn.ny, jn.nz, jn.hx, jn.hy, jn.hz, jn.nf)
    stream = torch.cuda.current_stream().cuda_stream
    nrhs = 3
    for call in range(2):
        x = np.stack([S.random_field((jn.nz, jn.ny, jn.nx), 500 + 10 * call + i)
                      for i in range(nrhs)])
        r = torch.from_numpy(x).cuda()
        z = torch.empty_like(r)
        rho = torch.empty((nrhs, 2), dtype=torch.float64, device="cuda")
        rr = torch.empty(nrhs, dtype=torch.float64, device="cuda")
        rc = lib.iobm_precond_dots_noalloc(C.byref(grid), alpha, C.c_void_p(r.data_ptr()),
                                           C.c_void_p(z.data_ptr()), nrhs,
                                           C.c_void_p(rho.data_ptr()), C.c_void_p(rr.data_ptr()),
                                           C.c_void_p(stream))
        assert rc == _lib.IOBM_OK
        torch.cuda.synchronize()
        ref = regular.apply_precond(r)
        scale = ref.abs().max().item()
        assert (z - ref).abs().max().item() < 1e-13 * scale
        rho_ref = (r * ref).reshape(nrhs, -1).sum(dim=1)
        rr_ref = (r.abs() ** 2).reshape(nrhs, -1).sum(dim=1)
        rho_c = torch.complex(rho[:, 0], rho[:, 1])
        assert ((rho_c - rho_ref).abs() / rho_ref.abs()).max().item() < 1e-12
        assert ((rr - rr_ref).abs() / rr_ref).max().item() < 1e-12
    regular.close()


def test_noalloc_rejects_oversized_requests():
    # every RHS needs at least one partial slot, so more RHS than slots is refused
    # on the host before anything touches the device (no buffer is read or written)
    from paper_1009_5300_gb300 import _lib
    lib = _lib.load()
    grid = _lib.Grid(8, 8, 8, 0.3, 0.3, 0.3, 1)
    rc = lib.iobm_precond_dots_noalloc(C.byref(grid), 1.8, C.c_void_p(16), C.c_void_p(16),
                                       (1 << 16) + 1, C.c_void_p(16), C.c_void_p(16), None)
    assert rc == _lib.IOBM_E_UNSUPPORTED


def test_noalloc_rejects_grid_z_overflow_and_aliasing():
    # 65536 RHS of a small grid fit the slot array (one slot each) but not the launch's
    # grid z dimension; and an in-place call (r == z, or overlapping ranges) would let
    # blocks read halo values of r that others already overwrote.  Both are refused
    # on the host before any device access (the pointers are never dereferenced).
    from paper_1009_5300_gb300 import _lib
    lib = _lib.load()
    grid = _lib.Grid(8, 8, 8, 0.3, 0.3, 0.3, 1)
    rc = lib.iobm_precond_dots_noalloc(C.byref(grid), 1.8, C.c_void_p(16), C.c_void_p(1 << 40),
                                       1 << 16, C.c_void_p(16), C.c_void_p(16), None)
    assert rc == _lib.IOBM_E_UNSUPPORTED
    nbytes = 8 * 8 * 8 * 16
    for zoff in (0, 16, nbytes - 16):
        rc = lib.iobm_precond_dots_noalloc(C.byref(grid), 1.8, C.c_void_p(1 << 20),
                                           C.c_void_p((1 << 20) + zoff), 1, C.c_void_p(16),
                                           C.c_void_p(16), None)
        assert rc == _lib.IOBM_E_ARG
