"""Python front end of the IOBM C ABI (same names, argument marshalling only).

PyTorch provides device memory (the solve workspace, operand tensors) and the
CUDA stream; every step of the transport solve runs in libiobm.so.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import check


@dataclasses.dataclass
class SolveResult:
    energies: np.ndarray          # [nE]
    G: np.ndarray                 # [nE] conductance (G_0), summed over solved incident channels
    n_open: np.ndarray            # [nE]
    T: np.ndarray                 # [nrhs][max_open]
    R: np.ndarray                 # [nrhs][max_open]
    energy_index: np.ndarray      # [nrhs]
    channel: np.ndarray           # [nrhs]
    status: np.ndarray            # [nrhs]
    iterations: np.ndarray        # [nrhs]
    replacements: np.ndarray      # [nrhs]
    residual: np.ndarray          # [nrhs] FP64 ||b - A psi|| / ||b||
    device_ms: float              # device time of the iteration phase
    launches: int                 # kernel launches of the iteration phase
    iterations_total: int

    @property
    def nrhs(self) -> int:
        return len(self.status)

    @property
    def converged(self) -> bool:
        return bool(np.all(self.status == _lib.IOBM_OK))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def default_options(**kw) -> _lib.Options:
    lib = _lib.load()
    o = _lib.Options()
    lib.iobm_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": _lib.IOBM_FP64, "mixed": _lib.IOBM_MIXED}[v]
        if k == "use_precond" and isinstance(v, str):
            v = {"none": _lib.IOBM_PRECOND_NONE, "eq10": _lib.IOBM_PRECOND_EQ10,
                 "fourier": _lib.IOBM_PRECOND_FOURIER,
                 "eq10_fourier": _lib.IOBM_PRECOND_EQ10_FOURIER}[v]
        if k == "op_form" and isinstance(v, str):
            v = {"auto": _lib.IOBM_OP_AUTO, "explicit": _lib.IOBM_OP_EXPLICIT}[v]
        if k == "sigma_form" and isinstance(v, str):
            v = {"fft": _lib.IOBM_SIGMA_FFT, "dense": _lib.IOBM_SIGMA_DENSE}[v]
        setattr(o, k, v)
    return o


def channels_host(nx, ny, hx, hy, hz, nf, E, max_out=None, want_sigma=False, kappa=(0.0, 0.0)):
    """Host-side channel tables of the library (no GPU needed): iobm_channels_host_bloch
    (at lateral Bloch vector kappa; iobm_channels_host at kappa = 0)."""
    lib = _lib.load()
    g = _lib.Grid(nx, ny, 2 * nf + 1, hx, hy, hz, nf)
    n = C.c_int(0)
    kx, ky = float(kappa[0]), float(kappa[1])
    if max_out is None:
        check(lib.iobm_channels_host_bloch(C.byref(g), kx, ky, E, C.byref(n), 0, None, None, None,
                                           None, None, None))
        max_out = n.value
    nu = np.zeros((max(max_out, 1), 2), np.int32)
    vel = np.zeros(max(max_out, 1))
    lam = np.zeros((max(max_out, 1), 2))
    bt = np.zeros((max(max_out, 1), nf, 2))
    mrow = np.zeros((max(max_out, 1), nf, 2))
    sig = np.zeros((ny, nx, nf, nf, 2)) if want_sigma else None
    check(lib.iobm_channels_host_bloch(C.byref(g), kx, ky, E, C.byref(n), max_out, _ptr(nu),
                                       _ptr(vel), _ptr(lam), _ptr(bt), _ptr(mrow),
                                       _ptr(sig) if want_sigma else None))
    k = n.value
    out = dict(n_open=k, nu=nu[:k], vel=vel[:k], lam=lam[:k, 0] + 1j * lam[:k, 1],
               btilde=bt[:k, :, 0] + 1j * bt[:k, :, 1], mrow=mrow[:k, :, 0] + 1j * mrow[:k, :, 1])
    if want_sigma:
        out["sigma"] = sig[..., 0] + 1j * sig[..., 1]
    return out


class IOBMSolver:
    """One junction: iobm_create / iobm_solve / iobm_transmission / iobm_grad_V."""

    def __init__(self, nx, ny, nz, hx, hy, hz, nf, V, rs, projectors=None, options=None,
                 device="cuda", **option_kw):
        self.lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("IOBMSolver needs a CUDA device")
        self.device = torch.device(device)
        self.shape = (nz, ny, nx)
        self.nf = nf
        self.grid = _lib.Grid(nx, ny, nz, hx, hy, hz, nf)
        self.opts = options if options is not None else default_options(**option_kw)
        V = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(nz, ny, nx))
        self._keep = []
        if projectors is not None:
            row_ptr, idx, val, coupling = projectors
            row_ptr = np.ascontiguousarray(row_ptr, np.int64)
            idx = np.ascontiguousarray(idx, np.int32)
            val = np.ascontiguousarray(val, np.float64)
            coupling = np.ascontiguousarray(coupling, np.float64)
            self._keep += [row_ptr, idx, val, coupling]
            proj = _lib.Projectors(len(coupling), row_ptr.ctypes.data_as(C.POINTER(C.c_int64)),
                                   idx.ctypes.data_as(C.POINTER(C.c_int32)),
                                   val.ctypes.data_as(C.POINTER(C.c_double)),
                                   coupling.ctypes.data_as(C.POINTER(C.c_double)))
            pproj = C.byref(proj)
        else:
            pproj = None
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            rc = self.lib.iobm_create(C.byref(self.grid), _ptr(V), pproj, float(rs),
                                      C.byref(self.opts), C.c_void_p(stream), C.byref(h))
        if rc != _lib.IOBM_OK:
            msg = self.lib.iobm_last_error(h).decode() if h.value else ""
            if h.value:
                self.lib.iobm_destroy(h)
            raise _lib.IOBMError(rc, self.lib.iobm_status_string(rc).decode() + ": " + msg)
        self.h = h
        self._ws = None
        self.kappa = (0.0, 0.0)

    @classmethod
    def from_junction(cls, jn, **kw):
        proj = jn.projector_csr() if jn.projectors else None
        return cls(jn.nx, jn.ny, jn.nz, jn.hx, jn.hy, jn.hz, jn.nf, jn.V, jn.rs, projectors=proj,
                   **kw)

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            torch.cuda.synchronize(self.device)
            self.lib.iobm_destroy(self.h)
            self.h = C.c_void_p()
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- queries -------------------------------------------------------
    @property
    def fermi_energy(self) -> float:
        return self.lib.iobm_fermi_energy(self.h)

    def open_channels(self, E: float):
        n = C.c_int(0)
        check(self.lib.iobm_open_channels(self.h, float(E), C.byref(n), 0, None, None), self.h)
        nu = np.zeros((max(n.value, 1), 2), np.int32)
        vel = np.zeros(max(n.value, 1))
        check(self.lib.iobm_open_channels(self.h, float(E), C.byref(n), n.value, _ptr(nu),
                                          _ptr(vel)), self.h)
        return nu[: n.value], vel[: n.value]

    def workspace_size(self, nrhs: int) -> int:
        b = C.c_size_t(0)
        check(self.lib.iobm_workspace_size(self.h, int(nrhs), C.byref(b)), self.h)
        return b.value

    def _ensure_workspace(self, nrhs: int):
        need = self.workspace_size(nrhs)
        if self._ws is None or self._ws.numel() < need:
            self._ws = None
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        check(self.lib.iobm_set_workspace(self.h, C.c_void_p(self._ws.data_ptr()),
                                          self._ws.numel()), self.h)

    def _count_rhs(self, E: np.ndarray, ch) -> int:
        n = C.c_int(0)
        check(self.lib.iobm_solve_rhs_count(self.h, _ptr(E), len(E),
                                            _ptr(ch) if ch is not None else None,
                                            0 if ch is None else len(ch), C.byref(n)), self.h)
        return n.value

    # ---- solves --------------------------------------------------------
    def solve(self, energies: Sequence[float], channels: Optional[Sequence[int]] = None,
              side: int = 0) -> SolveResult:
        E = np.ascontiguousarray(np.atleast_1d(np.asarray(energies, np.float64)))
        ch = None if channels is None else np.ascontiguousarray(channels, np.int32)
        nrhs = self._count_rhs(E, ch)
        self._ensure_workspace(max(nrhs, 1))
        with torch.cuda.device(self.device):
            check(self.lib.iobm_solve(self.h, _ptr(E), len(E), _ptr(ch) if ch is not None else None,
                                      0 if ch is None else len(ch), int(side)), self.h)
        return self.transmission(E)

    def release_workspace(self):
        """Detach and free the torch-allocated workspace; the results of the last solve
        are no longer readable afterwards (read them first)."""
        check(self.lib.iobm_set_workspace(self.h, None, 0), self.h)
        self._ws = None

    def autotune(self, nrhs: int):
        """Pick the stencil tiling for nrhs RHS on this grid (iobm_autotune); (zchunk, variant)."""
        self._ensure_workspace(max(int(nrhs), 1))
        z = C.c_int(0)
        v = C.c_int(0)
        with torch.cuda.device(self.device):
            check(self.lib.iobm_autotune(self.h, int(nrhs), C.byref(z), C.byref(v)), self.h)
        return z.value, v.value

    def set_tiling(self, zchunk: int, variant: int = 0):
        check(self.lib.iobm_set_tiling(self.h, int(zchunk), int(variant)), self.h)

    def time_operator(self, nrhs: int, reps: int = 20) -> float:
        """Average ms of one fused COCG operator launch on nrhs RHS, all active
        (iobm_time_operator; overwrites the workspace)."""
        self._ensure_workspace(max(int(nrhs), 1))
        ms = C.c_double(0)
        with torch.cuda.device(self.device):
            check(self.lib.iobm_time_operator(self.h, int(nrhs), int(reps), C.byref(ms)), self.h)
        return ms.value

    def set_bloch(self, kappa):
        """Lateral Bloch vector (kappa_x, kappa_y) of the later solves (iobm_set_bloch).
        At kappa != 0 a solve also returns the -kappa problem: energy slots nE + e."""
        kx, ky = float(kappa[0]), float(kappa[1])
        check(self.lib.iobm_set_bloch(self.h, kx, ky), self.h)
        self.kappa = (kx, ky)

    def transmission(self, E) -> SolveResult:
        nrhs = self.lib.iobm_num_rhs(self.h)
        if self.kappa != (0.0, 0.0):
            E = np.concatenate([np.asarray(E), np.asarray(E)])   # +kappa slots, then -kappa
        nE = len(E)
        n_open = np.zeros(nE, np.int32)
        G = np.zeros(nE)
        max_open = max(1, self.lib.iobm_max_open(self.h))
        T = np.zeros((max(nrhs, 1), max_open))
        R = np.zeros((max(nrhs, 1), max_open))
        reps = (_lib.Report * max(nrhs, 1))()
        check(self.lib.iobm_transmission(self.h, _ptr(T), _ptr(R), max_open, _ptr(G), _ptr(n_open),
                                         reps), self.h)
        ms = C.c_double(0)
        la = C.c_longlong(0)
        it = C.c_longlong(0)
        self.lib.iobm_last_solve_stats(self.h, C.byref(ms), C.byref(la), C.byref(it))
        rep = list(reps)[:nrhs]
        return SolveResult(
            energies=np.asarray(E), G=G, n_open=n_open, T=T[:nrhs], R=R[:nrhs],
            energy_index=np.array([r.energy_index for r in rep], np.int32),
            channel=np.array([r.channel for r in rep], np.int32),
            status=np.array([r.status for r in rep], np.int32),
            iterations=np.array([r.iterations for r in rep], np.int32),
            replacements=np.array([r.replacements for r in rep], np.int32),
            residual=np.array([r.residual for r in rep]),
            device_ms=ms.value, launches=la.value, iterations_total=it.value)

    def eigenchannels(self, e: int = 0) -> np.ndarray:
        """Eigenchannel transmissions (eigenvalues of T^dagger T, descending) of energy
        index e of the last solve, which must have solved every open channel."""
        n = C.c_int(0)
        check(self.lib.iobm_eigenchannels(self.h, int(e), None, 0, C.byref(n)), self.h)
        tau = np.zeros(max(n.value, 1))
        check(self.lib.iobm_eigenchannels(self.h, int(e), _ptr(tau), n.value, C.byref(n)), self.h)
        return tau[: n.value]

    def solution(self, rhs: int) -> torch.Tensor:
        out = torch.empty(self.shape, dtype=torch.complex128, device=self.device)
        check(self.lib.iobm_solution(self.h, int(rhs), C.c_void_p(out.data_ptr()), 1), self.h)
        return out

    def grad_V(self, E: float):
        """(dG/dV as a [nz][ny][nx] float64 CUDA tensor, G) at energy E."""
        n = self.open_channels(E)[0].shape[0]
        # forward and adjoint RHS (real profiles; at kappa != 0 one Bi-CG pair per channel)
        self._ensure_workspace(max(2 * n, 1))
        g = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        G = C.c_double(0)
        with torch.cuda.device(self.device):
            check(self.lib.iobm_grad_V(self.h, float(E), C.c_void_p(g.data_ptr()), 1, C.byref(G)),
                  self.h)
        return g, G.value

    def set_potential(self, V):
        if isinstance(V, torch.Tensor):
            Vt = V.detach().to(device=self.device, dtype=torch.float64).contiguous()
            torch.cuda.current_stream(self.device).synchronize()
            check(self.lib.iobm_set_potential(self.h, C.c_void_p(Vt.data_ptr()), 1), self.h)
        else:
            Vn = np.ascontiguousarray(np.asarray(V, np.float64).reshape(self.shape))
            check(self.lib.iobm_set_potential(self.h, _ptr(Vn), 0), self.h)

    def set_wait_limit(self, cycles: int = 0, inject_stall: bool = False):
        """Bounded-wait limit of the bulk-copy kernels (0: default, about one second), and
        optionally an extra wait on a barrier no copy completes (iobm_set_wait_limit)."""
        check(self.lib.iobm_set_wait_limit(self.h, int(cycles), 1 if inject_stall else 0), self.h)

    PROFILE_STAGES = {"operator": 1, "update_fft": 2, "zsweep": 3, "ifft": 4}

    def profile(self, enable=True):
        """Time one kernel of every captured COCG iteration with CUDA events: True or
        "operator" (the fused stencil, or the direction/operator update of the implicit
        form), "update_fft" (x, r update + forward plane FFTs), "zsweep", "ifft"
        (inverse FFTs + dot partials); False stops."""
        stage = self.PROFILE_STAGES[enable] if isinstance(enable, str) else (1 if enable else 0)
        check(self.lib.iobm_profile(self.h, stage), self.h)

    def kernel_stats(self):
        """(total ms, launches) of the kernel timed since profile(...)."""
        ms = C.c_double(0)
        n = C.c_longlong(0)
        check(self.lib.iobm_kernel_stats(self.h, C.byref(ms), C.byref(n)), self.h)
        return ms.value, n.value

    # ---- operator access -------------------------------------------------
    def apply(self, E: float, x: torch.Tensor, double_float: bool = False) -> torch.Tensor:
        """y = (E - H_T - H~) x for x [nrhs][nz][ny][nx] complex64/complex128 on the device.
        double_float: complex128 data with the stencil in double-float arithmetic (the
        arithmetic of the mixed solver's FP64 residual)."""
        x = x.contiguous()
        elem = _lib.IOBM_ELEM_C64 if x.dtype == torch.complex128 else _lib.IOBM_ELEM_C32
        if double_float:
            if x.dtype != torch.complex128:
                raise TypeError("double_float needs complex128 data")
            elem = _lib.IOBM_ELEM_C64_DF
        if x.dtype not in (torch.complex64, torch.complex128):
            raise TypeError("x must be complex64 or complex128")
        nrhs = x.numel() // int(np.prod(self.shape))
        y = torch.empty_like(x)
        with torch.cuda.device(self.device):
            check(self.lib.iobm_apply(self.h, float(E), elem, C.c_void_p(x.data_ptr()),
                                      C.c_void_p(y.data_ptr()), nrhs), self.h)
        return y

    def apply_precond(self, x: torch.Tensor, E: float = 0.0) -> torch.Tensor:
        """y = P x (Eq. 10, or the lateral-Fourier free propagator at energy E)."""
        x = x.contiguous()
        elem = _lib.IOBM_ELEM_C64 if x.dtype == torch.complex128 else _lib.IOBM_ELEM_C32
        nrhs = x.numel() // int(np.prod(self.shape))
        y = torch.empty_like(x)
        with torch.cuda.device(self.device):
            check(self.lib.iobm_apply_precond(self.h, float(E), elem, C.c_void_p(x.data_ptr()),
                                              C.c_void_p(y.data_ptr()), nrhs), self.h)
        return y


def solve_batch(solvers: Sequence["IOBMSolver"], energies: Sequence[Sequence[float]], side: int = 0,
                autotune: bool = False):
    """Solve several junctions together (iobm_solve_batch): one CUDA graph launch runs
    every junction's COCG iterations concurrently.  energies[j] are the energies of
    solvers[j]; every open incident channel is solved.  With autotune, each junction's
    stencil tiling is picked for its RHS count first.  Returns one SolveResult per solver."""
    lib = _lib.load()
    n = len(solvers)
    if n == 0:
        return []
    Es = [np.ascontiguousarray(np.atleast_1d(np.asarray(e, np.float64))) for e in energies]
    if len(Es) != n:
        raise ValueError("one energy list per solver")
    for sol, E in zip(solvers, Es):
        nrhs = sol._count_rhs(E, None)
        sol._ensure_workspace(max(nrhs, 1))
        if autotune and nrhs > 0:
            sol.autotune(nrhs)
    handles = (C.c_void_p * n)(*[sol.h.value for sol in solvers])
    eptrs = (C.c_void_p * n)(*[E.ctypes.data for E in Es])
    ne = (C.c_int * n)(*[len(E) for E in Es])
    with torch.cuda.device(solvers[0].device):
        code = lib.iobm_solve_batch(n, handles, eptrs, ne, int(side))
    if code != _lib.IOBM_OK:
        failing = next((sol.h for sol in solvers if lib.iobm_last_error(sol.h)), solvers[0].h)
        check(code, failing)
    return [sol.transmission(E) for sol, E in zip(solvers, Es)]
