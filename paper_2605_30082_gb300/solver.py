"""User-facing wrapper over the C ABI: a Solver object and an autograd Function.

``Solver`` owns one ``mg_handle`` (all device memory allocated at creation)
and raises :class:`MgError` for every non-zero status.  ``PoissonSolve`` is a
``torch.autograd.Function`` whose forward is ``mg_rhs`` + ``mg_solve`` and
whose backward is ``mg_adjoint`` (a second multigrid solve plus one fused
gradient kernel); autograd saves only the inputs and the solution p, no
V-cycle state.
"""
from __future__ import annotations

import torch

from . import _lib as L


class MgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{L.ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Solver:
    """Multigrid pressure Poisson solver for one grid on the current CUDA device.

    Parameters mirror ``mg_opts``: dims = (nx, ny, nz), h, precision ('fp64',
    'mixed' or 'mixed_df'), pre/post sweeps, coarsest, prolong ('trilinear' or
    'constant'), rtol, max_cycles, warm_start, inner_cycles (mixed modes: FP32 V-cycles, or
    flexible-CG iterations, per outer FP64 residual; 0: adaptive V-cycle count), method ('vcycle' or 'fcg': conjugate
    gradients preconditioned by one V-cycle), fused_sweeps (True: finest-level fused red-black
    sweeps where the layout allows, bitwise the same results as the default half sweeps).
    """

    def __init__(self, dims, h=None, precision="mixed", pre=2, post=2, coarsest=None,
                 prolong="trilinear", rtol=1e-10, max_cycles=200, warm_start=False, stream=None,
                 inner_cycles=1, method="vcycle", fused_sweeps=False):
        nx, ny, nz = (int(v) for v in dims)
        o = L.mg_default_opts()
        o.nx, o.ny, o.nz = nx, ny, nz
        o.h = float(h if h is not None else 1.0 / max(nx, ny, nz))
        o.precision = {"fp64": L.MG_FP64, "mixed": L.MG_MIXED, "mixed_df": L.MG_MIXED_DF}[precision]
        o.pre, o.post = int(pre), int(post)
        o.coarsest = int(coarsest if coarsest is not None else (4 if precision == "fp64" else 8))
        o.prolong = {"trilinear": L.MG_PROLONG_TRILINEAR, "constant": L.MG_PROLONG_CONSTANT}[prolong]
        o.rtol = float(rtol)
        o.max_cycles = int(max_cycles)
        o.warm_start = int(bool(warm_start))
        o.inner_cycles = int(inner_cycles)
        o.method = {"vcycle": L.MG_METHOD_VCYCLE, "fcg": L.MG_METHOD_FCG}[method]
        o.fused_sweeps = int(bool(fused_sweeps))
        self.opts = o
        self.dims = (nx, ny, nz)
        self.h = o.h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        st, self._h = L.mg_create(o, self.stream)
        if st != L.MG_OK:
            raise MgError(st, "mg_create failed (bad options, or out of device memory)")
        self.coef_version = None  # identity of the coefficients currently loaded
        self.last_stats = None

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            L.mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != L.MG_OK and st not in allow:
            raise MgError(st, L.mg_last_error(self._h))
        return st

    # -- shapes --
    @property
    def cell_shape(self):
        return L.cell_shape(self.dims)

    @property
    def face_shapes(self):
        return L.face_shapes(self.dims)

    @property
    def num_levels(self):
        return L.mg_num_levels(self._h)

    def level_dims(self, level):
        st, d = L.mg_level_dims(self._h, level)
        self._check(st)
        return d

    def empty_cells(self, dtype=torch.float64):
        return torch.empty(self.cell_shape, dtype=dtype, device=self.device)

    # -- operator set-up --
    def density_from_fractions(self, fracs, rho_phase, out=None):
        out = self.empty_cells() if out is None else out
        self._check(L.mg_density_from_fractions(self._h, list(fracs), list(rho_phase), out, self.dims))
        return out

    def set_density(self, rho):
        self._check(L.mg_set_density(self._h, rho, self.dims))
        self.coef_version = ("rho", rho.data_ptr(), rho._version)

    def set_face_coeffs(self, bx, by, bz):
        self._check(L.mg_set_face_coeffs(self._h, bx, by, bz, self.dims))
        self.coef_version = ("faces", bx.data_ptr(), by.data_ptr(), bz.data_ptr(),
                             bx._version, by._version, bz._version)

    def level_faces(self, level):
        d = self.level_dims(level)
        out = [torch.empty(s, dtype=torch.float64, device=self.device) for s in L.face_shapes(d)]
        self._check(L.mg_get_level_faces(self._h, level, *out, d))
        return tuple(out)

    # -- right-hand side --
    def csf_faces(self, f, kappa):
        out = [torch.empty(s, dtype=torch.float64, device=self.device) for s in self.face_shapes]
        self._check(L.mg_csf_faces(self._h, f, kappa, *out, self.dims))
        return tuple(out)

    def rhs(self, u=None, csf=None, sigma=0.0, b0=None, out=None):
        """b = b0 + D u + sigma D(beta csf) on the device (each term optional)."""
        out = self.empty_cells() if out is None else out
        self._check(L.mg_rhs(self._h, b0, u, csf, sigma, out, self.dims))
        return out

    # -- solves --
    def solve(self, b, p=None, raise_on_nonconvergence=True):
        p = torch.zeros(self.cell_shape, dtype=torch.float64, device=self.device) if p is None else p
        stats = L.mg_stats()
        st = L.mg_solve(self._h, b, p, self.dims, stats)
        self.last_stats = stats
        self._check(st, allow=() if raise_on_nonconvergence else (L.MG_ERR_NOT_CONVERGED,))
        return p

    def adjoint(self, w, p, csf=None, sigma=0.0, grads=True, lam=None):
        """Returns (lam, (gbx, gby, gbz) or None, dL/dsigma)."""
        lam = self.empty_cells() if lam is None else lam
        g = None
        if grads:
            g = tuple(torch.empty(s, dtype=torch.float32, device=self.device) for s in self.face_shapes)
        stats = L.mg_stats()
        st, ds = L.mg_adjoint(self._h, w, p, lam, g, csf, sigma, self.dims, stats)
        self.last_stats = stats
        self._check(st)
        return lam, g, ds

    # -- either side of the solve --
    def project(self, p, u, csf=None, sigma=0.0, out=None):
        """Velocity correction of the projection step: u + beta (G p + sigma csf) on the interior
        faces, u on the walls (u: three float64 face tensors).  Written into `out` (three face
        tensors), or into u itself when out is None.  Returns the corrected velocities."""
        out = tuple(u) if out is None else tuple(out)
        self._check(L.mg_project(self._h, p, csf, sigma, u, out, self.dims))
        return out

    def density_grads(self, rho, grads, rho_phase=None, out=None):
        """dL/drho from the float32 face gradients of `adjoint`; with rho_phase (nfrac + 1 phase
        densities) also dL/df_q.  Returns drho, or (drho, [dL/df_q]); `out` gives those arrays."""
        if out is not None:
            drho, dfrac = (out, None) if rho_phase is None else (out[0], list(out[1]))
        else:
            drho = self.empty_cells()
            dfrac = None if rho_phase is None else [self.empty_cells() for _ in range(len(rho_phase) - 1)]
        self._check(L.mg_density_grads(self._h, rho, grads, drho, self.dims, rho_phase, dfrac))
        return drho if dfrac is None else (drho, dfrac)

    # -- instrumentation --
    def profile(self, enable=True):
        self._check(L.mg_profile(self._h, enable))

    def profile_read(self, cls):
        st, n, ms = L.mg_profile_read(self._h, cls)
        self._check(st)
        return n, ms


class PoissonSolve(torch.autograd.Function):
    """p = A(beta)^+ (b - mean b), b = b_u + sigma D(beta csf) (csf optional).

    forward(solver, b_u, bx, by, bz, sigma=None, csf=None) -> p
    Gradients: dL/db_u (float64 cells), dL/dbx, dL/dby, dL/dbz (float32 faces, walls 0),
    dL/dsigma (float64 scalar tensor, when sigma is a tensor and csf is given).
    The backward re-loads the face coefficients into the solver when another
    operator was set in between (recomputation instead of stored state).
    """

    @staticmethod
    def forward(ctx, solver: Solver, b_u, bx, by, bz, sigma=None, csf=None):
        solver.set_face_coeffs(bx, by, bz)
        sig = float(sigma) if sigma is not None else 0.0
        b = b_u if csf is None else solver.rhs(csf=csf, sigma=sig, b0=b_u)
        p = solver.solve(b)
        ctx.solver = solver
        ctx.sig = sig
        ctx.has_sigma = sigma is not None and isinstance(sigma, torch.Tensor)
        ctx.csf = csf
        ctx.save_for_backward(bx, by, bz, p)
        ctx.version = solver.coef_version
        return p

    @staticmethod
    def backward(ctx, grad_p):
        solver = ctx.solver
        bx, by, bz, p = ctx.saved_tensors
        if solver.coef_version != ctx.version:
            solver.set_face_coeffs(bx, by, bz)
        w = grad_p.contiguous()
        lam, g, ds = solver.adjoint(w, p, csf=ctx.csf, sigma=ctx.sig, grads=True)
        dsig = None
        if ctx.has_sigma:
            dsig = torch.tensor(ds, dtype=torch.float64, device=p.device)
        return None, lam, g[0], g[1], g[2], dsig, None



class PoissonSolveFractions(torch.autograd.Function):
    """p = A(beta(rho))^+ (b - mean b), rho = Eq. (5) of the phase fractions, b = b_u + sigma
    D(beta csf) (csf optional), with gradients back to the fractions.

    forward(solver, b_u, rho_phase, sigma, csf, *fracs) -> p
    rho_phase: nfrac + 1 phase densities (floats); fracs: nfrac float64 cell tensors.
    Gradients: dL/db_u, dL/dsigma (when sigma is a tensor and csf is given) and dL/df_q, the
    last through the density only (csf is held fixed).  The backward is mg_adjoint followed by
    mg_density_grads (which forms dL/drho and every dL/df_q in one pass); the density is
    recomputed from the saved fractions when another operator was set in between.
    """

    @staticmethod
    def forward(ctx, solver: Solver, b_u, rho_phase, sigma, csf, *fracs):
        rho = solver.density_from_fractions(list(fracs), list(rho_phase))
        solver.set_density(rho)
        sig = float(sigma) if sigma is not None else 0.0
        b = b_u if csf is None else solver.rhs(csf=csf, sigma=sig, b0=b_u)
        p = solver.solve(b)
        ctx.solver = solver
        ctx.sig = sig
        ctx.has_sigma = sigma is not None and isinstance(sigma, torch.Tensor)
        ctx.csf = csf
        ctx.rho_phase = tuple(float(r) for r in rho_phase)
        ctx.save_for_backward(rho, p)
        ctx.version = solver.coef_version
        return p

    @staticmethod
    def backward(ctx, grad_p):
        solver = ctx.solver
        rho, p = ctx.saved_tensors
        if solver.coef_version != ctx.version:
            solver.set_density(rho)
        lam, g, ds = solver.adjoint(grad_p.contiguous(), p, csf=ctx.csf, sigma=ctx.sig, grads=True)
        _, dfrac = solver.density_grads(rho, g, ctx.rho_phase)
        dsig = None
        if ctx.has_sigma:
            dsig = torch.tensor(ds, dtype=torch.float64, device=p.device)
        return (None, lam, None, dsig, None) + tuple(dfrac)
