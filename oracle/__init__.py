"""FP64 CPU oracle for the multigrid pressure Poisson solve (TEST INFRASTRUCTURE).

A numpy/ctypes front end over ``mg_oracle.c``.  Only the test suite, the
smoke check and the benchmark's CPU-baseline leg use it; the product path
(``paper_2605_30082_gb300``) never imports it, and it imports nothing from the
product.  Every array is float64, C-contiguous, in the layouts documented in
``mg_oracle.c``: cells (nz, ny, nx); x-faces (nz, ny, nx+1); y-faces
(nz, ny+1, nx); z-faces (nz+1, ny, nx).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_OOM = 0, -1, -3, -4, -6
TRILINEAR, CONSTANT = 0, 1

_lib = None
_dp = C.POINTER(C.c_double)


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        i, d, v, ll = C.c_int, C.c_double, C.c_void_p, C.c_longlong
        sig = {
            "or_num_threads": (i, []),
            "or_set_num_threads": (None, [i]),
            "or_mean": (d, [i, i, i, v]),
            "or_norm2": (d, [i, i, i, v]),
            "or_density": (None, [ll, i, v, v, v]),
            "or_faces_from_density": (None, [i, i, i, v, v, v, v]),
            "or_apply": (None, [i, i, i, d, v, v, v, v, v]),
            "or_residual": (None, [i, i, i, d, v, v, v, v, v, v]),
            "or_divergence": (None, [i, i, i, d, v, v, v, v]),
            "or_csf_faces": (None, [i, i, i, d, v, v, v, v, v]),
            "or_rhs": (None, [i, i, i, d, v, v, v, v, v, v, v, v, v, d, v]),
            "or_rbgs_half": (None, [i, i, i, d, v, v, v, v, v, i]),
            "or_rbgs": (None, [i, i, i, d, v, v, v, v, v, i, i]),
            "or_restrict": (None, [i, i, i, v, v]),
            "or_prolong_correct": (None, [i, i, i, v, v, i]),
            "or_coarsen_faces": (None, [i, i, i, v, v, v, v, v, v]),
            "or_assemble_dense": (None, [i, i, i, d, v, v, v, v]),
            "or_coarse_solve": (i, [i, i, i, d, v, v, v, v, v]),
            "or_num_levels": (i, [i, i, i, i]),
            "or_mg_create": (v, [i, i, i, d, v, v, v, i, i, i, i, C.POINTER(i)]),
            "or_mg_free": (None, [v]),
            "or_mg_nlevels": (i, [v]),
            "or_mg_level_dims": (None, [v, i, C.POINTER(i)]),
            "or_mg_level_faces": (None, [v, i, v, v, v]),
            "or_mg_vcycle": (None, [v, v, v]),
            "or_mg_solve": (i, [v, v, v, d, i, i, i, v, i, C.POINTER(i), C.POINTER(d)]),
            "or_mg_fcg": (i, [v, v, v, d, i, v, i, C.POINTER(i), C.POINTER(d), v, v, i]),
            "or_project": (None, [i, i, i, d, v, v, v, v, v, v, v, d, v, v, v]),
            "or_density_grads": (None, [i, i, i, v, v, v, v, v, i, v, v]),
            "or_adjoint_grads": (None, [i, i, i, d, v, v, v, v, v, v, v, v, d, v, v, v, C.POINTER(d)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous, "oracle arrays: float64, C-contiguous"
    return a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dims(cells):
    nz, ny, nx = cells.shape
    return nx, ny, nz


def face_shapes(nx, ny, nz):
    return (nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


def mean(x):
    x = _f64(x)
    return lib().or_mean(*_dims(x), _p(x))


def density(fracs, rho_phase):
    """Eq. (5): rho = sum_i rho_i f_i, the last phase filling 1 - sum of the given fractions."""
    fracs = [_f64(f) for f in fracs]
    rho_phase = _f64(rho_phase)
    assert rho_phase.size == len(fracs) + 1
    out = np.empty_like(fracs[0])
    ptrs = (C.c_void_p * len(fracs))(*[f.ctypes.data for f in fracs])
    lib().or_density(out.size, len(fracs), C.cast(ptrs, C.c_void_p), _p(rho_phase), _p(out))
    return out


def faces_from_density(rho):
    rho = _f64(rho)
    nx, ny, nz = _dims(rho)
    bx, by, bz = (np.empty(s) for s in face_shapes(nx, ny, nz))
    lib().or_faces_from_density(nx, ny, nz, _p(rho), _p(bx), _p(by), _p(bz))
    return bx, by, bz


def apply(faces, p, h):
    p = _f64(p)
    bx, by, bz = (_f64(f) for f in faces)
    out = np.empty_like(p)
    lib().or_apply(*_dims(p), h, _p(bx), _p(by), _p(bz), _p(p), _p(out))
    return out


def residual(faces, b, p, h):
    p, b = _f64(p), _f64(b)
    bx, by, bz = (_f64(f) for f in faces)
    out = np.empty_like(p)
    lib().or_residual(*_dims(p), h, _p(bx), _p(by), _p(bz), _p(b), _p(p), _p(out))
    return out


def divergence(u, h):
    ux, uy, uz = (_f64(a) for a in u)
    nz, ny, nxp = ux.shape
    out = np.empty((nz, ny, nxp - 1))
    lib().or_divergence(nxp - 1, ny, nz, h, _p(ux), _p(uy), _p(uz), _p(out))
    return out


def csf_faces(f, kappa, h):
    f, kappa = _f64(f), _f64(kappa)
    nx, ny, nz = _dims(f)
    cx, cy, cz = (np.empty(s) for s in face_shapes(nx, ny, nz))
    lib().or_csf_faces(nx, ny, nz, h, _p(f), _p(kappa), _p(cx), _p(cy), _p(cz))
    return cx, cy, cz


def rhs(u, faces, h, csf=None, sigma=0.0):
    """b = D u + sigma D(beta * csf)."""
    ux, uy, uz = (_f64(a) for a in u)
    bx, by, bz = (_f64(a) for a in faces)
    nz, ny, nxp = ux.shape
    out = np.empty((nz, ny, nxp - 1))
    cs = [None, None, None] if csf is None else [_f64(a) for a in csf]
    lib().or_rhs(nxp - 1, ny, nz, h, _p(ux), _p(uy), _p(uz), _p(bx), _p(by), _p(bz),
                 _p(cs[0]), _p(cs[1]), _p(cs[2]), float(sigma), _p(out))
    return out


def rbgs_half(faces, b, p, h, colour):
    """In place on a copy: one half sweep of colour (0 red, 1 black); returns the new p."""
    p = _f64(p).copy()
    b = _f64(b)
    bx, by, bz = (_f64(f) for f in faces)
    lib().or_rbgs_half(*_dims(p), h, _p(bx), _p(by), _p(bz), _p(b), _p(p), int(colour))
    return p


def rbgs(faces, b, p, h, sweeps, order=0):
    p = _f64(p).copy()
    b = _f64(b)
    bx, by, bz = (_f64(f) for f in faces)
    lib().or_rbgs(*_dims(p), h, _p(bx), _p(by), _p(bz), _p(b), _p(p), int(sweeps), int(order))
    return p


def restrict(r):
    r = _f64(r)
    nx, ny, nz = _dims(r)
    out = np.empty((nz // 2, ny // 2, nx // 2))
    lib().or_restrict(nx, ny, nz, _p(r), _p(out))
    return out


def prolong_correct(ec, e, kind=TRILINEAR):
    ec = _f64(ec)
    e = _f64(e).copy()
    lib().or_prolong_correct(*_dims(ec), _p(ec), _p(e), int(kind))
    return e


def coarsen_faces(faces):
    bx, by, bz = (_f64(f) for f in faces)
    nz, ny, nxp = bx.shape
    nx = nxp - 1
    cx, cy, cz = (np.empty(s) for s in face_shapes(nx // 2, ny // 2, nz // 2))
    lib().or_coarsen_faces(nx, ny, nz, _p(bx), _p(by), _p(bz), _p(cx), _p(cy), _p(cz))
    return cx, cy, cz


def assemble_dense(faces, h):
    bx, by, bz = (_f64(f) for f in faces)
    nz, ny, nxp = bx.shape
    n = (nxp - 1) * ny * nz
    A = np.empty((n, n))
    lib().or_assemble_dense(nxp - 1, ny, nz, h, _p(bx), _p(by), _p(bz), _p(A))
    return A


def coarse_solve(faces, r, h):
    r = _f64(r)
    bx, by, bz = (_f64(f) for f in faces)
    e = np.empty_like(r)
    st = lib().or_coarse_solve(*_dims(r), h, _p(bx), _p(by), _p(bz), _p(r), _p(e))
    if st != OK:
        raise ValueError(f"or_coarse_solve failed: {st}")
    return e


def num_levels(nx, ny, nz, coarsest):
    return lib().or_num_levels(nx, ny, nz, coarsest)


def adjoint_grads(faces, lam, p, h, csf=None, sigma=0.0):
    """Face gradients (walls 0) and dL/dsigma for L = sum w p, given lambda = A^+(w - mean w)."""
    lam, p = _f64(lam), _f64(p)
    bx, by, bz = (_f64(f) for f in faces)
    nx, ny, nz = _dims(p)
    gx, gy, gz = (np.empty(s) for s in face_shapes(nx, ny, nz))
    cs = [None, None, None] if csf is None else [_f64(a) for a in csf]
    ds = C.c_double(0.0)
    lib().or_adjoint_grads(nx, ny, nz, h, _p(bx), _p(by), _p(bz), _p(lam), _p(p),
                           _p(cs[0]), _p(cs[1]), _p(cs[2]), float(sigma),
                           _p(gx), _p(gy), _p(gz), C.byref(ds))
    return (gx, gy, gz), ds.value


def project(u, faces, p, h, csf=None, sigma=0.0):
    """The corrected face velocities u + beta (G p + sigma csf) (copies; walls unchanged)."""
    ux, uy, uz = (_f64(a).copy() for a in u)
    bx, by, bz = (_f64(f) for f in faces)
    p = _f64(p)
    nx, ny, nz = _dims(p)
    cs = [None, None, None] if csf is None else [_f64(a) for a in csf]
    lib().or_project(nx, ny, nz, float(h), _p(bx), _p(by), _p(bz), _p(p), _p(cs[0]), _p(cs[1]), _p(cs[2]),
                     float(sigma), _p(ux), _p(uy), _p(uz))
    return ux, uy, uz


def density_grads(rho, grads, rho_phase=None):
    """dL/drho from the face gradients dL/dbeta; with rho_phase (nfrac + 1 densities) also the
    fraction gradients dL/df_q.  Returns drho or (drho, [dfrac_q])."""
    rho = _f64(rho)
    gx, gy, gz = (_f64(g) for g in grads)
    nx, ny, nz = _dims(rho)
    drho = np.empty_like(rho)
    if rho_phase is None:
        lib().or_density_grads(nx, ny, nz, _p(rho), _p(gx), _p(gy), _p(gz), _p(drho), 0, None, None)
        return drho
    ph = np.ascontiguousarray(rho_phase, dtype=np.float64)
    nfrac = len(ph) - 1
    dfrac = np.empty((nfrac,) + rho.shape)
    lib().or_density_grads(nx, ny, nz, _p(rho), _p(gx), _p(gy), _p(gz), _p(drho), nfrac, _p(ph), _p(dfrac))
    return drho, list(dfrac)


class Multigrid:
    """The oracle's V-cycle hierarchy for one set of fine-grid face coefficients."""

    def __init__(self, faces, h, coarsest=4, pre=2, post=2, prolong=TRILINEAR):
        self._faces = tuple(_f64(f) for f in faces)
        bx, by, bz = self._faces
        nz, ny, nxp = bx.shape
        self.nx, self.ny, self.nz, self.h = nxp - 1, ny, nz, float(h)
        st = C.c_int(0)
        self._h = lib().or_mg_create(self.nx, self.ny, self.nz, self.h, _p(bx), _p(by), _p(bz),
                                     int(coarsest), int(pre), int(post), int(prolong), C.byref(st))
        if not self._h:
            raise ValueError(f"or_mg_create failed ({st.value})")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_mg_free(self._h)
            self._h = None

    @property
    def nlevels(self):
        return lib().or_mg_nlevels(self._h)

    def level_dims(self, l):
        d = (C.c_int * 3)()
        lib().or_mg_level_dims(self._h, l, d)
        return tuple(d)  # (nx, ny, nz)

    def level_faces(self, l):
        nx, ny, nz = self.level_dims(l)
        out = [np.empty(s) for s in face_shapes(nx, ny, nz)]
        lib().or_mg_level_faces(self._h, l, *(_p(a) for a in out))
        return tuple(out)

    def vcycle(self, b, x):
        b = _f64(b)
        x = _f64(x).copy()
        lib().or_mg_vcycle(self._h, _p(b), _p(x))
        return x

    def solve(self, b, rtol=1e-10, max_cycles=200, p0=None, hist_len=256, stop_on_stall=False):
        """Return (p, status, cycles, relres, history)."""
        b = _f64(b)
        warm = p0 is not None
        p = _f64(p0).copy() if warm else np.zeros_like(b)
        hist = np.zeros(hist_len)
        nc = C.c_int(0)
        rr = C.c_double(0.0)
        st = lib().or_mg_solve(self._h, _p(b), _p(p), float(rtol), int(max_cycles), int(warm),
                               int(stop_on_stall), _p(hist), hist_len, C.byref(nc), C.byref(rr))
        return p, st, nc.value, rr.value, hist[: min(nc.value + 1, hist_len)].copy()

    def fcg(self, b, rtol=1e-10, max_it=200, hist_len=256, record=0):
        """Flexible CG preconditioned by one V-cycle (see or_mg_fcg).

        Returns (p, status, iterations, true relres, history[, (r_k, z_k) for k < record])."""
        b = _f64(b)
        p = np.zeros_like(b)
        hist = np.zeros(hist_len)
        nit = C.c_int(0)
        rr = C.c_double(0.0)
        rec_r = np.zeros((record,) + b.shape) if record else None
        rec_z = np.zeros((record,) + b.shape) if record else None
        st = lib().or_mg_fcg(self._h, _p(b), _p(p), float(rtol), int(max_it), _p(hist), hist_len,
                             C.byref(nit), C.byref(rr), _p(rec_r) if record else None,
                             _p(rec_z) if record else None, int(record))
        out = (p, st, nit.value, rr.value, hist[: min(nit.value + 1, hist_len)].copy())
        return out + ((rec_r, rec_z),) if record else out

    def solve_exact(self, b, max_cycles=400):
        """The zero-mean discrete solution p* = A^+(b - mean b): V-cycles to stagnation.

        Cycles until the relative residual is <= 1e-15 or has stopped falling
        for two cycles.  Returns (p, relres, cycles).
        """
        p, st, nc, rr, _ = self.solve(b, rtol=1e-15, max_cycles=max_cycles, stop_on_stall=True)
        if st != OK:
            raise RuntimeError(f"oracle solve to stagnation failed: status {st}, relres {rr}")
        return p, rr, nc
