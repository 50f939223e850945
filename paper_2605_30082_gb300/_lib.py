"""ctypes binding of libmgpoisson.so (the C ABI in include/mg.h).

Argument marshalling only: every function checks the torch tensors it is given
(device, dtype, contiguity, shape), passes their device pointers to the C
entry point of the same name and returns the C status code.  Nothing here
computes; there is no CPU path.  Loading fails loudly when the library has not
been built.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmgpoisson.so")

MG_OK, MG_ERR_ARG, MG_ERR_DENSITY, MG_ERR_NOT_CONVERGED = 0, -1, -2, -3
MG_ERR_DIVERGED, MG_ERR_CUDA, MG_ERR_OOM, MG_ERR_STATE = -4, -5, -6, -7
MG_FP64, MG_MIXED, MG_MIXED_DF = 0, 1, 2
MG_PROLONG_TRILINEAR, MG_PROLONG_CONSTANT = 0, 1
MG_METHOD_VCYCLE, MG_METHOD_FCG = 0, 1
MG_F64, MG_F32 = 0, 1
MG_MAX_LEVELS, MG_MAX_COARSE, MG_HIST_LEN = 24, 1024, 256
MG_NOALLOC_MAX_CELLS = 512
MG_INJECT_FUSED_WAIT, MG_INJECT_DIVERGE = 1, 2
(MG_PROF_SMOOTH, MG_PROF_RESID_RESTRICT, MG_PROF_PROLONG, MG_PROF_COARSE,
 MG_PROF_FINE_RESIDUAL, MG_PROF_UPDATE, MG_PROF_ADJOINT_GRAD, MG_PROF_PROJECT,
 MG_PROF_DENSITY_GRAD, MG_PROF_COARSE_LEVELS, MG_PROF_SETUP, MG_PROF_RHS, MG_PROF_DENSITY,
 MG_PROF_NCLASS) = range(14)

ERROR_NAMES = {
    MG_OK: "MG_OK", MG_ERR_ARG: "MG_ERR_ARG", MG_ERR_DENSITY: "MG_ERR_DENSITY",
    MG_ERR_NOT_CONVERGED: "MG_ERR_NOT_CONVERGED", MG_ERR_DIVERGED: "MG_ERR_DIVERGED",
    MG_ERR_CUDA: "MG_ERR_CUDA", MG_ERR_OOM: "MG_ERR_OOM", MG_ERR_STATE: "MG_ERR_STATE",
}


class mg_opts(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double),
                ("precision", C.c_int), ("pre", C.c_int), ("post", C.c_int),
                ("coarsest", C.c_int), ("prolong", C.c_int), ("rtol", C.c_double),
                ("max_cycles", C.c_int), ("warm_start", C.c_int), ("inner_cycles", C.c_int),
                ("method", C.c_int), ("fused_sweeps", C.c_int)]


class mg_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("outer", C.c_int), ("relres", C.c_double),
                ("relres_hist", C.c_double * MG_HIST_LEN), ("ms", C.c_double)]

    def history(self):
        """relres after each outer iteration (one per V-cycle unless inner_cycles > 1)."""
        return list(self.relres_hist[: min(self.outer + 1, MG_HIST_LEN)])


MG_DD_MAX_RANKS = 64


class mg_dd_plan(C.Structure):
    _fields_ = [("ranks", C.c_int), ("levels", C.c_int), ("switch_level", C.c_int),
                ("nx", C.c_int * MG_MAX_LEVELS), ("ny", C.c_int * MG_MAX_LEVELS), ("nz", C.c_int * MG_MAX_LEVELS),
                ("planes", C.c_int * MG_MAX_LEVELS)]


_lib = None

# every exported symbol with (restype, argtypes)
_i, _d, _v, _ll = C.c_int, C.c_double, C.c_void_p, C.c_longlong
SIGNATURES = {
    "mg_default_opts": (None, [C.POINTER(mg_opts)]),
    "mg_create": (_i, [C.POINTER(mg_opts), _v, C.POINTER(_v)]),
    "mg_destroy": (_i, [_v]),
    "mg_last_error": (C.c_char_p, [_v]),
    "mg_num_levels": (_i, [_v]),
    "mg_level_dims": (_i, [_v, _i, C.POINTER(_i)]),
    "mg_density_from_fractions": (_i, [_v, _i, C.POINTER(_v), C.POINTER(_d), _v]),
    "mg_set_density": (_i, [_v, _v]),
    "mg_set_face_coeffs": (_i, [_v, _v, _v, _v]),
    "mg_get_level_faces": (_i, [_v, _i, _v, _v, _v]),
    "mg_csf_faces": (_i, [_v, _v, _v, _v, _v, _v]),
    "mg_rhs": (_i, [_v, _v, _v, _v, _v, _v, _v, _v, _d, _v]),
    "mg_solve": (_i, [_v, _v, _v, C.POINTER(mg_stats)]),
    "mg_adjoint": (_i, [_v, _v, _v, _v, _v, _v, _v, _v, _v, _v, _d, C.POINTER(_d), C.POINTER(mg_stats)]),
    "mg_project": (_i, [_v, _v, _v, _v, _v, _d, _v, _v, _v, _v, _v, _v]),
    "mg_density_grads": (_i, [_v, _v, _v, _v, _v, _v, _i, C.POINTER(_d), C.POINTER(_v)]),
    "mg_apply": (_i, [_v, _i, _i, _v, _v]),
    "mg_smooth": (_i, [_v, _i, _i, _v, _v, _i, _i]),
    "mg_presmooth_restrict": (_i, [_v, _i, _i, _v, _v, _i, _i, _v]),
    "mg_prolong_postsmooth": (_i, [_v, _i, _i, _v, _v, _v, _i]),
    "mg_residual": (_i, [_v, _i, _i, _v, _v, _v, C.POINTER(_d)]),
    "mg_residual_restrict": (_i, [_v, _i, _i, _v, _v, _v]),
    "mg_prolong_correct": (_i, [_v, _i, _i, _v, _v]),
    "mg_coarse_solve": (_i, [_v, _i, _v, _v]),
    "mg_profile": (_i, [_v, _i]),
    "mg_profile_read": (_i, [_v, _i, C.POINTER(_ll), C.POINTER(_d)]),
    "mg_kernel_launches": (_ll, []),
    "mg_dense_solve_noalloc": (_i, [_i, _i, _i, _d, _v, _v, _v, _v, _v, _v]),
    "mg_fp64_fma_rate": (_i, [_v, _v, _i, _i, C.POINTER(_d), C.POINTER(_d)]),
    "mg_debug_inject": (_i, [_v, _i]),
    "mg_dd_make_plan": (_i, [_i, _i, _i, _i, _i, _i, C.POINTER(mg_dd_plan)]),
    "mg_dd_create": (_i, [C.POINTER(mg_opts), _i, _i, _v, C.POINTER(_v)]),
    "mg_dd_destroy": (_i, [_v]),
    "mg_dd_last_error": (C.c_char_p, [_v]),
    "mg_dd_get_plan": (_i, [_v, C.POINTER(mg_dd_plan)]),
    "mg_dd_traffic": (_i, [_v, C.POINTER(_ll), C.POINTER(_ll)]),
    "mg_dd_set_density": (_i, [_v, _v]),
    "mg_dd_vcycle": (_i, [_v, _v, _v]),
    "mg_dd_solve": (_i, [_v, _v, _v, C.POINTER(mg_stats)]),
}


def lib():
    """The loaded CUDA library.  Raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ---- tensor checks ----------------------------------------------------------------

def _dev(t, dtype=torch.float64, shape=None, name="array"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor (the library has no CPU path)")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


def cell_shape(dims):
    nx, ny, nz = dims
    return (nz, ny, nx)


def face_shapes(dims):
    nx, ny, nz = dims
    return (nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)


def _dtype_code(t):
    if t.dtype == torch.float64:
        return MG_F64
    if t.dtype == torch.float32:
        return MG_F32
    raise ValueError("component arrays must be float64 or float32")


# ---- entry points (same names as the C ABI) ------------------------------------------

def mg_default_opts():
    o = mg_opts()
    lib().mg_default_opts(C.byref(o))
    return o


def mg_create(opts: mg_opts, stream=None):
    """Returns (status, handle).  stream: torch.cuda.Stream or None (current stream)."""
    if stream is None:
        stream = torch.cuda.current_stream()
    h = C.c_void_p()
    st = lib().mg_create(C.byref(opts), C.c_void_p(stream.cuda_stream), C.byref(h))
    return st, h


def mg_destroy(h):
    return lib().mg_destroy(h)


def mg_last_error(h) -> str:
    s = lib().mg_last_error(h)
    return s.decode() if s else ""


def mg_num_levels(h):
    return lib().mg_num_levels(h)


def mg_level_dims(h, level):
    d = (C.c_int * 3)()
    st = lib().mg_level_dims(h, level, d)
    return st, (d[0], d[1], d[2])


def mg_density_from_fractions(h, fracs, rho_phase, rho, dims):
    ptrs = (C.c_void_p * len(fracs))(*[_dev(f, shape=cell_shape(dims), name="fraction").value for f in fracs])
    rp = (C.c_double * len(rho_phase))(*[float(r) for r in rho_phase])
    return lib().mg_density_from_fractions(h, len(fracs), ptrs, rp, _dev(rho, shape=cell_shape(dims), name="rho"))


def mg_set_density(h, rho, dims):
    return lib().mg_set_density(h, _dev(rho, shape=cell_shape(dims), name="rho"))


def mg_set_face_coeffs(h, bx, by, bz, dims):
    fs = face_shapes(dims)
    return lib().mg_set_face_coeffs(h, _dev(bx, shape=fs[0], name="bx"), _dev(by, shape=fs[1], name="by"),
                                    _dev(bz, shape=fs[2], name="bz"))


def mg_get_level_faces(h, level, bx, by, bz, dims):
    fs = face_shapes(dims)
    return lib().mg_get_level_faces(h, level, _dev(bx, shape=fs[0], name="bx"), _dev(by, shape=fs[1], name="by"),
                                    _dev(bz, shape=fs[2], name="bz"))


def mg_csf_faces(h, f, kappa, cx, cy, cz, dims):
    fs = face_shapes(dims)
    cs = cell_shape(dims)
    return lib().mg_csf_faces(h, _dev(f, shape=cs, name="f"), _dev(kappa, shape=cs, name="kappa"),
                              _dev(cx, shape=fs[0], name="csfx"), _dev(cy, shape=fs[1], name="csfy"),
                              _dev(cz, shape=fs[2], name="csfz"))


def mg_rhs(h, b0, u, csf, sigma, b, dims):
    """b = b0 + D u + sigma D(beta csf); b0, u (3 faces), csf (3 faces) may be None."""
    fs = face_shapes(dims)
    cs = cell_shape(dims)
    ux = uy = uz = cx = cy = cz = None
    if u is not None:
        ux, uy, uz = (_dev(a, shape=s, name="u") for a, s in zip(u, fs))
    if csf is not None:
        cx, cy, cz = (_dev(a, shape=s, name="csf") for a, s in zip(csf, fs))
    return lib().mg_rhs(h, _dev(b0, shape=cs, name="b0"), ux, uy, uz, cx, cy, cz, float(sigma),
                        _dev(b, shape=cs, name="b"))


def mg_solve(h, b, p, dims, stats: mg_stats | None = None):
    cs = cell_shape(dims)
    return lib().mg_solve(h, _dev(b, shape=cs, name="b"), _dev(p, shape=cs, name="p"),
                          C.byref(stats) if stats is not None else None)


def mg_adjoint(h, w, p, lam, grads, csf, sigma, dims, stats: mg_stats | None = None):
    """grads: (gbx, gby, gbz) float32 face tensors or None; returns (status, dL/dsigma)."""
    cs = cell_shape(dims)
    fs = face_shapes(dims)
    g = [None, None, None] if grads is None else [_dev(a, torch.float32, s, "grad") for a, s in zip(grads, fs)]
    c = [None, None, None] if csf is None else [_dev(a, shape=s, name="csf") for a, s in zip(csf, fs)]
    ds = C.c_double(0.0)
    st = lib().mg_adjoint(h, _dev(w, shape=cs, name="w"), _dev(p, shape=cs, name="p"),
                          _dev(lam, shape=cs, name="lam"), g[0], g[1], g[2], c[0], c[1], c[2],
                          float(sigma), C.byref(ds), C.byref(stats) if stats is not None else None)
    return st, ds.value


def mg_project(h, p, csf, sigma, u, out, dims):
    """u, out: (x, y, z) float64 face tensors (out may be u itself: in place); csf may be None."""
    fs = face_shapes(dims)
    c = [None, None, None] if csf is None else [_dev(a, shape=s, name="csf") for a, s in zip(csf, fs)]
    ui = [_dev(a, shape=s, name="u") for a, s in zip(u, fs)]
    uo = [_dev(a, shape=s, name="out") for a, s in zip(out, fs)]
    return lib().mg_project(h, _dev(p, shape=cell_shape(dims), name="p"), c[0], c[1], c[2], float(sigma),
                            *ui, *uo)


def mg_density_grads(h, rho, grads, drho, dims, rho_phase=None, dfrac=None):
    """grads: (gbx, gby, gbz) float32 face tensors; drho float64 cells; dfrac: nfrac float64 cell
    tensors (with rho_phase, nfrac + 1 densities) or None."""
    fs = face_shapes(dims)
    cs = cell_shape(dims)
    g = [_dev(a, torch.float32, s, "grad") for a, s in zip(grads, fs)]
    nfrac, rp, ptrs = 0, None, None
    if dfrac is not None:
        nfrac = len(dfrac)
        if rho_phase is None or len(rho_phase) != nfrac + 1:
            raise ValueError("rho_phase needs len(dfrac) + 1 densities")
        rp = (C.c_double * (nfrac + 1))(*[float(r) for r in rho_phase])
        ptrs = (C.c_void_p * nfrac)(*[_dev(a, shape=cs, name="dfrac").value for a in dfrac])
    return lib().mg_density_grads(h, _dev(rho, shape=cs, name="rho"), g[0], g[1], g[2],
                                  _dev(drho, shape=cs, name="drho"), nfrac, rp, ptrs)


def _lvl_shape(h, level):
    st, d = mg_level_dims(h, level)
    if st != MG_OK:
        raise ValueError(f"level {level} out of range")
    return cell_shape(d)


def mg_apply(h, level, x, y):
    dt = _dtype_code(x)
    s = _lvl_shape(h, level)
    return lib().mg_apply(h, level, dt, _dev(x, x.dtype, s, "x"), _dev(y, x.dtype, s, "y"))


def mg_smooth(h, level, x, b, sweeps, order=0):
    dt = _dtype_code(x)
    s = _lvl_shape(h, level)
    return lib().mg_smooth(h, level, dt, _dev(x, x.dtype, s, "x"), _dev(b, x.dtype, s, "b"), int(sweeps), int(order))


def mg_presmooth_restrict(h, level, x, b, sweeps, bc, x_is_zero=False):
    dt = _dtype_code(x)
    s = _lvl_shape(h, level)
    sc = _lvl_shape(h, level + 1)
    return lib().mg_presmooth_restrict(h, level, dt, _dev(x, x.dtype, s, "x"), _dev(b, x.dtype, s, "b"),
                                       int(sweeps), int(bool(x_is_zero)), _dev(bc, x.dtype, sc, "bc"))


def mg_prolong_postsmooth(h, level, ec, x, b, sweeps):
    dt = _dtype_code(x)
    s = _lvl_shape(h, level)
    sc = _lvl_shape(h, level + 1)
    return lib().mg_prolong_postsmooth(h, level, dt, _dev(ec, x.dtype, sc, "ec"), _dev(x, x.dtype, s, "x"),
                                       _dev(b, x.dtype, s, "b"), int(sweeps))


def mg_residual(h, level, x, b, r, want_norm=False):
    dt = _dtype_code(x)
    s = _lvl_shape(h, level)
    nrm = C.c_double(0.0)
    st = lib().mg_residual(h, level, dt, _dev(x, x.dtype, s, "x"), _dev(b, x.dtype, s, "b"),
                           _dev(r, x.dtype, s, "r"), C.byref(nrm) if want_norm else None)
    return st, nrm.value


def mg_residual_restrict(h, level, x, b, bc):
    dt = _dtype_code(x)
    s = _lvl_shape(h, level)
    sc = _lvl_shape(h, level + 1)
    return lib().mg_residual_restrict(h, level, dt, _dev(x, x.dtype, s, "x"), _dev(b, x.dtype, s, "b"),
                                      _dev(bc, x.dtype, sc, "bc"))


def mg_prolong_correct(h, level, ec, x):
    dt = _dtype_code(x)
    s = _lvl_shape(h, level)
    sc = _lvl_shape(h, level + 1)
    return lib().mg_prolong_correct(h, level, dt, _dev(ec, x.dtype, sc, "ec"), _dev(x, x.dtype, s, "x"))


def mg_coarse_solve(h, r, e):
    dt = _dtype_code(r)
    s = _lvl_shape(h, mg_num_levels(h) - 1)
    return lib().mg_coarse_solve(h, dt, _dev(r, r.dtype, s, "r"), _dev(e, r.dtype, s, "e"))


def mg_profile(h, enable):
    return lib().mg_profile(h, int(enable))


def mg_profile_read(h, cls):
    n = C.c_longlong(0)
    ms = C.c_double(0.0)
    st = lib().mg_profile_read(h, int(cls), C.byref(n), C.byref(ms))
    return st, n.value, ms.value


def mg_kernel_launches():
    return lib().mg_kernel_launches()


def mg_debug_inject(h, faults):
    """Arm one-shot test faults (MG_INJECT_* bits) on the handle; returns the status."""
    return lib().mg_debug_inject(h, int(faults))


def mg_dense_solve_noalloc(dims, h, bx, by, bz, r, e, stream=None):
    """Allocation-free exact small-grid solve (see include/mg.h); returns the status."""
    if stream is None:
        stream = torch.cuda.current_stream()
    fs = face_shapes(dims)
    cs = cell_shape(dims)
    nx, ny, nz = dims
    return lib().mg_dense_solve_noalloc(nx, ny, nz, float(h), _dev(bx, shape=fs[0], name="bx"),
                                        _dev(by, shape=fs[1], name="by"), _dev(bz, shape=fs[2], name="bz"),
                                        _dev(r, shape=cs, name="r"), _dev(e, shape=cs, name="e"),
                                        C.c_void_p(stream.cuda_stream))


def mg_fp64_fma_rate(sink, iters, stream=None):
    """FP64 FMA rate of the current device: one timed launch of len(sink) blocks (sink: float64
    CUDA tensor, overwritten).  Returns (status, TFLOP/s, ms)."""
    if stream is None:
        stream = torch.cuda.current_stream()
    tf = C.c_double(0.0)
    ms = C.c_double(0.0)
    st = lib().mg_fp64_fma_rate(C.c_void_p(stream.cuda_stream), _dev(sink, name="sink"), int(sink.numel()),
                                int(iters), C.byref(tf), C.byref(ms))
    return st, tf.value, ms.value


# ---- domain decomposition (z slabs held on one GPU) ----------------------------------------

def mg_dd_make_plan(dims, coarsest, ranks, max_decomposed=0):
    """Host only: returns (status, mg_dd_plan)."""
    nx, ny, nz = dims
    pl = mg_dd_plan()
    st = lib().mg_dd_make_plan(int(nx), int(ny), int(nz), int(coarsest), int(ranks), int(max_decomposed),
                               C.byref(pl))
    return st, pl


def mg_dd_create(opts: mg_opts, ranks, max_decomposed=0, stream=None):
    """Returns (status, dd handle)."""
    if stream is None:
        stream = torch.cuda.current_stream()
    h = C.c_void_p()
    st = lib().mg_dd_create(C.byref(opts), int(ranks), int(max_decomposed), C.c_void_p(stream.cuda_stream),
                            C.byref(h))
    return st, h


def mg_dd_destroy(dd):
    return lib().mg_dd_destroy(dd)


def mg_dd_last_error(dd) -> str:
    s = lib().mg_dd_last_error(dd)
    return s.decode() if s else ""


def mg_dd_get_plan(dd):
    pl = mg_dd_plan()
    st = lib().mg_dd_get_plan(dd, C.byref(pl))
    return st, pl


def mg_dd_traffic(dd):
    ex, by = C.c_longlong(0), C.c_longlong(0)
    st = lib().mg_dd_traffic(dd, C.byref(ex), C.byref(by))
    return st, ex.value, by.value


def mg_dd_set_density(dd, rho, dims):
    return lib().mg_dd_set_density(dd, _dev(rho, shape=cell_shape(dims), name="rho"))


def mg_dd_vcycle(dd, b, x, dims):
    cs = cell_shape(dims)
    return lib().mg_dd_vcycle(dd, _dev(b, shape=cs, name="b"), _dev(x, shape=cs, name="x"))


def mg_dd_solve(dd, b, p, dims, stats: mg_stats | None = None):
    cs = cell_shape(dims)
    return lib().mg_dd_solve(dd, _dev(b, shape=cs, name="b"), _dev(p, shape=cs, name="p"),
                             C.byref(stats) if stats is not None else None)
