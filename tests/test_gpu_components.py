"""Step-by-step parity of the CUDA kernels with the FP64 oracle (through the C ABI).

Grids span several thread blocks with ragged tails in every direction; each
multigrid level of each grid is checked.  FP64 kernels must agree with the
oracle to rounding (1e-13 relative L2); FP32 kernels, run on the FP32 copies
of the coefficients, to 2e-6 (a few units of FP32 rounding, amplified by at
most the stencil's 7 terms).
"""
import numpy as np
import pytest
import torch

import dropfilm as D
import oracle as O
from paper_2605_30082_gb300 import MG_ERR_DENSITY, MG_ERR_STATE, MgError, Solver
from paper_2605_30082_gb300 import _lib as L

from _helpers import RHO_PHASE, dev, dropfilm_case, host, random_rho, rel

pytestmark = pytest.mark.gpu

DIMS = [(72, 40, 24), (40, 24, 56), (32, 32, 32)]
# rows of >= 128 four-cell vectors per colour take the z-marching half sweep: 64 and 48 vectors
# per row (a half-idle second block), z-chunks of 16 with a ragged last chunk, odd coarse dims
WIDE = [(256, 12, 20), (384, 4, 36)]
TOL = {torch.float64: 1e-13, torch.float32: 2e-6}


def make(dims, precision, seed=3, prolong="trilinear", coarsest=4, coeffs="rho"):
    """A solver and the oracle hierarchy on the same random density.

    coeffs="rho" loads the operator with mg_set_density (the finest FP32 level then
    sweeps with s = 1/rho per cell); "faces" loads the same coefficients with
    mg_set_face_coeffs (the finest FP32 level sweeps with the three face arrays)."""
    nx, ny, nz = dims
    h = 1.0 / 64
    s = Solver(dims, h=h, precision=precision, coarsest=coarsest, prolong=prolong)
    rho = random_rho(dims, seed)
    if coeffs == "rho":
        s.set_density(dev(rho))
    else:
        s.set_face_coeffs(*(dev(f) for f in O.faces_from_density(rho)))
    M = O.Multigrid(O.faces_from_density(rho), h, coarsest=coarsest,
                    prolong=O.TRILINEAR if prolong == "trilinear" else O.CONSTANT)
    return s, M


def rnd(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_levels_and_faces_match_oracle(dims, precision):
    """The device forms beta = (s_L + s_R)/2 from s = 1/rho (a Newton reciprocal from an FP32
    seed), the oracle (rho_L + rho_R)/(2 rho_L rho_R): both within 2 FP64 roundings of the same
    number, so every face agrees to 1e-15 relative."""
    s, M = make(dims, precision)
    assert s.num_levels == M.nlevels
    for l in range(M.nlevels):
        assert s.level_dims(l) == M.level_dims(l)
        for g, o in zip(s.level_faces(l), M.level_faces(l)):
            g = host(g)
            assert rel(g, o) < 1e-15
            nz = o != 0
            assert np.array_equal(g != 0, nz)
            assert np.max(np.abs(g[nz] - o[nz]) / o[nz]) <= 1e-15


@pytest.mark.parametrize("dims", [(72, 40, 24), (40, 24, 56), (36, 20, 12)])
def test_density_and_face_loading_give_bitwise_the_same_fp64_solve(dims):
    """mg_set_density forms the finest faces from s = 1/rho; mg_set_face_coeffs takes them as
    given.  Loaded with the same faces, the two FP64 hierarchies (coarsened faces, diagonals and
    their reciprocals, the dense coarse inverse) must be the same bit for bit, and so must the
    FP64 solves."""
    nx, ny, nz = dims
    h = 1.0 / 64
    a = Solver(dims, h=h, precision="fp64", coarsest=4, rtol=1e-10)
    a.set_density(dev(random_rho(dims, 17)))
    b_ = Solver(dims, h=h, precision="fp64", coarsest=4, rtol=1e-10)
    b_.set_face_coeffs(*a.level_faces(0))
    rhs = dev(rnd((nz, ny, nx), 5))
    pa, pb = a.solve(rhs), b_.solve(rhs)
    assert a.last_stats.cycles == b_.last_stats.cycles
    assert torch.equal(pa, pb)
    a.close()
    b_.close()


def test_density_from_fractions_and_face_round_trip():
    n = 24
    fd, ff = D.fractions_ramp(D.scaled_geometry(n))
    s = Solver((n, n, n), precision="fp64")
    rho = s.density_from_fractions([fd.cuda(), ff.cuda()], RHO_PHASE)
    rho_o = O.density([fd.numpy(), ff.numpy()], RHO_PHASE)
    assert np.abs(host(rho) - rho_o).max() <= 1e-15 * rho_o.max()
    faces = O.faces_from_density(rho_o)
    s.set_face_coeffs(*(dev(f) for f in faces))
    for g, o in zip(s.level_faces(0), faces):
        assert rel(host(g), o) == 0.0
    # wall entries are ignored on input and written back as zero
    bad = [f.copy() for f in faces]
    bad[0][:, :, 0] = -5.0
    bad[2][-1] = np.nan
    s.set_face_coeffs(*(dev(f) for f in bad))
    for g, o in zip(s.level_faces(0), faces):
        assert rel(host(g), o) == 0.0


def test_csf_faces_and_rhs_match_oracle():
    c = dropfilm_case(32)
    h = c["h"]
    s = Solver((32, 32, 32), precision="fp64")
    s.set_density(dev(c["rho"]))
    kappa = D.curvature_band(c["fd"], c["geom"])
    csf = s.csf_faces(c["fd"].cuda(), kappa.cuda())
    csf_o = O.csf_faces(c["fd"].numpy(), kappa.numpy(), h)
    for g, o in zip(csf, csf_o):
        assert rel(host(g), o) < 1e-14
    u = tuple(a.cuda() for a in c["u"])
    b = s.rhs(u=u)
    assert rel(host(b), c["b"]) < 1e-14
    b0 = rnd((32, 32, 32), 1)
    b2 = s.rhs(u=u, csf=csf, sigma=0.03, b0=dev(b0))
    want = b0 + O.rhs([a.numpy() for a in c["u"]], c["faces"], h, csf=csf_o, sigma=0.03)
    assert rel(host(b2), want) < 1e-14


@pytest.mark.parametrize("dims", DIMS + WIDE)
@pytest.mark.parametrize("dtype,coeffs", [(torch.float64, "rho"), (torch.float32, "rho"), (torch.float32, "faces")])
def test_apply_smooth_residual_match_oracle(dims, dtype, coeffs):
    s, M = make(dims, "fp64" if dtype == torch.float64 else "mixed", coeffs=coeffs)
    tol = TOL[dtype]
    for l in range(M.nlevels):
        nx, ny, nz = M.level_dims(l)
        H = s.h * 2**l
        faces = M.level_faces(l)
        if dtype == torch.float32:  # the oracle sees the same FP32-rounded coefficients
            faces = tuple(f.astype(np.float32).astype(np.float64) for f in faces)
        x = rnd((nz, ny, nx), 10 + l).astype(np.float32 if dtype == torch.float32 else np.float64)
        b = rnd((nz, ny, nx), 20 + l).astype(x.dtype)
        xg, bg = dev(x, dtype), dev(b, dtype)
        y = torch.empty_like(xg)
        assert L.mg_apply(s._h, l, xg, y) == 0
        assert rel(host(y), O.apply(faces, x, H)) < tol
        r = torch.empty_like(xg)
        st, nrm = L.mg_residual(s._h, l, xg, bg, r, want_norm=True)
        r_o = O.residual(faces, b, x, H)
        assert st == 0 and rel(host(r), r_o) < tol
        assert abs(nrm - np.linalg.norm(r_o)) <= 10 * tol * np.linalg.norm(r_o)
        for sweeps, order in ((1, 0), (1, 1), (2, 0)):
            xs = xg.clone()
            assert L.mg_smooth(s._h, l, xs, bg, sweeps, order) == 0
            assert rel(host(xs), O.rbgs(faces, b, x, H, sweeps, order)) < tol
        # after one pre sweep (red then black) the black rows are solved exactly
        xs = xg.clone()
        L.mg_smooth(s._h, l, xs, bg, 1, 0)
        k, j, i = np.meshgrid(range(nz), range(ny), range(nx), indexing="ij")
        black = (i + j + k) % 2 == 1
        rb = O.residual(faces, b, host(xs), H)
        assert np.abs(rb[black]).max() <= 50 * tol * np.abs(O.apply(faces, host(xs), H)).max()


def test_staged_half_sweep_matches_oracle_ragged_rows():
    """Grids of at least 4 x 152 x 8 z-marching blocks sweep their s-form regular half sweeps
    with each plane's loads staged in shared memory (the 512^3 workload's kernel).  320 cells
    per row give 40 four-cell vectors per colour: two rows per 64-thread block and a second
    block with 8 of its 32 lanes active per row; 192 x 416 rows and planes make 4992 blocks."""
    dims = (320, 192, 416)
    s, M = make(dims, "mixed")
    nx, ny, nz = dims
    faces = tuple(f.astype(np.float32).astype(np.float64) for f in M.level_faces(0))
    x = rnd((nz, ny, nx), 31).astype(np.float32)
    b = rnd((nz, ny, nx), 32).astype(np.float32)
    xg, bg = dev(x, torch.float32), dev(b, torch.float32)
    for sweeps, order in ((1, 0), (1, 1), (2, 0)):
        xs = xg.clone()
        assert L.mg_smooth(s._h, 0, xs, bg, sweeps, order) == 0
        assert rel(host(xs), O.rbgs(faces, b, x, s.h, sweeps, order)) < TOL[torch.float32]


def test_staged_face_form_half_sweep_matches_oracle_ragged_rows():
    """Face-form regular half sweeps (the levels below the finest, and a finest level loaded
    from face coefficients) are staged in shared memory where the grid gives at least
    4 x 152 x 11 blocks of 4 planes.  320 cells per row give 40 four-cell vectors per colour:
    two rows per 64-thread block and a second block with 8 of its 32 lanes active per row;
    192 rows and 160 planes make 7680 blocks."""
    dims = (320, 192, 160)
    s, M = make(dims, "mixed", coeffs="faces")
    nx, ny, nz = dims
    faces = tuple(f.astype(np.float32).astype(np.float64) for f in M.level_faces(0))
    x = rnd((nz, ny, nx), 33).astype(np.float32)
    b = rnd((nz, ny, nx), 34).astype(np.float32)
    xg, bg = dev(x, torch.float32), dev(b, torch.float32)
    for sweeps, order in ((1, 0), (1, 1), (2, 0)):
        xs = xg.clone()
        assert L.mg_smooth(s._h, 0, xs, bg, sweeps, order) == 0
        assert rel(host(xs), O.rbgs(faces, b, x, s.h, sweeps, order)) < TOL[torch.float32]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("prolong", ["trilinear", "constant"])
def test_transfers_match_oracle(dims, dtype, prolong):
    s, M = make(dims, "fp64" if dtype == torch.float64 else "mixed", prolong=prolong)
    tol = TOL[dtype]
    kind = O.TRILINEAR if prolong == "trilinear" else O.CONSTANT
    for l in range(M.nlevels - 1):
        nx, ny, nz = M.level_dims(l)
        cx, cy, cz = M.level_dims(l + 1)
        H = s.h * 2**l
        faces = M.level_faces(l)
        if dtype == torch.float32:
            faces = tuple(f.astype(np.float32).astype(np.float64) for f in faces)
        npd = np.float32 if dtype == torch.float32 else np.float64
        x = rnd((nz, ny, nx), 30 + l).astype(npd)
        b = rnd((nz, ny, nx), 40 + l).astype(npd)
        bc = torch.empty((cz, cy, cx), dtype=dtype, device="cuda")
        assert L.mg_residual_restrict(s._h, l, dev(x, dtype), dev(b, dtype), bc) == 0
        assert rel(host(bc), O.restrict(O.residual(faces, b, x, H))) < tol
        ec = rnd((cz, cy, cx), 50 + l).astype(npd)
        xg = dev(x, dtype)
        assert L.mg_prolong_correct(s._h, l, dev(ec, dtype), xg) == 0
        assert rel(host(xg), O.prolong_correct(ec, x, kind)) < tol


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_coarse_solve_matches_oracle(dims, dtype):
    s, M = make(dims, "fp64" if dtype == torch.float64 else "mixed")
    l = M.nlevels - 1
    nx, ny, nz = M.level_dims(l)
    H = s.h * 2**l
    npd = np.float32 if dtype == torch.float32 else np.float64
    r = rnd((nz, ny, nx), 60).astype(npd)
    e = torch.empty((nz, ny, nx), dtype=dtype, device="cuda")
    assert L.mg_coarse_solve(s._h, dev(r, dtype), e) == 0
    want = O.coarse_solve(M.level_faces(l), r.astype(np.float64), H)
    assert rel(host(e), want) < (1e-11 if dtype == torch.float64 else 1e-6)


@pytest.mark.parametrize("dims", [(8, 6, 4), (7, 5, 3), (9, 9, 9), (31, 1, 1)])
def test_single_level_grid_is_a_dense_solve(dims):
    """The dense coarse pseudo-inverse (blocked Gauss-Jordan, 32 pivots per step) on grids of
    192, 105, 729 and 31 cells: whole blocks, a ragged last block, a single short block."""
    s, M = make(dims, "fp64", coarsest=max(dims))
    assert s.num_levels == 1 and M.nlevels == 1
    nx, ny, nz = dims
    b = rnd((nz, ny, nx), 70)
    p = s.solve(dev(b))
    assert s.last_stats.cycles == 1
    want, _, _ = M.solve_exact(b)
    assert rel(host(p), want) < 1e-11


def test_density_errors_are_reported_not_faulted():
    n = 16
    s = Solver((n, n, n), precision="mixed", coarsest=8)
    rho = np.full((n, n, n), 1.0)
    rho[3, 4, 5] = 0.0
    with pytest.raises(MgError) as ei:
        s.set_density(dev(rho))
    assert ei.value.code == MG_ERR_DENSITY
    with pytest.raises(MgError) as ei:
        s.solve(dev(np.ones((n, n, n))))
    assert ei.value.code == MG_ERR_STATE
    rho[3, 4, 5] = np.nan
    with pytest.raises(MgError):
        s.set_density(dev(rho))
    faces = list(O.faces_from_density(np.ones((n, n, n))))
    faces[1][2, 3, 4] = -1.0
    with pytest.raises(MgError) as ei:
        s.set_face_coeffs(*(dev(f) for f in faces))
    assert ei.value.code == MG_ERR_DENSITY
    rho[3, 4, 5] = 2.0
    s.set_density(dev(rho))  # recovers
    s.solve(dev(rnd((n, n, n), 1)))


@pytest.mark.parametrize("dims", DIMS + WIDE)
@pytest.mark.parametrize("dtype,coeffs", [(torch.float64, "rho"), (torch.float32, "rho"), (torch.float32, "faces")])
@pytest.mark.parametrize("sweeps,zero", [(0, False), (1, True), (2, True), (2, False), (3, False)])
def test_fused_presmooth_restrict_matches_oracle(dims, dtype, coeffs, sweeps, zero):
    """The V-cycle's downward step as one fused pass chain: sweeps + residual + 8:1 restriction."""
    s, M = make(dims, "fp64" if dtype == torch.float64 else "mixed", coeffs=coeffs)
    tol = TOL[dtype]
    npd = np.float32 if dtype == torch.float32 else np.float64
    for l in range(M.nlevels - 1):
        nx, ny, nz = M.level_dims(l)
        cx, cy, cz = M.level_dims(l + 1)
        H = s.h * 2**l
        faces = M.level_faces(l)
        if dtype == torch.float32:
            faces = tuple(f.astype(np.float32).astype(np.float64) for f in faces)
        x = np.zeros((nz, ny, nx), npd) if zero else rnd((nz, ny, nx), 80 + l).astype(npd)
        b = rnd((nz, ny, nx), 90 + l).astype(npd)
        xg = dev(x, dtype) if not zero else torch.full((nz, ny, nx), 123.0, dtype=dtype, device="cuda")
        bc = torch.empty((cz, cy, cx), dtype=dtype, device="cuda")
        assert L.mg_presmooth_restrict(s._h, l, xg, dev(b, dtype), sweeps, bc, x_is_zero=zero) == 0
        xs = O.rbgs(faces, b, x, H, sweeps, 0)
        assert rel(host(xg), xs) < tol if sweeps else np.array_equal(host(xg), x)
        # restriction of the residual of the returned x
        bc_from_x = O.restrict(O.residual(faces, b, host(xg), H))
        assert rel(host(bc), bc_from_x) < (1e-13 if dtype == torch.float64 else 1e-5)
        assert rel(host(bc), O.restrict(O.residual(faces, b, xs, H))) < (1e-12 if dtype == torch.float64 else 2e-5)


@pytest.mark.parametrize("dims", DIMS + WIDE)
@pytest.mark.parametrize("dtype,coeffs", [(torch.float64, "rho"), (torch.float32, "rho"), (torch.float32, "faces")])
@pytest.mark.parametrize("prolong", ["trilinear", "constant"])
@pytest.mark.parametrize("sweeps", [0, 1, 2, 3])
def test_fused_prolong_postsmooth_matches_oracle(dims, dtype, coeffs, prolong, sweeps):
    """The V-cycle's upward step: correction x + P ec then post sweeps (black first), fused."""
    s, M = make(dims, "fp64" if dtype == torch.float64 else "mixed", prolong=prolong, coeffs=coeffs)
    tol = TOL[dtype]
    kind = O.TRILINEAR if prolong == "trilinear" else O.CONSTANT
    npd = np.float32 if dtype == torch.float32 else np.float64
    for l in range(M.nlevels - 1):
        nx, ny, nz = M.level_dims(l)
        cx, cy, cz = M.level_dims(l + 1)
        H = s.h * 2**l
        faces = M.level_faces(l)
        if dtype == torch.float32:
            faces = tuple(f.astype(np.float32).astype(np.float64) for f in faces)
        x = rnd((nz, ny, nx), 100 + l).astype(npd)
        b = rnd((nz, ny, nx), 110 + l).astype(npd)
        ec = rnd((cz, cy, cx), 120 + l).astype(npd)
        xg = dev(x, dtype)
        assert L.mg_prolong_postsmooth(s._h, l, dev(ec, dtype), xg, dev(b, dtype), sweeps) == 0
        want = O.rbgs(faces, b, O.prolong_correct(ec, x, kind), H, sweeps, 1)
        assert rel(host(xg), want) < tol


def test_smoothing_components_need_the_cycle_precision():
    s, _ = make((16, 16, 16), "mixed")
    x = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda")
    assert L.mg_smooth(s._h, 0, x, x.clone(), 1) == L.MG_ERR_ARG
