"""Pins of the FP64 CPU oracle against facts fixed by mathematics (no GPU).

Each test ties an oracle routine to something other than itself: closed-form
discrete eigenpairs, a hand-derived stencil, second-order convergence to an
analytic solution, dense LAPACK solves, operator invariants, brute-force finite
differences.  A dropped term, a wrong sign or index or a transposed operand in
the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import torch

import dropfilm as D
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def const_faces(nx, ny, nz, beta):
    fx, fy, fz = (np.full(s, float(beta)) for s in O.face_shapes(nx, ny, nz))
    fx[:, :, 0] = fx[:, :, -1] = 0.0
    fy[:, 0, :] = fy[:, -1, :] = 0.0
    fz[0] = fz[-1] = 0.0
    return fx, fy, fz


def random_faces(nx, ny, nz, seed, lo=1.2, hi=998.0):
    """Face coefficients 1/rho with rho log-uniform in [lo, hi] per cell (harmonic faces)."""
    n = nx * ny * nz
    u = D.uniform53(seed, torch.arange(n)).numpy().reshape(nz, ny, nx)
    rho = lo * (hi / lo) ** u
    return O.faces_from_density(rho), rho


def cosine_mode(nx, ny, nz, m):
    x = np.cos(math.pi * m[0] * (np.arange(nx) + 0.5) / nx)
    y = np.cos(math.pi * m[1] * (np.arange(ny) + 0.5) / ny)
    z = np.cos(math.pi * m[2] * (np.arange(nz) + 0.5) / nz)
    return z[:, None, None] * y[None, :, None] * x[None, None, :]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------- generators

def test_splitmix64_published_values():
    rows = [l.split() for l in open(os.path.join(GOLD, "splitmix64_seed0.txt")) if l[0] != "#"]
    out = D.splitmix64(0, torch.tensor([int(r[0]) for r in rows]))
    got = [int(v) & (2**64 - 1) for v in out]
    assert got == [int(r[1], 16) for r in rows]


def test_subcell_fractions_brute_force():
    # tiny sphere on an 8^3 grid, 4^3 sample points per cell: compare with explicit loops
    g = D.Geometry(n=8, center=(4, 4, 5), radius=2, z_film=2)
    fd, ff = D.fractions_subcell(g)
    bd = np.zeros((8, 8, 8))
    bf = np.zeros((8, 8, 8))
    for k in range(8):
        for j in range(8):
            for i in range(8):
                cd = cf = 0
                for c in range(4):
                    for b in range(4):
                        for a in range(4):
                            x, y, z = i + (a + 0.5) / 4, j + (b + 0.5) / 4, k + (c + 0.5) / 4
                            cd += (x - 4) ** 2 + (y - 4) ** 2 + (z - 5) ** 2 <= 4
                            cf += z < 2
                bd[k, j, i] = cd / 64
                bf[k, j, i] = min(cf / 64, 1 - cd / 64)
    assert np.array_equal(fd.numpy(), bd)
    assert np.array_equal(ff.numpy(), bf)


def test_ramp_fractions_volume_and_purity():
    g = D.scaled_geometry(64)
    fd, ff = D.fractions_ramp(g)
    vol = fd.sum().item()
    assert abs(vol - 4 / 3 * math.pi * 16**3) / vol < 0.01
    assert ff.sum().item() == 64 * 64 * 12  # film z < 12 with a symmetric ramp
    assert fd[40, 32, 32] == 1.0 and fd[0, 0, 0] == 0.0
    assert ((fd >= 0) & (fd <= 1)).all() and ((fd + ff) <= 1).all()


def test_face_velocity_walls_and_range():
    ux, uy, uz = D.face_velocities(6, seed=0)
    assert ux.shape == (6, 6, 7) and uy.shape == (6, 7, 6) and uz.shape == (7, 6, 6)
    assert (ux[:, :, 0] == 0).all() and (ux[:, :, -1] == 0).all()
    assert (uy[:, 0] == 0).all() and (uz[-1] == 0).all()
    inner = ux[:, :, 1:-1]
    assert inner.abs().max() < 1 and inner.abs().min() > 0
    # stream order: ux first, counter = flat index
    u0 = 2 * D.uniform53(0, torch.tensor([1])) - 1
    assert ux[0, 0, 1].item() == u0.item()


# ---------------------------------------------------------------- Eq. (5), faces

def test_density_mixture_rule():
    fd = np.array([[[1.0, 0.0, 0.0, 0.5]]])
    ff = np.array([[[0.0, 1.0, 0.0, 0.25]]])
    rho = O.density([fd, ff], [998.0, 880.0, 1.2])
    assert np.allclose(rho.ravel(), [998.0, 880.0, 1.2, 0.5 * 998 + 0.25 * 880 + 0.25 * 1.2], rtol=1e-15)


def test_face_coefficient_inverse_harmonic_mean():
    rho = np.array([[[998.0, 1.2, 1.2, 880.0]]])
    bx, by, bz = O.faces_from_density(rho)
    want = [(998.0 + 1.2) / (2 * 998.0 * 1.2), 1 / 1.2, (1.2 + 880.0) / (2 * 1.2 * 880.0)]
    assert np.allclose(bx[0, 0, 1:4], want, rtol=1e-15)
    assert bx[0, 0, 0] == 0 and bx[0, 0, 4] == 0 and (by == 0).all() and (bz == 0).all()


# ---------------------------------------------------------------- the operator

def test_stencil_hand_derived_rows():
    nx = ny = nz = 2
    fx, fy, fz = (np.zeros(s) for s in O.face_shapes(2, 2, 2))
    for k in range(2):
        for j in range(2):
            fx[k, j, 1] = 1 + j + 2 * k
    for k in range(2):
        for i in range(2):
            fy[k, 1, i] = 5 + i + 2 * k
    for j in range(2):
        for i in range(2):
            fz[1, j, i] = 9 + i + 2 * j
    A = O.assemble_dense((fx, fy, fz), 0.5)
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLD, "stencil_2x2x2.txt")) if l[0] != "#"]
    for r in rows:
        assert np.array_equal(A[int(r[0])], np.array(r[1:]))
    # or_apply agrees with the dense matrix column by column
    for c in range(8):
        e = np.zeros(8)
        e[c] = 1
        col = O.apply((fx, fy, fz), e.reshape(2, 2, 2), 0.5).ravel()
        assert np.array_equal(col, A[:, c])


@pytest.mark.parametrize("dims,m", [((16, 16, 16), (1, 2, 3)), ((16, 8, 32), (3, 1, 5)), ((8, 8, 8), (7, 0, 1))])
def test_discrete_cosine_eigenpair(dims, m):
    nx, ny, nz = dims
    h = 1.0 / 16
    beta = 0.5
    p = cosine_mode(nx, ny, nz, m)
    lam = beta / h**2 * sum(4 * math.sin(math.pi * md / (2 * nd)) ** 2 for md, nd in zip(m, (nx, ny, nz)))
    Ap = O.apply(const_faces(nx, ny, nz, beta), p, h)
    assert rel(Ap, lam * p) < 1e-13


def test_operator_invariants():
    faces, _ = random_faces(6, 5, 4, seed=11)
    h = 0.25
    ones = np.ones((4, 5, 6))
    assert np.array_equal(O.apply(faces, ones, h), np.zeros_like(ones))  # A 1 = 0 exactly
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal((2, 4, 5, 6))
    Au, Av = O.apply(faces, u, h), O.apply(faces, v, h)
    assert abs((v * Au).sum() - (u * Av).sum()) <= 1e-13 * np.abs(v * Au).sum()
    assert (u * Au).sum() > 0  # PSD and u is not constant
    assert abs(Au.sum()) <= 1e-13 * np.abs(Au).sum()  # fluxes telescope


def test_divergence_is_minus_gradient_transpose():
    nx, ny, nz, h = 5, 4, 3, 0.5
    rng = np.random.default_rng(1)
    u = [rng.standard_normal(s) for s in O.face_shapes(nx, ny, nz)]
    for a, ax in zip(u, (2, 1, 0)):
        idx = [slice(None)] * 3
        idx[ax] = 0
        a[tuple(idx)] = 0
        idx[ax] = -1
        a[tuple(idx)] = 0
    phi = rng.standard_normal((nz, ny, nx))
    lhs = (phi * O.divergence(u, h)).sum()
    gx = np.zeros_like(u[0]); gx[:, :, 1:-1] = (phi[:, :, 1:] - phi[:, :, :-1]) / h
    gy = np.zeros_like(u[1]); gy[:, 1:-1] = (phi[:, 1:] - phi[:, :-1]) / h
    gz = np.zeros_like(u[2]); gz[1:-1] = (phi[1:] - phi[:-1]) / h
    rhs = -sum((a * g).sum() for a, g in zip(u, (gx, gy, gz)))
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    # A = -D diag(beta) G: the operator equals minus the divergence of beta * gradient
    faces, _ = random_faces(nx, ny, nz, seed=3)
    flux = [f * g for f, g in zip(faces, (gx, gy, gz))]
    assert rel(O.apply(faces, phi, h), -O.divergence(flux, h)) < 1e-13


def test_csf_faces_linear_fields_closed_form():
    """CSF face quantity kappa_f (f_R - f_L)/h, pinned by closed forms.

    f linear in the cell centres has the same difference quotient on every interior face
    of an axis (its slope), and the mean of a linear kappa over the two cells of a face is
    kappa at the face centre.  So csf on an x-face at x_f is (a0 + a1 x_f) * sx exactly up to
    rounding: a flipped difference changes the sign, a one-sided kappa shifts x_f by h/2,
    a transposed axis picks up the wrong slope.  Wall faces are 0."""
    nx, ny, nz, h = 7, 5, 6, 0.25
    sx, sy, sz = 0.7, -1.3, 2.1
    cx = (np.arange(nx) + 0.5) * h
    cy = (np.arange(ny) + 0.5) * h
    cz = (np.arange(nz) + 0.5) * h
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    f = 0.3 + sx * X + sy * Y + sz * Z
    a0, ax, ay, az = 2.0, 0.5, -0.25, 0.125
    kappa = a0 + ax * X + ay * Y + az * Z
    gx, gy, gz = O.csf_faces(f, kappa, h)
    # face centres: x-face i sits at x = i h, y-face j at y = j h, z-face k at z = k h
    fxk = a0 + ax * (np.arange(nx + 1) * h)[None, None, :] + ay * cy[None, :, None] + az * cz[:, None, None]
    fyk = a0 + ax * cx[None, None, :] + ay * (np.arange(ny + 1) * h)[None, :, None] + az * cz[:, None, None]
    fzk = a0 + ax * cx[None, None, :] + ay * cy[None, :, None] + az * (np.arange(nz + 1) * h)[:, None, None]
    np.testing.assert_allclose(gx[:, :, 1:-1], (fxk * sx)[:, :, 1:-1], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(gy[:, 1:-1, :], (fyk * sy)[:, 1:-1, :], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(gz[1:-1], (fzk * sz)[1:-1], rtol=1e-13, atol=1e-13)
    for g, axis in ((gx, 2), (gy, 1), (gz, 0)):
        assert not np.take(g, [0, -1], axis=axis).any()
    # constant kappa: exactly kappa times the slope on every interior face
    gx, gy, gz = O.csf_faces(f, np.full_like(f, 3.0), h)
    np.testing.assert_allclose(gx[:, :, 1:-1], 3.0 * sx, rtol=1e-13)
    np.testing.assert_allclose(gy[:, 1:-1, :], 3.0 * sy, rtol=1e-13)
    np.testing.assert_allclose(gz[1:-1], 3.0 * sz, rtol=1e-13)


def test_csf_faces_unit_curvature_is_the_gradient():
    """With kappa = 1 the CSF face quantity is the discrete gradient G f, so the divergence of
    beta * csf is -A f for the (independently pinned) operator A with those faces: D diag(beta) G
    = -A.  Checked on random f and random harmonic faces, on a non-cubic grid."""
    nx, ny, nz, h = 6, 5, 4, 0.5
    f = np.random.default_rng(7).standard_normal((nz, ny, nx))
    faces, _ = random_faces(nx, ny, nz, seed=9)
    csf = O.csf_faces(f, np.ones_like(f), h)
    flux = [b * c for b, c in zip(faces, csf)]
    assert rel(O.divergence(flux, h), -O.apply(faces, f, h)) < 1e-13
    # the surface-tension RHS term assembled by or_rhs is the same quantity, scaled by sigma
    zero_u = [np.zeros(s) for s in O.face_shapes(nx, ny, nz)]
    assert rel(O.rhs(zero_u, faces, h, csf=csf, sigma=0.03), -0.03 * O.apply(faces, f, h)) < 1e-13


def test_manufactured_variable_coefficient_second_order():
    """p = cos(pi x)cos(pi y)cos(pi z), beta = 1 + xyz on [0,1]^3: error falls ~4x per refinement."""
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        c = (np.arange(n) + 0.5) * h
        f = np.arange(n + 1) * h
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        fx = 1 + np.einsum("k,j,i->kji", c, c, f)
        fy = 1 + np.einsum("k,j,i->kji", c, f, c)
        fz = 1 + np.einsum("k,j,i->kji", f, c, c)
        fx[:, :, 0] = fx[:, :, -1] = 0
        fy[:, 0] = fy[:, -1] = 0
        fz[0] = fz[-1] = 0
        pi = math.pi
        cx, cy, cz = np.cos(pi * X), np.cos(pi * Y), np.cos(pi * Z)
        sx, sy, sz = np.sin(pi * X), np.sin(pi * Y), np.sin(pi * Z)
        p = cx * cy * cz
        beta = 1 + X * Y * Z
        b = 3 * pi**2 * beta * p + pi * (Y * Z * sx * cy * cz + X * Z * cx * sy * cz + X * Y * cx * cy * sz)
        M = O.Multigrid((fx, fy, fz), h, coarsest=4)
        ph, rr, _ = M.solve_exact(b)
        errs.append(np.sqrt(np.mean((ph - (p - p.mean())) ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


# ---------------------------------------------------------------- smoother, transfers

def test_rbgs_half_sweep_zeroes_its_colour_residual():
    faces, _ = random_faces(8, 6, 4, seed=5)
    h = 1 / 8
    rng = np.random.default_rng(2)
    b = rng.standard_normal((4, 6, 8))
    p = rng.standard_normal((4, 6, 8))
    k, j, i = np.meshgrid(range(4), range(6), range(8), indexing="ij")
    red = (i + j + k) % 2 == 0
    p1 = O.rbgs_half(faces, b, p, h, 0)
    r1 = O.residual(faces, b, p1, h)
    assert np.abs(r1[red]).max() < 1e-12 * np.abs(b).max()
    assert np.array_equal(p1[~red], p[~red])  # black cells untouched
    p2 = O.rbgs_half(faces, b, p1, h, 1)
    r2 = O.residual(faces, b, p2, h)
    assert np.abs(r2[~red]).max() < 1e-12 * np.abs(b).max()
    # a full pre sweep is exactly red then black
    assert np.array_equal(O.rbgs(faces, b, p, h, 1, 0), p2)
    # Gauss-Seidel reduces the energy norm of the error
    x = O.Multigrid(faces, h, coarsest=8).solve_exact(b)[0]
    def energy(q):
        e = q - x
        return (e * O.apply(faces, e, h)).sum()
    assert energy(p2) < energy(p)


def test_restriction_conserves_sum():
    r = np.random.default_rng(3).standard_normal((8, 6, 10))
    rc = O.restrict(r)
    assert rc.shape == (4, 3, 5)
    assert abs(8 * rc.sum() - r.sum()) < 1e-12
    assert rc[1, 2, 3] == r[2:4, 4:6, 6:8].mean() or abs(rc[1, 2, 3] - r[2:4, 4:6, 6:8].mean()) < 1e-15


def test_prolongation_reproduces_constants_and_linears():
    ec = np.full((3, 4, 5), 2.5)
    for kind in (O.TRILINEAR, O.CONSTANT):
        e = O.prolong_correct(ec, np.zeros((6, 8, 10)), kind)
        assert np.allclose(e, 2.5, rtol=0, atol=1e-15)
    # trilinear is exact for a linear function away from the walls
    K, J, I = np.meshgrid(np.arange(3), np.arange(4), np.arange(5), indexing="ij")
    lin = lambda x, y, z: 0.3 * x - 1.1 * y + 2.0 * z
    ec = lin(I + 0.5, J + 0.5, K + 0.5)  # coarse centres in coarse-cell units
    e = O.prolong_correct(ec, np.zeros((6, 8, 10)), O.TRILINEAR)
    k, j, i = np.meshgrid(np.arange(6), np.arange(8), np.arange(10), indexing="ij")
    want = lin((i + 0.5) / 2, (j + 0.5) / 2, (k + 0.5) / 2)
    interior = (i > 0) & (i < 9) & (j > 0) & (j < 7) & (k > 0) & (k < 5)
    assert np.abs(e - want)[interior].max() < 1e-13
    # correction is additive
    base = np.random.default_rng(4).standard_normal((6, 8, 10))
    assert np.allclose(O.prolong_correct(ec, base, O.TRILINEAR) - base, e, atol=1e-14)


def test_face_coarsening_constant_and_mean():
    faces = const_faces(8, 4, 6, 0.7)
    cf = O.coarsen_faces(faces)
    want = const_faces(4, 2, 3, 0.7)
    for a, b in zip(cf, want):
        assert np.allclose(a, b, rtol=1e-15, atol=0)
    fx, fy, fz = random_faces(8, 4, 6, seed=7)[0]
    cx, cy, cz = O.coarsen_faces((fx, fy, fz))
    assert abs(cx[1, 1, 2] - fx[2:4, 2:4, 4].mean()) < 1e-16
    assert abs(cy[2, 1, 3] - fy[4:6, 2, 6:8].mean()) < 1e-16
    assert abs(cz[1, 0, 1] - fz[2, 0:2, 2:4].mean()) < 1e-16
    # with a constant coefficient the coarse operator is the same stencil with spacing 2h
    p = cosine_mode(4, 2, 3, (1, 1, 2))
    lam = 0.7 / (2 * 0.1) ** 2 * sum(4 * math.sin(math.pi * md / (2 * nd)) ** 2 for md, nd in zip((1, 1, 2), (4, 2, 3)))
    assert rel(O.apply(cf, p, 0.2), lam * p) < 1e-13


def test_level_rule():
    assert O.num_levels(32, 32, 32, 4) == 4
    assert O.num_levels(256, 256, 256, 8) == 6
    assert O.num_levels(512, 512, 512, 8) == 7
    assert O.num_levels(8, 16, 32, 4) == 4
    assert O.num_levels(6, 6, 6, 4) == 2
    assert O.num_levels(7, 7, 7, 4) == 1


# ---------------------------------------------------------------- coarse solve, full solve

def test_coarse_solve_is_zero_mean_pseudo_inverse():
    faces, _ = random_faces(4, 4, 4, seed=9)
    h = 0.25
    r = np.random.default_rng(5).standard_normal((4, 4, 4))
    e = O.coarse_solve(faces, r, h)
    assert abs(e.mean()) < 1e-13 * np.abs(e).max()
    assert rel(O.apply(faces, e, h), r - r.mean()) < 1e-12
    A = O.assemble_dense(faces, h)
    assert rel(e.ravel(), np.linalg.pinv(A, rcond=1e-10, hermitian=True) @ r.ravel()) < 1e-10


@pytest.mark.parametrize("field", ["dropfilm", "random"])
@pytest.mark.parametrize("coarsest", [2, 4])
def test_vcycle_solve_matches_dense_solve_8cubed(field, coarsest):
    n, h = 8, 1 / 8
    if field == "dropfilm":
        fd, ff = D.fractions_ramp(D.scaled_geometry(8))
        rho = O.density([fd.numpy(), ff.numpy()], [998.0, 880.0, 1.2])
        faces = O.faces_from_density(rho)
    else:
        faces, rho = random_faces(n, n, n, seed=13)
    u = [a.numpy() for a in D.face_velocities(n, seed=0)]
    b = O.divergence(u, h)
    A = O.assemble_dense(faces, h)
    ref = np.linalg.lstsq(np.vstack([A, np.ones((1, n**3))]), np.concatenate([b.ravel() - b.mean(), [0.0]]), rcond=None)[0]
    M = O.Multigrid(faces, h, coarsest=coarsest)
    p, st, nc, rr, hist = M.solve(b, rtol=1e-13, max_cycles=300)
    assert st == O.OK and rr <= 1e-13
    assert abs(p.mean()) < 1e-14 * np.abs(p).max()
    assert rel(p.ravel(), ref) < 1e-11
    assert all(hist[1:] < hist[:-1])  # monotone residual decrease


@pytest.mark.parametrize("field", ["dropfilm", "random"])
@pytest.mark.parametrize("prolong", [O.TRILINEAR, O.CONSTANT])
def test_fcg_solve_matches_dense_solve_8cubed(field, prolong):
    """Flexible CG preconditioned by the V-cycle reaches the same zero-mean discrete solution."""
    n, h = 8, 1 / 8
    if field == "dropfilm":
        fd, ff = D.fractions_ramp(D.scaled_geometry(8))
        faces = O.faces_from_density(O.density([fd.numpy(), ff.numpy()], [998.0, 880.0, 1.2]))
    else:
        faces, _ = random_faces(n, n, n, seed=13)
    b = O.divergence([a.numpy() for a in D.face_velocities(n, seed=0)], h)
    M = O.Multigrid(faces, h, coarsest=2, prolong=prolong)
    p, st, nit, rr, hist = M.fcg(b, rtol=1e-13)
    assert st == O.OK and rr <= 1e-12
    assert abs(p.mean()) < 1e-14 * np.abs(p).max()
    assert rel(p, _dense_p(faces, b, h)) < 1e-11
    assert nit < M.solve(b, rtol=1e-13)[2]  # fewer iterations than the plain V-cycle


def test_fcg_residuals_are_preconditioner_orthogonal():
    """With constant prolongation (restriction = P^T / 8, post-smoother the adjoint of the
    pre-smoother) the V-cycle is a symmetric preconditioner M, and preconditioned CG makes its
    residuals M^-1-orthogonal: r_j . z_k = 0 for j != k, z_k = M^-1 r_k.  With trilinear
    prolongation only the flexible method's local condition r_(k+1) . z_k = 0 holds.  A wrong
    step length or direction update breaks either."""
    n = 16
    faces, _ = random_faces(n, n, n, seed=4)
    b = np.random.default_rng(1).standard_normal((n, n, n))

    def gram(prolong):
        M = O.Multigrid(faces, 1 / n, coarsest=4, prolong=prolong)
        R, Z = M.fcg(b, rtol=1e-12, record=6)[5]
        return np.array([[np.vdot(R[j], Z[k]) / (np.linalg.norm(R[j]) * np.linalg.norm(Z[k])) for k in range(6)]
                         for j in range(6)])

    G = gram(O.CONSTANT)
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-12 and np.diag(G).min() > 0.1
    G = gram(O.TRILINEAR)
    assert max(abs(G[k + 1, k]) for k in range(5)) < 1e-12
    assert np.abs(G - np.diag(np.diag(G))).max() > 1e-6  # not symmetric: the global condition fails


def test_solve_cosine_mode_exact_on_dropfilm_free_grid():
    # constant coefficient: b = lambda * p* must return p* (zero mean)
    nx = ny = nz = 32
    h = 1 / 32
    p = cosine_mode(nx, ny, nz, (2, 1, 3))
    lam = 1.0 / h**2 * sum(4 * math.sin(math.pi * md / (2 * 32)) ** 2 for md in (2, 1, 3))
    M = O.Multigrid(const_faces(nx, ny, nz, 1.0), h, coarsest=4)
    ph, rr, nc = M.solve_exact(lam * p)
    assert rel(ph, p) < 1e-12


def test_solve_edge_cases():
    faces = const_faces(8, 8, 8, 1.0)
    M = O.Multigrid(faces, 1 / 8, coarsest=4)
    # zero and constant RHS give p = 0 in zero cycles
    for b in (np.zeros((8, 8, 8)), np.full((8, 8, 8), 3.0)):
        p, st, nc, rr, _ = M.solve(b)
        assert st == O.OK and nc == 0 and not p.any()
    # max_cycles exhausted
    b = np.random.default_rng(6).standard_normal((8, 8, 8))
    p, st, nc, rr, _ = M.solve(b, rtol=1e-30, max_cycles=2)
    assert st == O.ERR_NOT_CONVERGED and nc == 2
    # warm start from the solution needs no cycle
    p, st, nc, rr, _ = M.solve(b, rtol=1e-10)
    p2, st2, nc2, _, _ = M.solve(b, rtol=1e-10, p0=p)
    assert st2 == O.OK and nc2 == 0


# ---------------------------------------------------------------- adjoint

def _dense_p(faces, b, h):
    A = O.assemble_dense(faces, h)
    n = A.shape[0]
    return np.linalg.lstsq(np.vstack([A, np.ones((1, n))]), np.concatenate([b.ravel() - b.mean(), [0.0]]), rcond=None)[0].reshape(b.shape)


def test_adjoint_gradients_vs_central_differences_8cubed():
    n, h = 8, 1 / 8
    faces, _ = random_faces(n, n, n, seed=17, lo=1.0, hi=20.0)
    fd, _ = D.fractions_ramp(D.scaled_geometry(8))
    kappa = D.curvature_band(fd, D.scaled_geometry(8)).numpy()
    csf = O.csf_faces(fd.numpy(), kappa, h)
    u = [a.numpy() for a in D.face_velocities(n, seed=0)]
    sigma = 0.03
    w = D.normal_weights((n, n, n), seed=1).numpy()

    def loss(fc, s, bu_shift=None):
        b = O.rhs(u, fc, h, csf=csf, sigma=s)
        if bu_shift is not None:
            b = b + bu_shift
        return (w * _dense_p(fc, b, h)).sum()

    b = O.rhs(u, faces, h, csf=csf, sigma=sigma)
    p = _dense_p(faces, b, h)
    lam = _dense_p(faces, w, h)
    (gx, gy, gz), dsig = O.adjoint_grads(faces, lam, p, h, csf=csf, sigma=sigma)
    # dL/dsigma: L is linear in sigma
    eps = 1e-4
    fdsig = (loss(faces, sigma + eps) - loss(faces, sigma - eps)) / (2 * eps)
    assert abs(fdsig - dsig) <= 1e-7 * abs(dsig)
    # dL/dbeta on a few faces of each axis
    rng = np.random.default_rng(7)
    for axis, g in enumerate((gx, gy, gz)):
        for _ in range(3):
            shp = faces[axis].shape
            idx = tuple(int(rng.integers(1 if d == 2 - axis else 0, s - 1 if d == 2 - axis else s)) for d, s in enumerate(shp))
            e = 1e-6 * faces[axis][idx]
            fp = [f.copy() for f in faces]; fp[axis][idx] += e
            fm = [f.copy() for f in faces]; fm[axis][idx] -= e
            fdg = (loss(fp, sigma) - loss(fm, sigma)) / (2 * e)
            # FD rounding floor: ~1e-14 |L| / (2e-6 beta) relative to the largest gradient
            assert abs(fdg - g[idx]) <= 1e-6 * abs(g[idx]) + 1e-7 * np.abs(g).max(), (axis, idx, fdg, g[idx])
    # walls carry no gradient
    assert not gx[:, :, 0].any() and not gx[:, :, -1].any()
    # dL/db = lambda: directional derivative along a random cell field
    v = rng.standard_normal((n, n, n))
    fdb = (loss(faces, sigma, 1e-3 * v) - loss(faces, sigma, -1e-3 * v)) / 2e-3
    assert abs(fdb - (lam * v).sum()) <= 1e-8 * abs(fdb)


def _dropfilm8_with_csf():
    n, h = 8, 1 / 8
    g = D.scaled_geometry(8)
    fd, ff = D.fractions_ramp(g)
    kappa = D.curvature_band(fd, g).numpy()
    csf = O.csf_faces(fd.numpy(), kappa, h)
    u = [a.numpy() for a in D.face_velocities(n, seed=0)]
    return n, h, fd.numpy(), ff.numpy(), csf, u


def test_projection_removes_the_divergence_8cubed():
    """u + beta (G p + sigma csf) with p the exact solution of A p = D u + sigma D(beta csf)
    has zero discrete divergence (A = -D diag(beta) G); walls are unchanged; p = 0 without a
    surface term leaves u as it is."""
    n, h, fd, ff, csf, u = _dropfilm8_with_csf()
    faces = O.faces_from_density(O.density([fd, ff], [998.0, 880.0, 1.2]))
    b = O.rhs(u, faces, h, csf=csf, sigma=0.03)
    p = _dense_p(faces, b, h)
    un = O.project(u, faces, p, h, csf=csf, sigma=0.03)
    assert np.abs(O.divergence(un, h)).max() <= 1e-10 * np.abs(b).max()
    assert np.all(un[0][:, :, [0, -1]] == u[0][:, :, [0, -1]])
    assert np.all(un[1][:, [0, -1], :] == u[1][:, [0, -1], :])
    assert np.all(un[2][[0, -1]] == u[2][[0, -1]])
    same = O.project(u, faces, np.zeros_like(p), h)
    assert all(np.array_equal(a, c) for a, c in zip(same, u))


def test_density_and_fraction_gradients_vs_central_differences_8cubed():
    """dL/drho and dL/df_q (L = sum w p, b = D u + sigma D(beta(rho) csf)) against central
    differences of dense solves, rho from the fractions by Eq. (5)."""
    n, h, fd, ff, csf, u = _dropfilm8_with_csf()
    phase = [998.0, 880.0, 1.2]
    w = D.normal_weights((n, n, n), seed=1).numpy()
    sigma = 0.03

    def loss_rho(rho):
        faces = O.faces_from_density(rho)
        return float((w * _dense_p(faces, O.rhs(u, faces, h, csf=csf, sigma=sigma), h)).sum())

    rho = O.density([fd, ff], phase)
    faces = O.faces_from_density(rho)
    b = O.rhs(u, faces, h, csf=csf, sigma=sigma)
    p = _dense_p(faces, b, h)
    lam = _dense_p(faces, w, h)
    g, _ = O.adjoint_grads(faces, lam, p, h, csf=csf, sigma=sigma)
    drho, (dfd, dff) = O.density_grads(rho, g, phase)
    rng = np.random.default_rng(3)
    cells = [tuple(rng.integers(0, n, 3)) for _ in range(6)] + [(2, 3, 4)]
    for c in cells:
        # step 1e-3 rho: truncation ~1e-6 relative, while the dense solves' rounding (~1e-14 of
        # L ~ 300) stays far below the difference quotient
        e = 1e-3 * rho[c]
        rp, rm = rho.copy(), rho.copy()
        rp[c] += e
        rm[c] -= e
        fdiff = (loss_rho(rp) - loss_rho(rm)) / (2 * e)
        assert abs(fdiff - drho[c]) <= 1e-5 * max(abs(drho[c]), 1e-3 * np.abs(drho).max()), (c, fdiff, drho[c])
        # fraction of the drop: rho changes by (998 - 1.2) per unit f_drop
        assert dfd[c] == drho[c] * (998.0 - 1.2) and dff[c] == drho[c] * (880.0 - 1.2)
