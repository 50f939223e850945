"""The passes either side of the solve: the velocity correction of the projection step
(mg_project) and the density adjoint (mg_density_grads), through the C ABI.

Velocity correction: the GPU result equals the oracle's u + beta (G p + sigma csf) at the
same p (both FP64; the fused multiply-adds round differently, so 1e-14 of the largest
velocity), the walls are untouched bitwise, and -- a property the oracle does not enter --
the corrected field's divergence is the solve's residual: |D u_new| <= 1.05 rtol |b - mean b|.

Density adjoint: the GPU takes FP32 face gradients and forms the per-cell sum and the factor
-1/(2 rho^2) in FP32.  Against the oracle's FP64 formula on the same FP32 gradients each cell
must lie within the rounding bound of that arithmetic,
    |d_gpu - d_oracle| <= 8 u (sum_f |g_f|) / (2 rho^2),   u = 2^-24
(five additions with relative error <= u each on partial sums bounded by sum |g_f|, the
rounding of rho to FP32 (doubled by the square), the product and the reciprocal: at most
5u + 2u + 2u of sum |g_f| / (2 rho^2), taken as 8u plus the FP64 side's own rounding, which
is far smaller); dL/df_q adds one more FP32 product and the FP32 rounding of rho_q - rho_last
(2u relative).  Against the oracle's exact FP64 chain (its own lambda and p) the relative L2
error is bounded by that of the FP32 face gradients (1e-6 in the adjoint tests), times the
cancellation between a cell's faces; 1e-5 is asserted.  The autograd Function is checked by
central differences of FP64 solves in the fractions.
"""
import numpy as np
import pytest
import torch

import dropfilm as D
import oracle as O
from paper_2605_30082_gb300 import PoissonSolveFractions, Solver

from _helpers import RHO_PHASE, csf_case, dev, host, random_rho, rel

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _walls_unchanged(un, u):
    return (np.array_equal(un[0][:, :, [0, -1]], u[0][:, :, [0, -1]])
            and np.array_equal(un[1][:, [0, -1], :], u[1][:, [0, -1], :])
            and np.array_equal(un[2][[0, -1]], u[2][[0, -1]]))


@pytest.mark.parametrize("prec,with_csf", [("mixed", True), ("fp64", True), ("mixed", False),
                                           ("mixed_df", True)])
def test_projection_32cubed(prec, with_csf):
    c = csf_case(32)
    h, sigma = c["h"], 0.03
    csf_h = c["csf"] if with_csf else None
    s = Solver((32, 32, 32), h=h, precision=prec, coarsest=8, rtol=1e-10)
    s.set_density(dev(c["rho"]))
    csf = tuple(dev(a) for a in csf_h) if with_csf else None
    u_h = [a.numpy() for a in c["u"]]
    b = s.rhs(u=tuple(dev(a) for a in u_h), csf=csf, sigma=sigma)
    p = s.solve(b)
    u = [dev(a) for a in u_h]
    out = s.project(p, u, csf=csf, sigma=sigma, out=[torch.full_like(a, np.nan) for a in u])
    un = [host(a) for a in out]
    assert all(np.array_equal(host(a), b) for a, b in zip(u, u_h))  # input untouched
    s.project(p, u, csf=csf, sigma=sigma)  # in place: the same values
    assert all(np.array_equal(host(a), b) for a, b in zip(u, un))
    want = O.project(u_h, c["faces"], host(p), h, csf=csf_h, sigma=sigma)
    for a, w in zip(un, want):
        assert np.abs(a - w).max() <= 1e-14 * np.abs(w).max()
    assert _walls_unchanged(un, u_h)
    bh = host(b)
    div = O.divergence(un, h)
    nb = np.linalg.norm(bh - bh.mean())
    assert np.linalg.norm(div - bh.mean()) <= 1.05 * s.last_stats.relres * nb + 1e-12 * nb
    assert s.last_stats.relres <= 1e-10


def test_projection_rejects_bad_arguments():
    s = Solver((16, 16, 16), precision="mixed", coarsest=8)
    p = torch.zeros((16,) * 3, dtype=torch.float64, device="cuda")
    u = [torch.zeros(sh, dtype=torch.float64, device="cuda") for sh in s.face_shapes]
    from paper_2605_30082_gb300 import MgError, _lib as L
    with pytest.raises(MgError) as e:  # no operator yet
        s.project(p, u)
    assert e.value.code == L.MG_ERR_STATE
    s.set_density(torch.ones((16,) * 3, dtype=torch.float64, device="cuda"))
    # p = 0 and no surface term leave u as it is
    u0 = [torch.randn(sh, dtype=torch.float64, device="cuda") for sh in s.face_shapes]
    u1 = [a.clone() for a in u0]
    s.project(p, u1)
    assert all(torch.equal(a, b) for a, b in zip(u0, u1))
    assert L.lib().mg_project(s._h, None, None, None, None, 0.0, None, None, None, None, None,
                              None) == L.MG_ERR_ARG
    # out must be all three inputs or none of them
    o = [torch.empty_like(a) for a in u0]
    with pytest.raises(MgError) as e:
        s.project(p, u0, out=[u0[0], o[1], o[2]])
    assert e.value.code == L.MG_ERR_ARG


def _density_bound(rho, g, extra=0.0):
    """Per-cell rounding bound of the FP32 density adjoint on the same FP32 gradients."""
    gx, gy, gz = g
    nz, ny, nx = rho.shape
    a = np.zeros_like(rho)
    a[:, :, 1:] += np.abs(gx[:, :, 1:nx])
    a[:, :, :-1] += np.abs(gx[:, :, 1:nx])
    a[:, 1:, :] += np.abs(gy[:, 1:ny, :])
    a[:, :-1, :] += np.abs(gy[:, 1:ny, :])
    a[1:] += np.abs(gz[1:nz])
    a[:-1] += np.abs(gz[1:nz])
    return (8 + extra) * U32 * a / (2 * rho * rho) + 1e-300


def test_density_grads_32cubed():
    c = csf_case(32)
    h, sigma = c["h"], 0.03
    s = Solver((32, 32, 32), h=h, precision="mixed", coarsest=8)
    fr = [dev(c["fd"].numpy()), dev(c["ff"].numpy())]
    rho = s.density_from_fractions(fr, list(RHO_PHASE))
    s.set_density(rho)
    csf = tuple(dev(a) for a in c["csf"])
    b = s.rhs(u=tuple(a.cuda() for a in c["u"]), csf=csf, sigma=sigma)
    p = s.solve(b)
    lam, g, _ = s.adjoint(dev(c["w"]), p, csf=csf, sigma=sigma)
    drho, (dfd, dff) = s.density_grads(rho, g, RHO_PHASE)
    drho_only = s.density_grads(rho, g)
    assert torch.equal(drho, drho_only)
    gh = [host(a) for a in g]
    rh = host(rho)
    # the same FP32 gradients through the oracle's FP64 formula
    d_o, (fd_o, ff_o) = O.density_grads(rh, gh, RHO_PHASE)
    bound = _density_bound(rh, gh)
    assert np.all(np.abs(host(drho) - d_o) <= bound)
    for got, want, dr in ((dfd, fd_o, 998.0 - 1.2), (dff, ff_o, 880.0 - 1.2)):
        assert np.all(np.abs(host(got) - want) <= _density_bound(rh, gh, 2.0) * dr)
    # the oracle's exact chain: its own p and lambda, FP64 face gradients
    M = O.Multigrid(c["faces"], h, coarsest=8)
    bo = O.rhs([a.numpy() for a in c["u"]], c["faces"], h, csf=c["csf"], sigma=sigma)
    p_o = M.solve_exact(bo)[0]
    lam_o = M.solve_exact(c["w"])[0]
    g_o, _ = O.adjoint_grads(c["faces"], lam_o, p_o, h, csf=c["csf"], sigma=sigma)
    d_x, (fd_x, _) = O.density_grads(c["rho"], g_o, RHO_PHASE)
    assert rel(host(drho), d_x) < 1e-5
    assert rel(host(dfd), fd_x) < 1e-5


def test_density_grads_argument_checks():
    s = Solver((16, 16, 16), precision="mixed", coarsest=8)
    from paper_2605_30082_gb300 import _lib as L
    lib = L.lib()
    assert lib.mg_density_grads(s._h, None, None, None, None, None, 0, None, None) == L.MG_ERR_ARG
    rho = torch.ones((16,) * 3, dtype=torch.float64, device="cuda")
    g = [torch.zeros(sh, dtype=torch.float32, device="cuda") for sh in s.face_shapes]
    drho = torch.empty_like(rho)
    with pytest.raises(ValueError):
        L.mg_density_grads(s._h, rho, g, drho, s.dims, rho_phase=[1.0], dfrac=[torch.empty_like(rho)] * 2)
    import ctypes as C
    pr = lambda t: C.c_void_p(t.data_ptr())
    assert lib.mg_density_grads(s._h, pr(rho), pr(g[0]), pr(g[1]), pr(g[2]), pr(drho), 5, None,
                                None) == L.MG_ERR_ARG
    # zero face gradients give zero density and fraction gradients
    drho, (df,) = s.density_grads(rho, g, [2.0, 1.0])
    assert float(drho.abs().max()) == 0.0 and float(df.abs().max()) == 0.0


def test_fractions_autograd_finite_differences_32cubed():
    """dL/df_drop, dL/df_film of L = sum(w p) through Eq. (5), the face coefficients and the
    solve, against central differences of FP64 solves (rtol 1e-13) along random directions; dL/db_u and dL/dsigma match the face-coefficient Function's."""
    n = 32
    c = csf_case(n)
    h = c["h"]
    s = Solver((n, n, n), h=h, precision="fp64", coarsest=8, rtol=1e-13, max_cycles=400)
    fd = dev(c["fd"].numpy()).requires_grad_(True)
    ff = dev(c["ff"].numpy()).requires_grad_(True)
    b_u = dev(c["b"]).requires_grad_(True)
    sigma = torch.tensor(0.03, dtype=torch.float64, device="cuda", requires_grad=True)
    csf = tuple(dev(a) for a in c["csf"])
    w = dev(c["w"])
    p = PoissonSolveFractions.apply(s, b_u, RHO_PHASE, sigma, csf, fd, ff)
    (w * p).sum().backward()

    def L(a, b):
        with torch.no_grad():
            return float((w * PoissonSolveFractions.apply(s, b_u.detach(), RHO_PHASE, 0.03, csf, a, b)).sum())

    # directions scaled so that every cell's density moves by eps * z * rho (relative steps, as
    # in the face-coefficient check): dL/df_q . v with v = z rho / (rho_q - rho_last)
    rng = np.random.default_rng(7)
    rho = dev(c["rho"])
    eps = 1e-6
    for q, (x, other) in enumerate(((fd, ff), (ff, fd))):
        v = torch.tensor(rng.standard_normal((n, n, n)), device="cuda") * rho / (RHO_PHASE[q] - RHO_PHASE[2])
        xp, xm = x.detach() + eps * v, x.detach() - eps * v
        args = (xp, other.detach()) if q == 0 else (other.detach(), xp)
        argm = (xm, other.detach()) if q == 0 else (other.detach(), xm)
        fdiff = (L(*args) - L(*argm)) / (2 * eps)
        ad = float((x.grad * v).sum())
        assert abs(fdiff - ad) <= 1e-5 * abs(ad), (q, fdiff, ad)
    # dL/db_u is the zero-mean adjoint solution; dL/dsigma the oracle's
    M = O.Multigrid(c["faces"], h, coarsest=8)
    assert rel(host(b_u.grad), M.solve_exact(c["w"])[0]) < 1e-9
    lam_o = M.solve_exact(c["w"])[0]
    bo = O.rhs([a.numpy() for a in c["u"]], c["faces"], h, csf=c["csf"], sigma=0.03)
    _, ds_o = O.adjoint_grads(c["faces"], lam_o, M.solve_exact(bo)[0], h, csf=c["csf"], sigma=0.03)
    assert abs(float(sigma.grad) - ds_o) <= 1e-8 * abs(ds_o)


@pytest.mark.parametrize("with_csf", [False, True])
def test_projection_spacing_not_a_power_of_two(with_csf):
    """h = 1/48: the velocity correction multiplies by 1/h in FP64 (no exponent scaling)."""
    c = csf_case(48)
    h, sigma = c["h"], 0.03
    s = Solver((48, 48, 48), h=h, precision="mixed", coarsest=8)
    s.set_density(dev(c["rho"]))
    csf_h = c["csf"] if with_csf else None
    csf = tuple(dev(a) for a in csf_h) if with_csf else None
    u_h = [a.numpy() for a in c["u"]]
    p = s.solve(s.rhs(u=tuple(dev(a) for a in u_h), csf=csf, sigma=sigma))
    out = s.project(p, [dev(a) for a in u_h], csf=csf, sigma=sigma,
                    out=[torch.empty(a.shape, dtype=torch.float64, device="cuda") for a in u_h])
    want = O.project(u_h, c["faces"], host(p), h, csf=csf_h, sigma=sigma)
    for a, w in zip(out, want):
        assert np.abs(host(a) - w).max() <= 1e-14 * np.abs(w).max()


@pytest.mark.parametrize("nfrac", [1, 3, 4])
def test_density_grads_fraction_counts(nfrac):
    """1, 3 and 4 fractions (Eq. (5) with nfrac + 1 phases), random FP32 face gradients, against
    the oracle's formula on the same gradients within the FP32 rounding bound."""
    dims = (24, 20, 16)
    nx, ny, nz = dims
    rng = np.random.default_rng(20 + nfrac)
    phase = list(rng.uniform(1.0, 1000.0, nfrac + 1))
    rho = random_rho(dims, 30 + nfrac)
    s = Solver(dims, h=1.0 / 24, precision="mixed", coarsest=8)
    g = tuple(torch.tensor(rng.standard_normal(sh), dtype=torch.float32, device="cuda") for sh in s.face_shapes)
    drho, dfrac = s.density_grads(dev(rho), g, phase)
    assert len(dfrac) == nfrac
    gh = [host(a) for a in g]
    d_o, f_o = O.density_grads(rho, gh, phase)
    assert np.all(np.abs(host(drho) - d_o) <= _density_bound(rho, gh))
    for q in range(nfrac):
        dr = abs(phase[q] - phase[nfrac])
        assert np.all(np.abs(host(dfrac[q]) - f_o[q]) <= _density_bound(rho, gh, 2.0) * dr + 1e-300)


def test_density_grads_outside_the_fp32_range_use_fp64():
    """Densities outside [2^-20, 2^21) take the FP64 formula: tiny and huge densities give the
    oracle's values to FP32 precision of the summed gradients (no overflow, no underflow)."""
    dims = (16, 16, 16)
    rho = random_rho(dims, 41)
    rho[0, 0, :8] = 1e-9
    rho[3, 5, :8] = 1e9
    rho[7, 7, 7] = 2.0 ** -20  # the edge of the FP32 path
    s = Solver(dims, h=1.0 / 16, precision="mixed", coarsest=8)
    rng = np.random.default_rng(5)
    g = tuple(torch.tensor(rng.standard_normal(sh), dtype=torch.float32, device="cuda") for sh in s.face_shapes)
    drho = s.density_grads(dev(rho), g)
    gh = [host(a) for a in g]
    d_o = O.density_grads(rho, gh)
    got = host(drho)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - d_o) <= _density_bound(rho, gh))
    assert abs(got[0, 0, 0]) > 1e15  # -sum g / (2 rho^2) with rho = 1e-9
