"""Parity at the workload sizes, on the drop-on-film fields with the smoothed (ramp) interface.

256^3 (the plain FP64 and the mixed-precision configurations); the oracle runs the whole solve:
  - the FP64 GPU path reproduces the oracle's own V-cycle iteration at rtol 1e-10
    (same cycle count, p to 1e-12);
  - both mixed modes reach the exact discrete solution (the oracle's V-cycles run to
    stagnation) to relative L2 <= 1e-9 at rtol 1e-11.  At rtol 1e-10 the specified V(2,2)
    stops about 1.6e-9 from the exact solution at 256^3, the oracle's own iteration
    included, so the gate is applied at the tolerance that resolves it; the rtol 1e-10
    results are compared with the oracle's iteration instead.

512^3, in the launch configuration the benchmark times:
  - one level-0 RBGS sweep (FP32 s-form z-marching kernel, and FP64): sub-boxes of the grid
    are swept by the oracle; a red-then-black sweep depends on cells up to 2 away, so only
    cells at distance >= 2 from a sub-box face inside the grid are compared;
  - the benchmark's solve and adjoint: the oracle's FP64 residual of the returned p and
    lambda, the zero-mean gauge, and the face gradients against the oracle's adjoint
    formulas evaluated at the returned p and lambda.
"""
import numpy as np
import pytest
import torch

import dropfilm as D
import oracle as O
from paper_2605_30082_gb300 import Solver
from paper_2605_30082_gb300 import _lib as L

from _helpers import RHO_PHASE, dev, host, rel

pytestmark = pytest.mark.gpu


def fields(n):
    """The drop/film fields generated on the device, with host copies for the oracle."""
    g = D.scaled_geometry(n)
    cuda = torch.device("cuda")
    fd, ff = D.fractions_ramp(g, device=cuda)
    u = D.face_velocities(n, 0, device=cuda)
    fh = [host(fd), host(ff)]
    rho = O.density(fh, RHO_PHASE)
    return dict(n=n, h=1.0 / n, g=g, fd=fd, ff=ff, u=u, rho=rho, faces=O.faces_from_density(rho),
                b=O.divergence([host(a) for a in u], 1.0 / n))


def gpu_solver(c, precision, rtol, inner=1, method="vcycle"):
    s = Solver((c["n"],) * 3, h=c["h"], precision=precision, coarsest=8, rtol=rtol, max_cycles=200,
               inner_cycles=inner, method=method)
    rho = s.density_from_fractions([c["fd"], c["ff"]], list(RHO_PHASE))
    s.set_density(rho)
    return s, rho


@pytest.fixture(scope="module")
def c256():
    c = fields(256)
    M = O.Multigrid(c["faces"], c["h"], coarsest=8)
    c["iter"] = M.solve(c["b"], rtol=1e-10)
    c["exact"] = M.solve_exact(c["b"])[0]
    return c


def test_256_fp64_reproduces_oracle_iteration(c256):
    s, rho = gpu_solver(c256, "fp64", 1e-10)
    assert np.abs(host(rho) - c256["rho"]).max() <= 1e-13 * 998
    b = s.rhs(u=c256["u"])
    assert rel(host(b), c256["b"]) < 1e-13
    p = s.solve(b)
    p_o, _, nc_o, _, _ = c256["iter"]
    assert s.last_stats.cycles == nc_o
    assert rel(host(p), p_o) < 1e-12


@pytest.mark.parametrize("prec,inner,method", [("mixed", 1, "vcycle"), ("mixed_df", 1, "vcycle"),
                                               ("mixed", 2, "vcycle"), ("mixed_df", 2, "vcycle"),
                                               ("mixed", 4, "vcycle"), ("mixed_df", 4, "vcycle"),
                                               ("mixed", 0, "vcycle"), ("mixed_df", 0, "vcycle"),
                                               ("mixed", 4, "fcg"), ("mixed_df", 4, "fcg")])
def test_256_mixed_reaches_exact_solution(c256, prec, inner, method):
    s, _ = gpu_solver(c256, prec, 1e-11, inner, method)
    p = s.solve(s.rhs(u=c256["u"]))
    assert s.last_stats.relres <= 1e-11
    assert rel(host(p), c256["exact"]) <= 1e-9
    # at rtol 1e-10 the iteration error of V(2,2) itself dominates: compare with the oracle's
    # own iteration stopped at the same tolerance (both sit ~1.6e-9 from the exact solution)
    s.close()
    s, _ = gpu_solver(c256, prec, 1e-10, inner, method)
    p = host(s.solve(s.rhs(u=c256["u"])))
    p_o, _, nc_o, _, _ = c256["iter"]
    if method == "vcycle":  # the same iteration as the oracle's
        assert nc_o - 1 <= s.last_stats.cycles <= nc_o + (inner if inner else 2)
        if s.last_stats.cycles <= nc_o + 1:  # stopped at the oracle's cycle (or one later): its iterate
            assert rel(p, p_o) <= 1e-9
    else:  # another iteration: fewer V-cycles, its own iterate
        assert s.last_stats.cycles < nc_o
    assert rel(p, c256["exact"]) <= 3e-9


BOX = 20
# sub-box origins (x, y, z) with x + y + z even, so the colours agree with the full grid:
# a corner, the interior (through the drop), two boxes touching the high walls
ORIGINS = [(0, 0, 0), (246, 250, 310), (492, 0, 300), (100, 492, 492)]


def interior_mask(o, n):
    """Cells of the box at distance >= 2 from every box face that lies inside the grid."""
    m = np.ones((BOX,) * 3, bool)
    for ax, lo in zip((2, 1, 0), o):  # array axes are (z, y, x)
        sl = [slice(None)] * 3
        if lo > 0:
            sl[ax] = slice(0, 2)
            m[tuple(sl)] = False
        if lo + BOX < n:
            sl[ax] = slice(BOX - 2, BOX)
            m[tuple(sl)] = False
    return m


@pytest.mark.parametrize("prec,dtype", [("mixed", torch.float32), ("fp64", torch.float64)])
def test_512_level0_sweep_on_subboxes(prec, dtype):
    n = 512
    h = 1.0 / n
    g = D.scaled_geometry(n)
    fd, ff = D.fractions_ramp(g, device=torch.device("cuda"))
    s = Solver((n,) * 3, h=h, precision=prec, coarsest=8)
    rho = s.density_from_fractions([fd, ff], list(RHO_PHASE))
    s.set_density(rho)
    gen = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn((n,) * 3, generator=gen, device="cuda", dtype=dtype)
    b = torch.randn((n,) * 3, generator=gen, device="cuda", dtype=dtype)
    x0 = x.clone()
    assert L.mg_smooth(s._h, 0, x, b, 1, 0) == 0
    rho_h = host(rho)
    for o in ORIGINS:
        sl = (slice(o[2], o[2] + BOX), slice(o[1], o[1] + BOX), slice(o[0], o[0] + BOX))
        faces = O.faces_from_density(rho_h[sl])
        if dtype == torch.float32:  # the oracle sees the FP32-rounded coefficients
            faces = tuple(f.astype(np.float32).astype(np.float64) for f in faces)
        want = O.rbgs(faces, host(b[sl]), host(x0[sl]), h, 1, 0)
        m = interior_mask(o, n)
        got = host(x[sl])
        tol = 2e-6 if dtype == torch.float32 else 1e-13
        assert rel(got[m], want[m]) < tol, o


@pytest.mark.parametrize("prec,inner,method", [("mixed", 1, "vcycle"), ("mixed_df", 1, "vcycle"),
                                               ("mixed", 2, "vcycle"), ("mixed_df", 2, "vcycle"),
                                               ("mixed", 4, "vcycle"), ("mixed", 0, "vcycle"), ("mixed", 4, "fcg"),
                                               ("fp64", 1, "fcg")])
def test_512_benchmark_solve_and_adjoint(prec, inner, method):
    c = fields(512)
    h = c["h"]
    s, _ = gpu_solver(c, prec, 1e-10, inner, method)
    b = s.rhs(u=c["u"])
    assert rel(host(b), c["b"]) < 1e-13
    p = s.solve(b)
    assert s.last_stats.relres <= 1e-10
    ph = host(p)
    nb = np.linalg.norm(c["b"] - c["b"].mean())
    # the oracle's FP64 residual of the returned p (the two sides sum in different orders)
    assert np.linalg.norm(O.residual(c["faces"], c["b"], ph, h)) / nb <= 1.05e-10
    assert abs(ph.mean()) <= 1e-14 * np.abs(ph).max()
    w = D.normal_weights((512,) * 3, seed=1, device=torch.device("cuda"))
    lam, g, _ = s.adjoint(w, p)
    lh, wh = host(lam), host(w)
    assert np.linalg.norm(O.residual(c["faces"], wh - wh.mean(), lh, h)) / np.linalg.norm(wh - wh.mean()) <= 1.05e-10
    g_o, _ = O.adjoint_grads(c["faces"], lh, ph, h)
    for gg, go in zip(g, g_o):
        assert rel(host(gg), go) < 1e-6


def test_512_projection_and_density_adjoint():
    """The benchmark's step at 512^3 (mixed, adaptive inner cycles) followed by the velocity correction
    and the density adjoint, compared with the oracle on every face and cell: the projection
    to 1e-14 of the largest velocity, with zero divergence up to the solve's residual; dL/drho
    and dL/df_q within the FP32 rounding bound of the same gradients (tests/test_gpu_project.py
    derives it)."""
    from test_gpu_project import _density_bound

    c = fields(512)
    h = c["h"]
    s, rho = gpu_solver(c, "mixed", 1e-10, 0)
    b = s.rhs(u=c["u"])
    p = s.solve(b)
    u_h = [host(a) for a in c["u"]]
    s.project(p, c["u"])
    want = O.project(u_h, c["faces"], host(p), h)
    for a, wnt in zip(c["u"], want):
        assert np.abs(host(a) - wnt).max() <= 1e-14 * np.abs(wnt).max()
    del want
    div = O.divergence([host(a) for a in c["u"]], h)
    nb = np.linalg.norm(c["b"] - c["b"].mean())
    assert np.linalg.norm(div - c["b"].mean()) <= 1.05 * s.last_stats.relres * nb + 1e-12 * nb
    del div
    w = D.normal_weights((512,) * 3, seed=1, device=torch.device("cuda"))
    _, g, _ = s.adjoint(w, p)
    drho, dfrac = s.density_grads(rho, g, RHO_PHASE)
    gh = [host(a) for a in g]
    rh = c["rho"]
    d_o, f_o = O.density_grads(rh, gh, RHO_PHASE)
    assert np.all(np.abs(host(drho) - d_o) <= _density_bound(rh, gh))
    for got, want_q, dr in zip(dfrac, f_o, (998.0 - 1.2, 880.0 - 1.2)):
        assert np.all(np.abs(host(got) - want_q) <= _density_bound(rh, gh, 2.0) * dr)
