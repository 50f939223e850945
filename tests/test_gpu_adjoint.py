"""Adjoint path: mg_adjoint and the PoissonSolve autograd Function.

Checked against (a) the oracle's adjoint formulas evaluated at the oracle's
own exact lambda and p, and (b) central finite differences of the GPU forward
solve (FP64, solves to 1e-13) along random directions.  L = sum(w * p),
w ~ N(0, 1) from seed 1.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_30082_gb300 import PoissonSolve, Solver

from _helpers import csf_case, dev, host, random_rho, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_df"])
def test_adjoint_matches_oracle_32cubed(prec):
    c = csf_case(32)
    h, sigma = c["h"], 0.03
    b = O.rhs([a.numpy() for a in c["u"]], c["faces"], h, csf=c["csf"], sigma=sigma)
    M = O.Multigrid(c["faces"], h, coarsest=8)
    p_o = M.solve_exact(b)[0]
    lam_o = M.solve_exact(c["w"])[0]
    g_o, ds_o = O.adjoint_grads(c["faces"], lam_o, p_o, h, csf=c["csf"], sigma=sigma)

    s = Solver((32, 32, 32), h=h, precision=prec, coarsest=8)
    s.set_density(dev(c["rho"]))
    csf = tuple(dev(a) for a in c["csf"])
    bg = s.rhs(u=tuple(a.cuda() for a in c["u"]), csf=csf, sigma=sigma)
    assert rel(host(bg), b) < 1e-13
    p = s.solve(bg)
    lam, g, ds = s.adjoint(dev(c["w"]), p, csf=csf, sigma=sigma)
    assert s.last_stats.relres <= 1e-10
    assert rel(host(lam), lam_o) < 1e-9
    for gg, go in zip(g, g_o):
        assert gg.dtype == torch.float32
        assert rel(host(gg), go) < 1e-6
    assert abs(ds - ds_o) <= 1e-8 * abs(ds_o)


@pytest.mark.parametrize("dims,prec", [((32, 32, 32), "mixed"), ((48, 40, 72), "mixed"), ((40, 24, 36), "fp64"),
                                       ((96, 64, 80), "mixed_df"), ((136, 40, 72), "mixed"), ((21, 8, 6), "fp64")])
def test_face_gradients_without_surface_term_every_face(dims, prec):
    """Without a CSF term the face gradients come from FP32 pairs (no FP64 arithmetic): every
    face against the oracle's formula at the GPU's own lambda and p, within a few FP32 units
    (plus 1e-10 of the largest gradient for the pairs' 47-bit cancellation limit).
    Grids whose rows are not multiples of the warp's 64 cells (two per lane), of the 16-row
    tile and of the 32-plane z-run cover the ragged edges; an odd nx takes the one-cell-per-lane
    kernel."""
    nx, ny, nz = dims
    h = 1.0 / max(dims)
    rho = random_rho(dims, 17)
    faces = O.faces_from_density(rho)
    s = Solver(dims, h=h, precision=prec, coarsest=8)
    s.set_density(dev(rho))
    rng = np.random.default_rng(3)
    p = s.solve(dev(rng.standard_normal((nz, ny, nx))))
    lam, g, ds = s.adjoint(dev(rng.standard_normal((nz, ny, nx))), p)
    assert ds == 0.0
    g_o, _ = O.adjoint_grads(faces, host(lam), host(p), h)
    for gg, go in zip(g, g_o):
        got = host(gg)
        scale = np.abs(go).max()
        assert np.all(np.abs(got - go) <= 6 * 2.0**-24 * np.abs(go) + 1e-10 * scale)
    # the walls are zero
    assert not host(g[0])[:, :, [0, -1]].any() and not host(g[1])[:, [0, -1], :].any()
    assert not host(g[2])[[0, -1]].any()


def test_autograd_function_and_finite_differences_64cubed():
    """The BJ-style check on a 64^3 copy: central FD (eps 1e-6, FP64) of the forward solve."""
    n = 64
    c = csf_case(n)
    h = c["h"]
    s = Solver((n, n, n), h=h, precision="fp64", coarsest=8, rtol=1e-13, max_cycles=400)
    faces = [dev(f).requires_grad_(True) for f in c["faces"]]
    b_u = dev(c["b"]).requires_grad_(True)
    csf = tuple(dev(a) for a in c["csf"])
    sigma = torch.tensor(0.03, dtype=torch.float64, device="cuda", requires_grad=True)
    w = dev(c["w"])
    p = PoissonSolve.apply(s, b_u, *faces, sigma, csf)
    loss = (w * p).sum()
    loss.backward()

    def L(fs, bu, sg):
        with torch.no_grad():
            return float((w * PoissonSolve.apply(s, bu, *fs, sg, csf)).sum())

    rng = np.random.default_rng(11)
    # direction on the interior faces, scaled relative to beta
    base = [f.detach() for f in faces]
    dirs = []
    for f, axis in zip(base, (2, 1, 0)):
        v = torch.tensor(rng.standard_normal(f.shape), device="cuda") * f
        dirs.append(v)
    eps = 1e-6
    fp = [f + eps * v for f, v in zip(base, dirs)]
    fm = [f - eps * v for f, v in zip(base, dirs)]
    fd = (L(fp, b_u.detach(), 0.03) - L(fm, b_u.detach(), 0.03)) / (2 * eps)
    ad = sum(float((f.grad.double() * v).sum()) for f, v in zip(faces, dirs))
    assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
    # dL/db along a random cell direction
    vb = torch.tensor(rng.standard_normal((n, n, n)), device="cuda")
    fdb = (L(base, b_u.detach() + 1e-3 * vb, 0.03) - L(base, b_u.detach() - 1e-3 * vb, 0.03)) / 2e-3
    adb = float((b_u.grad * vb).sum())
    assert abs(fdb - adb) <= 1e-7 * abs(adb)
    # dL/dsigma: L is linear in sigma
    fds = (L(base, b_u.detach(), 0.03 + 1e-4) - L(base, b_u.detach(), 0.03 - 1e-4)) / 2e-4
    assert abs(fds - float(sigma.grad)) <= 1e-6 * abs(fds)
    # dL/db is the zero-mean adjoint solution
    assert abs(float(b_u.grad.mean())) < 1e-12 * float(b_u.grad.abs().max())


def test_backward_recomputes_operator_after_another_set():
    n = 32
    c = csf_case(n)
    s = Solver((n, n, n), h=c["h"], precision="mixed", coarsest=8)
    faces = [dev(f).requires_grad_(True) for f in c["faces"]]
    b_u = dev(c["b"]).requires_grad_(True)
    p = PoissonSolve.apply(s, b_u, *faces)
    # load a different operator into the same handle before backward
    s.set_density(dev(np.ones((n, n, n))))
    (dev(c["w"]) * p).sum().backward()
    lam_o = O.Multigrid(c["faces"], c["h"], coarsest=8).solve_exact(c["w"])[0]
    assert rel(host(b_u.grad), lam_o) < 1e-9
