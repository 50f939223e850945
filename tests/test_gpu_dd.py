"""The slab-decomposed FP64 V-cycle (mg_dd_*) against the whole-grid one, on the GPU.

Every cell of a slab sees the arithmetic of the whole-grid FP64 V-cycle in the same order (the
ghost planes hold the neighbours' values, the faces between slabs count as interior), so one
decomposed V-cycle must equal bitwise the whole-grid V-cycle assembled from the FP64 component
entry points (mg_presmooth_restrict, mg_coarse_solve, mg_prolong_postsmooth), for 1 to 8 slabs,
with the switch to the whole-grid levels at every allowed level, both prolongations and other
sweep counts.  The decomposed solve differs from the whole-grid one only in the order of its
norm and mean sums: same cycle count, p within 1e-12; and it reaches the oracle's exact
discrete solution.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_30082_gb300 import Solver
from paper_2605_30082_gb300 import _lib as L

from _helpers import RHO_PHASE, dev, dropfilm_case, host, random_rho, rel

pytestmark = pytest.mark.gpu


def _opts(dims, h, coarsest=4, pre=2, post=2, prolong=L.MG_PROLONG_TRILINEAR, rtol=1e-10):
    o = L.mg_default_opts()
    o.nx, o.ny, o.nz = dims
    o.h = h
    o.precision = L.MG_FP64
    o.coarsest, o.pre, o.post, o.prolong, o.rtol = coarsest, pre, post, prolong, rtol
    o.max_cycles = 200
    return o


class DD:
    def __init__(self, dims, ranks, max_dec=0, **kw):
        self.dims = dims
        st, self.h = L.mg_dd_create(_opts(dims, **kw), ranks, max_dec)
        assert st == L.MG_OK, st
        st, self.plan = L.mg_dd_get_plan(self.h)
        assert st == L.MG_OK

    def close(self):
        L.mg_dd_destroy(self.h)


def whole_vcycle(s, b, x):
    """The whole-grid FP64 V-cycle from x, by the component entry points."""
    nl = s.num_levels
    B, X = [b], [x]
    for l in range(1, nl):
        nx, ny, nz = s.level_dims(l)
        B.append(torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda"))
        X.append(torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda"))

    def cyc(l, zero):
        if l == nl - 1:
            assert L.mg_coarse_solve(s._h, B[l], X[l]) == L.MG_OK
            return
        assert L.mg_presmooth_restrict(s._h, l, X[l], B[l], s.opts.pre, B[l + 1], x_is_zero=zero) == L.MG_OK
        cyc(l + 1, True)
        assert L.mg_prolong_postsmooth(s._h, l, X[l + 1], X[l], B[l], s.opts.post) == L.MG_OK

    cyc(0, False)


CASES = [((64, 64, 64), 1, 0, {}), ((64, 64, 64), 2, 0, {}), ((64, 64, 64), 4, 0, {}),
         ((64, 48, 128), 8, 0, {}), ((64, 48, 128), 8, 1, {}), ((64, 48, 128), 4, 2, {}),
         ((64, 64, 32), 4, 0, {}), ((48, 40, 64), 4, 0, dict(prolong=L.MG_PROLONG_CONSTANT)),
         ((48, 40, 64), 2, 0, dict(pre=1, post=3)), ((64, 32, 64), 2, 0, dict(pre=0, post=2, coarsest=8))]


@pytest.mark.parametrize("dims,ranks,max_dec,kw", CASES)
def test_dd_vcycle_is_bitwise_the_whole_grid_vcycle(dims, ranks, max_dec, kw):
    nx, ny, nz = dims
    h = 1.0 / max(dims)
    rho = dev(random_rho(dims, 31))
    o = _opts(dims, h, **kw)
    s = Solver(dims, h=h, precision="fp64", coarsest=o.coarsest, pre=o.pre, post=o.post,
               prolong="constant" if o.prolong == L.MG_PROLONG_CONSTANT else "trilinear")
    s.set_density(rho)
    dd = DD(dims, ranks, max_dec, h=h, **kw)
    assert L.mg_dd_set_density(dd.h, rho, dims) == L.MG_OK
    assert dd.plan.levels == s.num_levels
    g = torch.Generator(device="cuda").manual_seed(4)
    b = torch.randn((nz, ny, nx), generator=g, device="cuda", dtype=torch.float64)
    x0 = torch.randn((nz, ny, nx), generator=g, device="cuda", dtype=torch.float64)
    for _ in range(2):  # a second cycle continues from the first
        xw = x0.clone()
        whole_vcycle(s, b, xw)
        xd = x0.clone()
        assert L.mg_dd_vcycle(dd.h, b, xd, dims) == L.MG_OK, L.mg_dd_last_error(dd.h)
        torch.cuda.synchronize()
        assert torch.equal(xd, xw), (dims, ranks, max_dec, float((xd - xw).abs().max()))
        x0 = xw
    st, ex, by = L.mg_dd_traffic(dd.h)
    k = 2 * o.pre + 2 * o.post + 1
    assert ex == k * dd.plan.switch_level
    assert by == sum(k * 2 * (ranks - 1) * 8 * dd.plan.nx[l] * dd.plan.ny[l] for l in range(dd.plan.switch_level))
    dd.close()
    s.close()


@pytest.mark.parametrize("ranks,max_dec", [(2, 0), (4, 0), (8, 1)])
def test_dd_solve_matches_whole_grid_and_oracle(ranks, max_dec):
    n = 64
    c = dropfilm_case(n)
    dims = (n, n, n)
    rho = dev(c["rho"])
    b = dev(c["b"])
    s = Solver(dims, h=c["h"], precision="fp64", coarsest=4, rtol=1e-11)
    s.set_density(rho)
    pw = s.solve(b)
    dd = DD(dims, ranks, max_dec, h=c["h"], rtol=1e-11)
    assert L.mg_dd_set_density(dd.h, rho, dims) == L.MG_OK
    pd = torch.zeros_like(b)
    st = L.mg_stats()
    assert L.mg_dd_solve(dd.h, b, pd, dims, st) == L.MG_OK, L.mg_dd_last_error(dd.h)
    assert st.relres <= 1e-11
    assert st.cycles == s.last_stats.cycles
    assert rel(host(pd), host(pw)) <= 1e-12
    assert abs(float(pd.mean())) <= 1e-14 * float(pd.abs().max())
    p_ex = O.Multigrid(c["faces"], c["h"], coarsest=4).solve_exact(c["b"])[0]
    assert rel(host(pd), p_ex) <= 1e-9
    dd.close()
    s.close()


def test_dd_errors():
    dims = (32, 32, 32)
    o = _opts(dims, 1 / 32)
    o.precision = L.MG_MIXED_DF
    assert L.mg_dd_create(o, 2)[0] == L.MG_ERR_ARG           # FP64 or MG_MIXED only
    assert L.mg_dd_create(_opts(dims, 1 / 32), 32)[0] == L.MG_ERR_ARG  # one plane per slab
    dd = DD(dims, 2, h=1 / 32)
    b = torch.zeros((32, 32, 32), dtype=torch.float64, device="cuda")
    assert L.mg_dd_solve(dd.h, b, b.clone(), dims) == L.MG_ERR_STATE  # no operator yet
    bad = torch.ones_like(b)
    bad[3, 4, 5] = -1.0
    assert L.mg_dd_set_density(dd.h, bad, dims) == L.MG_ERR_DENSITY
    dd.close()


def test_dd_solve_at_512_in_four_slabs():
    """The benchmark's 512^3 drop-on-film field, FP64 to rtol 1e-10, cut into 4 slabs: the same
    V-cycles as the whole-grid FP64 solve and the same pressure up to the order of the sums."""
    import dropfilm as D

    n = 512
    dims = (n, n, n)
    cuda = torch.device("cuda")
    g = D.scaled_geometry(n)
    fd, ff = D.fractions_ramp(g, device=cuda, z_chunk=32)
    u = D.face_velocities(n, 0, device=cuda, z_chunk=32)
    s = Solver(dims, h=1.0 / n, precision="fp64", coarsest=8, rtol=1e-10)
    rho = s.density_from_fractions([fd, ff], list(RHO_PHASE))
    s.set_density(rho)
    b = s.rhs(u=u)
    pw = s.solve(b)
    cycles = s.last_stats.cycles
    s.close()
    dd = DD(dims, 4, h=1.0 / n, coarsest=8, rtol=1e-10)
    assert L.mg_dd_set_density(dd.h, rho, dims) == L.MG_OK
    pd = torch.zeros_like(b)
    st = L.mg_stats()
    assert L.mg_dd_solve(dd.h, b, pd, dims, st) == L.MG_OK, L.mg_dd_last_error(dd.h)
    assert st.cycles == cycles
    rel_t = float(torch.linalg.vector_norm(pd - pw) / torch.linalg.vector_norm(pw))
    assert rel_t <= 1e-12, rel_t
    dd.close()


def _mixed_opts(dims, h, inner, rtol=1e-11, **kw):
    o = _opts(dims, h, rtol=rtol, **kw)
    o.precision = L.MG_MIXED
    o.inner_cycles = inner
    return o


def _same_as_whole_grid(sd, sw, pd, pw):
    """Every cell of the decomposed mixed solve sees the whole-grid arithmetic; what differs is
    the outer loop's sums.  Its residual kernel accumulates r^2 and p in FP32 per thread over a
    grid-stride share of the cells, and the slabs share the cells out differently: the norms
    agree to FP32 rounding (1e-6 relative with margin), and the per-iteration shift, which comes
    from the sum of p, moves the iterates by about 1e-14 of p, which the later, smaller residuals
    see as an absolute difference below 1e-10 of the first one.  The pressure agrees to 1e-13."""
    hd, hw = np.array(sd.history()), np.array(sw.history())
    assert np.allclose(hd, hw, rtol=1e-6, atol=1e-10), (hd, hw)
    assert rel(host(pd), host(pw)) <= 1e-13


@pytest.mark.parametrize("ranks,inner,max_dec", [(2, 1, 0), (4, 1, 0), (2, 3, 0), (4, 0, 0), (2, 0, 1), (4, 3, 1)])
def test_dd_mixed_solve_matches_whole_grid_and_oracle(ranks, inner, max_dec):
    """The mixed solve with its levels down to 16^3 cut into slabs (FP32 slab kernels with ghost
    planes, the coarser levels on one whole-grid handle, the FP64 outer loop slab by slab) follows the
    whole-grid mixed solve (the same V-cycles and outer iterations; residual histories and p
    as close as the outer loop's sums allow), and it reaches the oracle's exact discrete
    solution."""
    n = 64
    c = dropfilm_case(n)
    dims = (n, n, n)
    rho = dev(c["rho"])
    b = dev(c["b"])
    s = Solver(dims, h=c["h"], precision="mixed", coarsest=4, rtol=1e-11, inner_cycles=inner)
    s.set_density(rho)
    pw = s.solve(b)
    st, h = L.mg_dd_create(_mixed_opts(dims, c["h"], inner), ranks, max_dec)
    assert st == L.MG_OK, st
    st, plan = L.mg_dd_get_plan(h)
    # as deep as allowed, down to 16^3 (the prolongation into a cut level needs coarse rows of a
    # multiple of 8 cells), or the finest level only
    assert plan.switch_level == (max_dec or 3), plan.switch_level
    assert L.mg_dd_set_density(h, rho, dims) == L.MG_OK
    pd = torch.zeros_like(b)
    sts = L.mg_stats()
    assert L.mg_dd_solve(h, b, pd, dims, sts) == L.MG_OK, L.mg_dd_last_error(h)
    assert sts.relres <= 1e-11
    assert (sts.cycles, sts.outer) == (s.last_stats.cycles, s.last_stats.outer)
    _same_as_whole_grid(sts, s.last_stats, pd, pw)
    assert abs(float(pd.mean())) <= 1e-14 * float(pd.abs().max())
    p_ex = O.Multigrid(c["faces"], c["h"], coarsest=4).solve_exact(c["b"])[0]
    assert rel(host(pd), p_ex) <= 1e-9
    _, ex, by = L.mg_dd_traffic(h)
    k = 2 * 2 + 2 * 2 + 1
    assert ex == k * plan.switch_level
    assert by == sum(k * 2 * (ranks - 1) * 4 * (plan.nx[l] // 2) * plan.ny[l] for l in range(plan.switch_level))
    L.mg_dd_destroy(h)
    s.close()


def test_dd_mixed_rejects_what_it_does_not_cut():
    dims = (64, 64, 64)
    h = 1 / 64
    for kw, ranks in ((dict(pre=0), 2), (dict(post=0), 2), (dict(prolong=L.MG_PROLONG_CONSTANT), 2), ({}, 32)):
        assert L.mg_dd_create(_mixed_opts(dims, h, 1, **kw), ranks)[0] == L.MG_ERR_ARG, (kw, ranks)
    assert L.mg_dd_create(_mixed_opts((72, 64, 64), h, 1), 2)[0] == L.MG_ERR_ARG  # nx not a multiple of 16
    assert L.mg_dd_create(_mixed_opts((64, 64, 40), h, 1), 4)[0] == L.MG_ERR_ARG  # 10 planes per slab
    o = _mixed_opts(dims, h, 1)
    o.precision = L.MG_MIXED_DF
    assert L.mg_dd_create(o, 2)[0] == L.MG_ERR_ARG
    st, hd = L.mg_dd_create(_mixed_opts(dims, h, 1), 2)
    assert st == L.MG_OK
    b = torch.zeros(dims, dtype=torch.float64, device="cuda")
    assert L.mg_dd_vcycle(hd, b, b.clone(), dims) == L.MG_ERR_ARG  # FP64 decompositions only
    L.mg_dd_destroy(hd)


def test_dd_mixed_slabs_on_the_staged_sweep():
    """Slabs large enough for the staged half sweep (k_half_zs in its ghost variant: 320 rows
    x 4 sixteen-plane chunks per slab launch) follow the whole-grid mixed solve as closely as
    the small ones do."""
    dims = (256, 320, 128)
    nx, ny, nz = dims
    h = 1.0 / 256
    rho = dev(random_rho(dims, 23))
    g = torch.Generator(device="cuda").manual_seed(5)
    b = torch.randn((nz, ny, nx), generator=g, device="cuda", dtype=torch.float64)
    s = Solver(dims, h=h, precision="mixed", coarsest=8, rtol=1e-10, inner_cycles=0)
    s.set_density(rho)
    pw = s.solve(b)
    st, hd = L.mg_dd_create(_mixed_opts(dims, h, 0, rtol=1e-10, coarsest=8), 2, 0)
    assert st == L.MG_OK, st
    assert L.mg_dd_set_density(hd, rho, dims) == L.MG_OK
    pd = torch.zeros_like(b)
    sts = L.mg_stats()
    assert L.mg_dd_solve(hd, b, pd, dims, sts) == L.MG_OK, L.mg_dd_last_error(hd)
    assert (sts.cycles, sts.outer) == (s.last_stats.cycles, s.last_stats.outer)
    _same_as_whole_grid(sts, s.last_stats, pd, pw)
    L.mg_dd_destroy(hd)
    s.close()
