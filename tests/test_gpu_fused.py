"""Fused red-black sweeps of the finest level (shared-memory staging by bulk copies).

The fused sweep evaluates every cell update with the arithmetic of the half-sweep kernels,
so it must reproduce two half sweeps bitwise: checked through the smoothing components
(mg_smooth, mg_presmooth_restrict, mg_prolong_postsmooth) on grids whose tiles are partial in
y and z and split in x, and through whole solves (the same cycle count, bitwise the same p).
The half-sweep path itself is checked against the oracle elsewhere (test_gpu_components,
test_gpu_fullsize)."""
import numpy as np
import pytest
import torch

from paper_2605_30082_gb300 import Solver
from paper_2605_30082_gb300 import _lib as L

from _helpers import RHO_PHASE, dev, dropfilm_case, host, random_rho

pytestmark = pytest.mark.gpu

# (nx, ny, nz): nx % 128 == 0 (fused path); ny = 4, 12 give partial 8-row tiles; nz = 16, 80
# partial 64-plane chunks; nx = 256 two tiles in x
DIMS = [(128, 4, 64), (128, 12, 16), (256, 24, 80), (256, 48, 80)]


def pair(dims, seed):
    out = []
    rho = dev(random_rho(dims, seed))
    for fused in (True, False):
        s = Solver(dims, precision="mixed", coarsest=8, fused_sweeps=fused)
        s.set_density(rho)
        out.append(s)
    return out


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("sweeps", [1, 2, 3, 4])
@pytest.mark.parametrize("order", [0, 1])
def test_smooth_bitwise(dims, sweeps, order):
    sf, sh = pair(dims, 11)
    g = torch.Generator(device="cuda").manual_seed(3)
    shape = (dims[2], dims[1], dims[0])
    x0 = torch.randn(shape, generator=g, device="cuda", dtype=torch.float32)
    b = torch.randn(shape, generator=g, device="cuda", dtype=torch.float32)
    xf, xh = x0.clone(), x0.clone()
    assert L.mg_smooth(sf._h, 0, xf, b, sweeps, order) == 0
    assert L.mg_smooth(sh._h, 0, xh, b, sweeps, order) == 0
    torch.cuda.synchronize()
    assert torch.equal(xf, xh)
    assert not torch.equal(xf, x0)


@pytest.mark.parametrize("dims", DIMS)
def test_cycle_steps_bitwise(dims):
    """The V-cycle's fused steps: pre-smoothing from zero + restriction, prolongation +
    post-smoothing."""
    sf, sh = pair(dims, 12)
    nx, ny, nz = dims
    g = torch.Generator(device="cuda").manual_seed(4)
    b = torch.randn((nz, ny, nx), generator=g, device="cuda", dtype=torch.float32)
    cshape = (nz // 2, ny // 2, nx // 2)
    res = []
    for s in (sf, sh):
        x = torch.full((nz, ny, nx), float("nan"), device="cuda")
        bc = torch.empty(cshape, device="cuda")
        assert L.mg_presmooth_restrict(s._h, 0, x, b, 2, bc, x_is_zero=True) == 0
        ec = torch.randn(cshape, generator=torch.Generator(device="cuda").manual_seed(5), device="cuda")
        x2 = x.clone()
        assert L.mg_prolong_postsmooth(s._h, 0, ec, x2, b, 2) == 0
        res.append((x, bc, x2))
    torch.cuda.synchronize()
    for a, c in zip(*res):
        assert torch.equal(a, c)


@pytest.mark.parametrize("prec,inner", [("mixed", 1), ("mixed", 2), ("mixed", 3), ("mixed_df", 2)])
def test_solve_bitwise_256(prec, inner):
    c = dropfilm_case(256)
    rho = dev(c["rho"])
    b = dev(c["b"])
    ps, cyc = [], []
    for fused in (True, False):
        s = Solver((256,) * 3, h=c["h"], precision=prec, coarsest=8, inner_cycles=inner, fused_sweeps=fused)
        s.set_density(rho)
        ps.append(s.solve(b))
        cyc.append(s.last_stats.cycles)
        s.close()
    assert cyc[0] == cyc[1]
    assert torch.equal(ps[0], ps[1])


def test_fused_sweeps_option_validated():
    o = L.mg_default_opts()
    assert o.fused_sweeps == 0
    o.nx = o.ny = o.nz = 16
    o.fused_sweeps = 2
    st, h = L.mg_create(o, torch.cuda.current_stream())
    assert st == L.MG_ERR_ARG
