"""Failure paths, driven by one-shot faults armed on the host (mg_debug_inject); no GPU fault.

- A fused sweep's bounded mbarrier wait that runs out: one block announces a plane's bytes but
  issues no copy for it, waits about a second, records bit 4 of the device error word, drains
  its other copies and returns.  mg_solve must report MG_ERR_CUDA, clear the error word, and
  the next solve on the same handle must give bitwise the result of a clean solve.
- A lost residual norm (infinity read back) must end the solve with MG_ERR_DIVERGED, and the
  handle must solve normally afterwards.
"""
import pytest
import torch

from paper_2605_30082_gb300 import MgError, Solver
from paper_2605_30082_gb300 import _lib as L

from _helpers import dev, random_rho

pytestmark = pytest.mark.gpu


def _rhs(dims, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    nx, ny, nz = dims
    return torch.randn((nz, ny, nx), generator=g, device="cuda", dtype=torch.float64)


def test_fused_sweep_wait_runs_out_and_handle_recovers():
    dims = (128, 16, 32)
    s = Solver(dims, precision="mixed", coarsest=8, fused_sweeps=True, max_cycles=200)
    s.set_density(dev(random_rho(dims, 5)))
    b = _rhs(dims, 1)
    p_ref = s.solve(b).clone()
    assert L.mg_debug_inject(s._h, L.MG_INJECT_FUSED_WAIT) == L.MG_OK
    with pytest.raises(MgError) as ei:
        s.solve(b)
    assert ei.value.code == L.MG_ERR_CUDA
    assert "gave up waiting" in str(ei.value)
    # the error word was cleared: the same handle solves as before, bitwise
    p = s.solve(b)
    assert s.last_stats.status == L.MG_OK
    assert torch.equal(p, p_ref)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lost_residual_norm_reports_diverged(prec):
    dims = (32, 32, 32)
    s = Solver(dims, precision=prec, coarsest=8)
    s.set_density(dev(random_rho(dims, 6)))
    b = _rhs(dims, 2)
    p_ref = s.solve(b).clone()
    assert L.mg_debug_inject(s._h, L.MG_INJECT_DIVERGE) == L.MG_OK
    with pytest.raises(MgError) as ei:
        s.solve(b)
    assert ei.value.code == L.MG_ERR_DIVERGED
    assert s.last_stats.status == L.MG_ERR_DIVERGED
    p = s.solve(b)  # one-shot: the next solve is clean
    assert torch.equal(p, p_ref)
    s.close()


def test_inject_rejects_unknown_faults():
    s = Solver((16, 16, 16), precision="mixed", coarsest=8)
    assert L.mg_debug_inject(s._h, 8) == L.MG_ERR_ARG
    assert L.mg_debug_inject(s._h, 0) == L.MG_OK
    s.close()
