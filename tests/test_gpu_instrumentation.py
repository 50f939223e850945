"""Instrumentation entry points: the FP64 FMA rate (the FP64 rooflines' denominator), the
per-class kernel timing (finest-level kernels, the levels below as one interval per V-cycle,
the set-up calls) and the launch counter."""
import pytest
import torch

from paper_2605_30082_gb300 import Solver
from paper_2605_30082_gb300 import _lib as L

from _helpers import dev, random_rho

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_measured_and_plausible():
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.empty(8 * n_sm, dtype=torch.float64, device="cuda")
    l0 = L.mg_kernel_launches()
    st, tf, ms = L.mg_fp64_fma_rate(sink, 2000)
    assert st == L.MG_OK
    assert L.mg_kernel_launches() - l0 == 2  # one untimed, one timed launch
    assert ms > 0.0
    # GB300: about 1.26 TFLOP/s FP64 at 2070 MHz; far outside this band the kernel did not run
    assert 0.3 < tf < 3.0, tf
    assert torch.isfinite(sink).all()
    # bad arguments are refused on the host
    assert L.lib().mg_fp64_fma_rate(None, None, 8, 10, None, None) == L.MG_ERR_ARG
    st, _, _ = L.mg_fp64_fma_rate(sink, 0)
    assert st == L.MG_ERR_ARG


def test_profile_classes_count_the_finest_level_launches():
    dims = (64, 64, 64)
    s = Solver(dims, precision="mixed", coarsest=8, inner_cycles=1)
    s.set_density(dev(random_rho(dims, 2)))
    b = torch.randn((64, 64, 64), dtype=torch.float64, device="cuda")
    s.profile(True)
    s.solve(b)
    cycles, outer = s.last_stats.cycles, s.last_stats.outer
    n_upd, ms_upd = s.profile_read(L.MG_PROF_UPDATE)
    n_res, ms_res = s.profile_read(L.MG_PROF_FINE_RESIDUAL)
    n_sm, ms_sm = s.profile_read(L.MG_PROF_SMOOTH)
    assert n_upd == outer  # one fused update per outer iteration
    assert n_res == outer  # one per outer iteration (a cold start's opening residual is b~ itself)
    assert n_sm == cycles * 8 - outer  # V(2,2): 8 half sweeps, the last one carries the update
    assert ms_upd > 0 and ms_res > 0 and ms_sm > 0
    n_cl, ms_cl = s.profile_read(L.MG_PROF_COARSE_LEVELS)
    assert n_cl == cycles and ms_cl > 0  # one interval per V-cycle below the finest level
    s.profile(False)
    assert s.profile_read(L.MG_PROF_SMOOTH) == (0, 0.0)
    # the grouped classes around the set-up calls: one interval per call
    s.profile(True)
    fr = [torch.full((64, 64, 64), 0.3, dtype=torch.float64, device="cuda") for _ in range(2)]
    rho = s.density_from_fractions(fr, [998.0, 880.0, 1.2])
    s.set_density(rho)
    s.set_density(rho)
    s.rhs(b0=b)
    for cls, k in ((L.MG_PROF_DENSITY, 1), (L.MG_PROF_SETUP, 2), (L.MG_PROF_RHS, 1)):
        n_k, ms_k = s.profile_read(cls)
        assert n_k == k and ms_k > 0, (cls, n_k, ms_k)
    s.profile(False)
    s.close()
