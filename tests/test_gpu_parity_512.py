"""Parity gate at the benchmark's size: 512^3 drop-on-film, against the oracle's exact solution.

The oracle runs its FP64 V-cycle to rtol 1e-10 (its own iterate, 24 cycles) and then on to
stagnation (relative residual ~1e-15): that is the exact discrete solution p* = A^+(b - mean b),
and likewise lambda* = A^+(w - mean w) for the adjoint.  Compared with it, element by element
in relative L2:

  - the GPU FP64 V-cycle run to stagnation (the reference bench.py measures its errors
    against) equals p* to 1e-11;
  - the benchmark's configuration (mixed precision, adaptive inner cycles) at rtol 1e-10:
    the specified V(2,2) stops ~3.7e-9 from p*, the oracle's own iterate at the same rtol
    included, so the 1e-9 gate is not met at rtol 1e-10 by any implementation of this cycle.
    The GPU pressure must lie as close to p* as the oracle's iterate does (within 5 %), and
    lambda must meet 1e-9;
  - at rtol 1e-11, the tolerance bench.py times as the gate, the mixed, double-float and FP64
    pressures and the mixed lambda all meet 1e-9.
"""
import warnings

import pytest
import torch

import dropfilm as D
import oracle as O
from paper_2605_30082_gb300 import Solver

from _helpers import RHO_PHASE, host, rel

pytestmark = pytest.mark.gpu

N = 512
GATE_ERR = 1e-9
GATE_RTOL = 1e-11


@pytest.fixture(scope="module")
def c512():
    h = 1.0 / N
    cuda = torch.device("cuda")
    g = D.scaled_geometry(N)
    fd, ff = D.fractions_ramp(g, device=cuda, z_chunk=32)
    u = D.face_velocities(N, 0, device=cuda, z_chunk=32)
    w = D.normal_weights((N,) * 3, seed=1, device=cuda, chunk=1 << 26)
    rho = O.density([host(fd), host(ff)], RHO_PHASE)
    faces = O.faces_from_density(rho)
    del rho
    b = O.divergence([host(a) for a in u], h)
    wh = host(w)
    wm = wh - wh.mean()
    M = O.Multigrid(faces, h, coarsest=8)
    p_it, st, nc, rr, _ = M.solve(b, rtol=1e-10)
    assert st == O.OK and rr <= 1e-10
    p_ex, st, _, rr_ex, _ = M.solve(b, rtol=1e-15, max_cycles=400, p0=p_it, stop_on_stall=True)
    assert st == O.OK and rr_ex <= 1e-14
    l_ex, st, _, rl_ex, _ = M.solve(wm, rtol=1e-15, max_cycles=400, stop_on_stall=True)
    assert st == O.OK and rl_ex <= 1e-14
    del M, faces, wh, wm
    return dict(h=h, fd=fd, ff=ff, u=u, w=w, b=b, p_it=p_it, cycles_it=nc, p_ex=p_ex, l_ex=l_ex)


def _solver(c, prec, rtol, inner=0, max_cycles=200):
    s = Solver((N,) * 3, h=c["h"], precision=prec, coarsest=8, rtol=rtol, max_cycles=max_cycles,
               inner_cycles=inner)
    s.set_density(s.density_from_fractions([c["fd"], c["ff"]], list(RHO_PHASE)))
    return s


def test_512_gpu_fp64_stagnation_is_the_exact_solution(c512):
    s = _solver(c512, "fp64", 1e-15, 1, max_cycles=120)
    p = s.solve(s.rhs(u=c512["u"]), raise_on_nonconvergence=False)
    assert s.last_stats.relres <= 1e-14
    assert rel(host(p), c512["p_ex"]) <= 1e-11
    s.close()


def test_512_benchmark_configuration_at_rtol_1e10(c512):
    s = _solver(c512, "mixed", 1e-10, 0)
    p = s.solve(s.rhs(u=c512["u"]))
    assert s.last_stats.relres <= 1e-10
    err_p = rel(host(p), c512["p_ex"])
    err_oracle_iterate = rel(c512["p_it"], c512["p_ex"])
    # the V(2,2) iterate at rtol 1e-10 is this far from p*, whoever runs it
    assert err_p <= 1.05 * err_oracle_iterate, (err_p, err_oracle_iterate)
    assert s.last_stats.cycles <= c512["cycles_it"] + 1
    lam, _, _ = s.adjoint(c512["w"], p, grads=False)
    err_l = rel(host(lam), c512["l_ex"])
    assert err_l <= GATE_ERR, err_l
    # reported in the run's summary (a passing test's output is not shown)
    warnings.warn(f"512^3 parity, rtol 1e-10: |p - p*|/|p*| = {err_p:.3e} (oracle's own iterate "
                  f"{err_oracle_iterate:.3e}), |lam - lam*|/|lam*| = {err_l:.3e}", UserWarning)
    s.close()


@pytest.mark.parametrize("prec,inner", [("mixed", 0), ("mixed_df", 0), ("fp64", 1)])
def test_512_gate_at_rtol_1e11(c512, prec, inner):
    s = _solver(c512, prec, GATE_RTOL, inner)
    p = s.solve(s.rhs(u=c512["u"]))
    assert s.last_stats.relres <= GATE_RTOL
    cycles = s.last_stats.cycles
    err_p = rel(host(p), c512["p_ex"])
    assert err_p <= GATE_ERR, err_p
    assert abs(host(p).mean()) <= 1e-14 * float(p.abs().max())
    if prec == "mixed":
        lam, _, _ = s.adjoint(c512["w"], p, grads=False)
        err_l = rel(host(lam), c512["l_ex"])
        assert err_l <= GATE_ERR, err_l
    warnings.warn(f"512^3 parity, {prec} at rtol {GATE_RTOL:g}: |p - p*|/|p*| = {err_p:.3e}, "
                  f"{cycles} V-cycles", UserWarning)
    s.close()
