"""End-to-end parity of mg_solve with the FP64 oracle, and its error paths.

Reference values:
  O-iter  : the oracle's own V-cycle solve stopped at the same tolerance;
            the GPU FP64 path runs the same algorithm and must reproduce it
            (same cycle count, residual history, p to 1e-12).
  O-exact : the oracle's V-cycles run to stagnation (relative residual
            ~1e-15), i.e. the zero-mean discrete solution p*.  Both GPU
            precisions must reach it to relative L2 <= 1e-9 at rtol 1e-10.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_30082_gb300 import MG_ERR_ARG, MG_ERR_NOT_CONVERGED, MgError, Solver

from _helpers import dev, dropfilm_case, host, random_rho, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c32():
    c = dropfilm_case(32, subcell=True)
    for coarsest in (4, 8):
        M = O.Multigrid(c["faces"], c["h"], coarsest=coarsest)
        c[f"iter{coarsest}"] = M.solve(c["b"], rtol=1e-10)
        c[f"exact{coarsest}"] = M.solve_exact(c["b"])[0]
    return c


def test_fp64_reproduces_oracle_iteration_32cubed(c32):
    s = Solver((32, 32, 32), h=c32["h"], precision="fp64", coarsest=4)
    s.set_density(dev(c32["rho"]))
    p = s.solve(dev(c32["b"]))
    st = s.last_stats
    p_o, st_o, nc_o, rr_o, hist_o = c32["iter4"]
    assert st.cycles == nc_o
    # the GPU sums (h^2 r)^2 per thread in FP32: the history agrees to ~1e-5 relative
    assert np.allclose(st.history(), hist_o, rtol=1e-4, atol=0)
    assert rel(host(p), p_o) < 1e-12
    assert rel(host(p), c32["exact4"]) < 1e-9
    assert abs(host(p).mean()) < 1e-14 * np.abs(host(p)).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_df"])
def test_solution_matches_exact_32cubed(c32, prec):
    s = Solver((32, 32, 32), h=c32["h"], precision=prec, coarsest=8)
    s.set_density(dev(c32["rho"]))
    p = s.solve(dev(c32["b"]))
    assert s.last_stats.relres <= 1e-10
    assert rel(host(p), c32["exact8"]) < 1e-9
    nc_o = c32["iter8"][2]
    assert abs(s.last_stats.cycles - nc_o) <= 2


@pytest.mark.parametrize("dims", [(64, 64, 64), (64, 48, 32), (96, 40, 24), (256, 16, 24), (384, 4, 36)])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_df"])
def test_ragged_grids_match_exact(dims, prec):
    nx, ny, nz = dims
    h = 1.0 / 64
    rho = random_rho(dims, 5, lo=1.2, hi=998.0) if dims != (64, 64, 64) else dropfilm_case(64)["rho"]
    faces = O.faces_from_density(rho)
    b = np.random.default_rng(7).standard_normal((nz, ny, nx))
    M = O.Multigrid(faces, h, coarsest=8)
    exact = M.solve_exact(b)[0]
    s = Solver(dims, h=h, precision=prec, coarsest=8, max_cycles=400)
    s.set_density(dev(rho))
    p = s.solve(dev(b))
    assert s.last_stats.relres <= 1e-10
    assert rel(host(p), exact) < 1e-9
    if prec == "fp64":
        p_o, _, nc_o, _, _ = M.solve(b, rtol=1e-10, max_cycles=400)
        assert s.last_stats.cycles == nc_o and rel(host(p), p_o) < 1e-12


@pytest.mark.parametrize("prec", ["mixed", "mixed_df"])
@pytest.mark.parametrize("inner", [2, 3])
def test_inner_cycles_reach_exact_32cubed(c32, prec, inner):
    """Several FP32 V-cycles per outer FP64 residual: same discrete solution, the V-cycle
    count within one outer iteration of the one-cycle count."""
    s = Solver((32, 32, 32), h=c32["h"], precision=prec, coarsest=8, inner_cycles=inner)
    s.set_density(dev(c32["rho"]))
    p = s.solve(dev(c32["b"]))
    st = s.last_stats
    assert st.relres <= 1e-10
    assert rel(host(p), c32["exact8"]) < 1e-9
    assert st.cycles == inner * st.outer and len(st.history()) == st.outer + 1
    nc_o = c32["iter8"][2]
    assert nc_o - 2 <= st.cycles <= nc_o + inner + 1
    assert all(b < a for a, b in zip(st.history(), st.history()[1:]))


@pytest.mark.parametrize("prec", ["mixed", "mixed_df"])
def test_adaptive_inner_cycles_32cubed(c32, prec):
    """inner_cycles 0: the V-cycles of each outer iteration chosen from the observed contraction.
    The same discrete solution, at most two V-cycles more than one V-cycle per residual, and
    fewer outer iterations (FP64 residuals) than two V-cycles per residual."""
    s = Solver((32, 32, 32), h=c32["h"], precision=prec, coarsest=8, inner_cycles=0)
    s.set_density(dev(c32["rho"]))
    p = s.solve(dev(c32["b"]))
    st = s.last_stats
    assert st.relres <= 1e-10
    assert rel(host(p), c32["exact8"]) < 1e-9
    s1 = Solver((32, 32, 32), h=c32["h"], precision=prec, coarsest=8, inner_cycles=1)
    s1.set_density(dev(c32["rho"]))
    s1.solve(dev(c32["b"]))
    assert st.cycles <= s1.last_stats.cycles + 2
    assert st.outer < (s1.last_stats.cycles + 1) // 2
    assert len(st.history()) == st.outer + 1
    assert all(b < a for a, b in zip(st.history(), st.history()[1:]))
    # max_cycles bounds the adaptive count too
    s2 = Solver((32, 32, 32), h=c32["h"], precision=prec, coarsest=8, inner_cycles=0, rtol=1e-30, max_cycles=6)
    s2.set_density(dev(c32["rho"]))
    s2.solve(dev(c32["b"]), raise_on_nonconvergence=False)
    assert s2.last_stats.cycles == 6 and s2.last_stats.status == MG_ERR_NOT_CONVERGED


@pytest.mark.parametrize("prec,inner", [("fp64", 1), ("mixed", 2), ("mixed", 4), ("mixed_df", 4)])
def test_fcg_reaches_exact_32cubed(c32, prec, inner):
    """Conjugate gradients preconditioned by one V-cycle (flexible form): the same discrete
    solution, in fewer V-cycles than the V-cycle iteration.  The FP64 solve runs the
    oracle's algorithm (or_mg_fcg) step for step: same iteration count."""
    s = Solver((32, 32, 32), h=c32["h"], precision=prec, coarsest=8, inner_cycles=inner, method="fcg")
    s.set_density(dev(c32["rho"]))
    p = s.solve(dev(c32["b"]))
    st = s.last_stats
    assert st.relres <= 1e-10
    assert rel(host(p), c32["exact8"]) < 1e-9
    assert abs(host(p).mean()) < 1e-14 * np.abs(host(p)).max()
    nc_v = c32["iter8"][2]
    assert st.cycles < nc_v
    if prec == "fp64":
        M = O.Multigrid(c32["faces"], c32["h"], coarsest=8)
        p_o, st_o, nit_o, rr_o, hist_o = M.fcg(c32["b"], rtol=1e-10)
        assert abs(st.cycles - nit_o) <= 1
        assert rel(host(p), p_o) < 1e-11
        assert np.allclose(st.history()[: len(hist_o)][:5], hist_o[:5], rtol=1e-6)


@pytest.mark.parametrize("dims", [(64, 48, 32), (96, 40, 24)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fcg_ragged_grids_match_exact(dims, prec):
    nx, ny, nz = dims
    h = 1.0 / 64
    rho = random_rho(dims, 5, lo=1.2, hi=998.0)
    faces = O.faces_from_density(rho)
    b = np.random.default_rng(7).standard_normal((nz, ny, nx))
    exact = O.Multigrid(faces, h, coarsest=8).solve_exact(b)[0]
    s = Solver(dims, h=h, precision=prec, coarsest=8, max_cycles=400, inner_cycles=1 if prec == "fp64" else 3,
               method="fcg")
    s.set_density(dev(rho))
    p = s.solve(dev(b))
    assert s.last_stats.relres <= 1e-10
    assert rel(host(p), exact) < 1e-9


def test_fcg_limits():
    with pytest.raises(MgError):
        Solver((36, 32, 32), precision="mixed", method="fcg")  # mixed FCG needs nx % 8 == 0
    s = Solver((16, 16, 16), precision="fp64", coarsest=8, rtol=1e-30, max_cycles=3, method="fcg")
    s.set_density(dev(random_rho((16, 16, 16), 9)))
    s.solve(dev(np.random.default_rng(3).standard_normal((16, 16, 16))), raise_on_nonconvergence=False)
    assert s.last_stats.cycles == 3 and s.last_stats.status == MG_ERR_NOT_CONVERGED


def test_inner_cycles_limits():
    with pytest.raises(MgError):
        Solver((16, 16, 16), precision="fp64", inner_cycles=2)
    for bad in (-1, 9):
        with pytest.raises(MgError):
            Solver((16, 16, 16), precision="mixed", inner_cycles=bad)
    with pytest.raises(MgError):  # the adaptive count is for the V-cycle iteration only
        Solver((16, 16, 16), precision="mixed", inner_cycles=0, method="fcg")
    # max_cycles bounds the V-cycles: 5 allows two outer iterations of 2
    s = Solver((16, 16, 16), precision="mixed", coarsest=8, rtol=1e-30, max_cycles=5, inner_cycles=2)
    s.set_density(dev(random_rho((16, 16, 16), 9)))
    s.solve(dev(np.random.default_rng(3).standard_normal((16, 16, 16))), raise_on_nonconvergence=False)
    assert s.last_stats.cycles == 4 and s.last_stats.outer == 2


def test_solve_is_deterministic(c32):
    s = Solver((32, 32, 32), h=c32["h"], precision="mixed", coarsest=8)
    s.set_density(dev(c32["rho"]))
    b = dev(c32["b"])
    p1 = s.solve(b).clone()
    p2 = s.solve(b)
    assert torch.equal(p1, p2)


def _off16(a):
    """A copy of `a` whose data pointer sits 8 bytes past a 16-byte boundary."""
    buf = torch.empty(a.numel() + 2, dtype=a.dtype, device=a.device)
    k = 1 if buf.data_ptr() % 16 == 0 else 0
    v = buf[k:k + a.numel()].view(a.shape)
    v.copy_(a)
    assert v.data_ptr() % 16 == 8
    return v


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_df"])
def test_unaligned_rhs_32cubed(c32, prec):
    """The reductions over b read 16-byte vectors where the pointer allows it and single
    elements otherwise (b may have any alignment; p must be 16-byte aligned): an RHS 8 bytes
    off alignment gives the solve of the aligned one."""
    s = Solver((32, 32, 32), h=c32["h"], precision=prec, coarsest=8)
    s.set_density(dev(c32["rho"]))
    b = dev(c32["b"])
    p_al = s.solve(b).clone()
    p_un = s.solve(_off16(b))
    assert s.last_stats.relres <= 1e-10
    assert rel(host(p_un), host(p_al)) < 1e-12
    assert rel(host(p_un), c32["exact8"]) < 1e-9
    # an unaligned solution array is refused before any launch
    with pytest.raises(MgError) as ei:
        s.solve(b, p=_off16(torch.zeros_like(b)))
    assert ei.value.code == MG_ERR_ARG


def test_edge_cases():
    n = 16
    s = Solver((n, n, n), precision="mixed", coarsest=8)
    s.set_density(dev(random_rho((n, n, n), 9)))
    for b in (np.zeros((n, n, n)), np.full((n, n, n), 2.5)):
        p = s.solve(dev(b))
        assert s.last_stats.cycles == 0 and not host(p).any()
    b = dev(np.random.default_rng(3).standard_normal((n, n, n)))
    p = s.solve(b)
    # warm start from the solution: no cycle needed
    s2 = Solver((n, n, n), precision="mixed", coarsest=8, warm_start=True)
    s2.set_density(dev(random_rho((n, n, n), 9)))
    p2 = s2.solve(b, p=p.clone())
    assert s2.last_stats.cycles == 0 and rel(host(p2), host(p)) < 1e-12
    # warm start from a shifted solution: the gauge is restored
    p3 = s2.solve(b, p=p.clone() + 7.0)
    assert s2.last_stats.cycles == 0 and rel(host(p3), host(p)) < 1e-12
    # max_cycles exhausted: status returned, last iterate kept with zero mean
    s3 = Solver((n, n, n), precision="fp64", coarsest=8, rtol=1e-30, max_cycles=2)
    s3.set_density(dev(random_rho((n, n, n), 9)))
    with pytest.raises(MgError) as ei:
        s3.solve(b)
    assert ei.value.code == MG_ERR_NOT_CONVERGED
    p4 = s3.solve(b, raise_on_nonconvergence=False)
    assert s3.last_stats.cycles == 2 and abs(host(p4).mean()) < 1e-14
    # non-finite RHS
    bad = np.ones((n, n, n))
    bad[1, 2, 3] = np.inf
    with pytest.raises(MgError) as ei:
        s.solve(dev(bad))
    assert ei.value.code == MG_ERR_ARG


@pytest.mark.parametrize("coeffs", ["rho", "faces"])
def test_mixed_df_matches_mixed_and_needs_even_nx(coeffs):
    """The double-float outer loop reaches the same discrete solution as the FP64 one.

    coeffs="rho": the residual forms beta = (s_c + s_nb) / 2 from s = 1/rho in double-float;
    "faces": it reads the face coefficients and the diagonal as double-float pairs."""
    dims = (48, 32, 40)
    rho = random_rho(dims, 12)
    b = np.random.default_rng(8).standard_normal((40, 32, 48))
    ps = {}
    for prec in ("mixed", "mixed_df"):
        s = Solver(dims, h=1 / 48, precision=prec, coarsest=8, rtol=1e-12, max_cycles=400)
        if coeffs == "rho":
            s.set_density(dev(rho))
        else:
            s.set_face_coeffs(*(dev(f) for f in O.faces_from_density(rho)))
        ps[prec] = host(s.solve(dev(b)))
        assert s.last_stats.relres <= 1e-12
    assert rel(ps["mixed_df"], ps["mixed"]) < 1e-10
    with pytest.raises(MgError):
        Solver((47, 32, 40), precision="mixed_df")


def test_wrong_shapes_and_devices_are_rejected():
    s = Solver((16, 16, 16), precision="fp64")
    with pytest.raises(ValueError):
        s.set_density(torch.ones((16, 16, 15), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        s.set_density(torch.ones((16, 16, 16), dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        s.set_density(torch.ones((16, 16, 16), dtype=torch.float64))
