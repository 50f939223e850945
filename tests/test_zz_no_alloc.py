"""The allocation-free small-grid solve against the handle-based coarse solve and the oracle.

mg_dense_solve_noalloc serves callers that cannot allocate device memory when they need a
solve (device memory owned by another allocator, fixed memory budgets, loops that cannot pay
for the synchronisation of cudaMalloc/cudaFree).  It must give the same zero-mean solution as
mg_coarse_solve on a handle whose single level is the same grid, and as the oracle's exact
coarse solve.  Two calls in a row check that the shared scratch array, which keeps the
previous call's contents, is reset where it must be.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_30082_gb300 import Solver
from paper_2605_30082_gb300 import _lib as L

from _helpers import dev, host, random_rho, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(8, 8, 8), (7, 6, 5)])
def test_noalloc_solve_matches_handle_coarse_solve(dims):
    nx, ny, nz = dims
    h = 1.0 / 8
    faces = [dev(f) for f in O.faces_from_density(random_rho(dims, 21))]
    s = Solver(dims, h=h, precision="fp64", coarsest=max(dims))
    assert s.num_levels == 1
    s.set_face_coeffs(*faces)
    rng = np.random.default_rng(5)
    for call in range(2):
        r = dev(rng.standard_normal((nz, ny, nx)))
        e_ref = torch.empty_like(r)
        assert L.mg_coarse_solve(s._h, r, e_ref) == L.MG_OK
        e = torch.full_like(r, np.nan)
        st = L.mg_dense_solve_noalloc(dims, h, *faces, r, e)
        assert st == L.MG_OK, (call, st)
        torch.cuda.synchronize()
        assert rel(host(e), host(e_ref)) < 1e-11, call
        # and the oracle's exact zero-mean solve on the host
        e_or = O.coarse_solve([host(f) for f in faces], host(r), h)
        assert rel(host(e), e_or) < 1e-11, call


def test_noalloc_rejects_too_large_and_bad_coefficients():
    dims = (16, 8, 8)
    h = 1.0 / 16
    faces = [dev(f) for f in O.faces_from_density(np.ones((8, 8, 16)))]
    r = dev(np.ones((8, 8, 16)))
    e = torch.empty_like(r)
    assert L.mg_dense_solve_noalloc(dims, h, *faces, r, e) == L.MG_ERR_ARG
    dims = (8, 8, 8)
    f = [a.copy() for a in O.faces_from_density(np.ones((8, 8, 8)))]
    f[2][3, 2, 1] = -1.0
    r = dev(np.ones((8, 8, 8)))
    e = torch.empty_like(r)
    assert L.mg_dense_solve_noalloc(dims, 1 / 8, *(dev(a) for a in f), r, e) == L.MG_ERR_DENSITY
    # a good call after the failed one is unaffected by the error word it left
    g = [dev(a) for a in O.faces_from_density(np.ones((8, 8, 8)))]
    assert L.mg_dense_solve_noalloc(dims, 1 / 8, *g, r, e) == L.MG_OK
