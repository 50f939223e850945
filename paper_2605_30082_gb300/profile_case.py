"""A small solve for kernel profiling:
python -m paper_2605_30082_gb300.profile_case NX NY NZ [PRECISION [INNER [CYCLES [FUSED [RTOL]]]]]

Random density in [1.2, 998] and random right-hand side (torch generators, seeds 3 and 4),
`CYCLES` V-cycles (default 2) of the given precision ('fp64', 'mixed', 'mixed_df'), followed by
one adjoint solve of as many cycles, one velocity correction of random face velocities (seeds
5-7, out of place) and one density adjoint of random FP32 face gradients (seeds 8-10, two
fractions).  Sized by the caller so that every array is larger than L2 while the whole case
holds a few GB: e.g. 512 512 256 keeps the 512-cell rows (and so the launch configuration) of
the 512^3 workload at half its cells.  FUSED = 1 smooths the finest level with fused red-black
sweeps (mg_opts.fused_sweeps).  RTOL (default 1e-30: the cycle limit ends both solves) set to a
reachable tolerance lets the adjoint converge, so that its fused gradient kernel runs too.
"""
import sys

import torch

from . import _lib as L
from .solver import MgError, Solver


def main(argv):
    nx, ny, nz = (int(a) for a in argv[:3])
    prec = argv[3] if len(argv) > 3 else "mixed"
    inner = int(argv[4]) if len(argv) > 4 else 1
    cycles = int(argv[5]) if len(argv) > 5 else 2
    fused = len(argv) > 6 and argv[6] == "1"
    rtol = float(argv[7]) if len(argv) > 7 else 1e-30
    dev = torch.device("cuda")
    g = torch.Generator(device="cuda")
    rho = 1.2 + 996.8 * torch.rand((nz, ny, nx), generator=g.manual_seed(3), device=dev, dtype=torch.float64)
    b = torch.randn((nz, ny, nx), generator=g.manual_seed(4), device=dev, dtype=torch.float64)
    s = Solver((nx, ny, nz), h=1.0 / max(nx, ny, nz), precision=prec, coarsest=8, rtol=rtol,
               max_cycles=cycles, inner_cycles=inner if prec != "fp64" else 1, fused_sweeps=fused)
    s.set_density(rho)
    p = s.solve(b, raise_on_nonconvergence=False)
    try:
        s.adjoint(b, p)  # stops at the cycle limit, by design
    except MgError as e:
        if e.code != L.MG_ERR_NOT_CONVERGED:
            raise
    u = tuple(torch.randn(sh, generator=g.manual_seed(5 + q), device=dev, dtype=torch.float64)
              for q, sh in enumerate(s.face_shapes))
    s.project(p, u, out=tuple(torch.empty_like(a) for a in u))
    gr = tuple(torch.randn(sh, generator=g.manual_seed(8 + q), device=dev, dtype=torch.float32)
               for q, sh in enumerate(s.face_shapes))
    s.density_grads(rho, gr, [998.0, 880.0, 1.2])
    torch.cuda.synchronize()
    print("ok", s.last_stats.cycles, s.last_stats.relres)


if __name__ == "__main__":
    main(sys.argv[1:])
