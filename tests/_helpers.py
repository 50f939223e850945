"""Shared test helpers: inputs built from the seeded generators, oracle-side fields."""
import numpy as np
import torch

import dropfilm as D
import oracle as O

RHO_PHASE = (998.0, 880.0, 1.2)


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(x):
    return x.detach().cpu().numpy().astype(np.float64)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def random_rho(dims, seed, lo=1.2, hi=998.0):
    """log-uniform density per cell, shape (nz, ny, nx)."""
    nx, ny, nz = dims
    u = D.uniform53(seed, torch.arange(nx * ny * nz)).numpy().reshape(nz, ny, nx)
    return lo * (hi / lo) ** u


def dropfilm_case(n, subcell=False):
    """Fractions, oracle density/faces and the divergence RHS of the drop/film layout at n^3."""
    g = D.scaled_geometry(n)
    fd, ff = D.fractions_subcell(g) if subcell else D.fractions_ramp(g)
    h = 1.0 / n
    rho = O.density([fd.numpy(), ff.numpy()], RHO_PHASE)
    faces = O.faces_from_density(rho)
    u = D.face_velocities(n, seed=0)
    b = O.divergence([a.numpy() for a in u], h)
    return dict(n=n, h=h, geom=g, fd=fd, ff=ff, rho=rho, faces=faces, u=u, b=b)


def csf_case(n):
    """dropfilm_case plus the curvature band, the CSF face quantity and the loss weights w."""
    c = dropfilm_case(n)
    kappa = D.curvature_band(c["fd"], c["geom"]).numpy()
    c["kappa"] = kappa
    c["csf"] = O.csf_faces(c["fd"].numpy(), kappa, c["h"])
    c["w"] = D.normal_weights((n, n, n), seed=1).numpy()
    return c
