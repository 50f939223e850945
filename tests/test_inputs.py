"""The seeded input generators give the same values whole or in chunks (the chunked forms
bound the temporaries at 1024^3)."""
import torch

import dropfilm as D


def test_face_velocities_chunked_equal_whole():
    whole = D.face_velocities(12, seed=3)
    for z_chunk in (1, 5, 13):
        for a, b in zip(whole, D.face_velocities(12, seed=3, z_chunk=z_chunk)):
            assert torch.equal(a, b)


def test_normal_weights_chunked_equal_whole():
    whole = D.normal_weights((7, 9, 11), seed=1)
    for chunk in (1, 100, 693, 1000):
        assert torch.equal(whole, D.normal_weights((7, 9, 11), seed=1, chunk=chunk))


def test_curvature_band_is_two_over_r_on_the_band():
    g = D.scaled_geometry(80)  # more than one 64-slice chunk
    fd, _ = D.fractions_ramp(g)
    k = D.curvature_band(fd, g)
    band = (fd > 0) & (fd < 1)
    assert band.any() and (~band).any()
    assert torch.all(k[band] == 2.0 / (g.radius / g.n)) and torch.all(k[~band] == 0)
