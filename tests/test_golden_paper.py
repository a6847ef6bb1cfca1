"""Pins of the mesh counting and terrain profile against the values the paper
prints for its test case (tests/golden/paper_sec3_setup.txt, Sec. 3 and Sec. 3.3):
(r+1)^3 nodal unknowns per cell per scalar, the printed resolutions of the two
uniform meshes, and the -3/2 bell profile (terrain kind 2) at its centre and one
half-width away."""
import os

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_sec3_setup.txt")


def _records():
    rec = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, *v = line.split()
            rec[k] = [float(x) for x in v]
    return rec


def test_uniform_meshes_unknowns_and_resolution():
    r = _records()
    Lx, Ly, Lz = (1000.0 * v for v in r["domain_km"])
    for key in ("mesh_uniform", "mesh_coarse"):
        nx, ny, nz, nel, deg, unknowns, res = r[key]
        nx, ny, nz, deg = int(nx), int(ny), int(nz), int(deg)
        assert nx * ny * nz == nel
        m = O.make_mesh(nx, ny, nz, deg, Lx=Lx, Ly=Ly, Lz=Lz)
        n = O.ndofs(m)
        assert n == nel * (deg + 1) ** 3
        if unknowns:
            assert abs(n - unknowns) <= 0.005 * unknowns  # "about 38.5 million"
        # the printed resolution is the element size over the degree in every direction
        for L, ne in ((Lx, nx), (Ly, ny), (Lz, nz)):
            assert L / (ne * deg) == res


def test_nonconforming_mesh_unknowns():
    nel, deg, unknowns = _records()["mesh_nonconforming"]
    assert abs(nel * (deg + 1) ** 3 - unknowns) <= 0.005 * unknowns


def test_bell_profile():
    hc, ac, xc, yc = _records()["hill_m"]
    Lx, Ly, Lz = (1000.0 * v for v in _records()["domain_km"])
    m = O.make_mesh(4, 4, 2, 2, Lx=Lx, Ly=Ly, Lz=Lz, terrain=2, hc=hc, ac=ac, xc=xc, yc=yc)
    assert O.terrain_height(m, xc, yc) == hc
    assert abs(O.terrain_height(m, xc + ac, yc) - hc * 2.0 ** -1.5) <= 1e-12 * hc
    assert abs(O.terrain_height(m, xc + ac, yc + ac) - hc * 3.0 ** -1.5) <= 1e-12 * hc
