"""Field solver alone: white-noise E, B in an empty box (no particles, so J = 0) advanced by
the CUDA path and by the oracle.  Every point of every component, the Mur faces, edges and
corners included, and (3D) columns both away from and on the faces of the box, and columns
that end on the node planes x = n_x, y = n_y (which they write for the absent next column)."""
import numpy as np
import pytest

import synth
from _support import small_1d, small_2d, small_3d

pytestmark = pytest.mark.gpu

SHAPES = {1: (300, 1, 1), 2: (100, 70, 1), 3: (80, 40, 48)}
# 3D: x a multiple of the 32-point column and y of its 8 rows, so that the node planes
# x = n_x and y = n_y (and their edge) are written by the columns that end on them
SHAPE_3D_ENDS = (64, 40, 33)


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_11393_gb300 import _build, pic

    _build.build()
    pic.load()
    return pic


def noise_fields(n, dim, seed):
    """(9, ext_z, ext_y, ext_x) with E, B ~ N(0, 1) on the points each component has (Yee
    stagger: E_c is staggered along c, B_c along the other axes) and J = 0."""
    ext = [n[d] + 1 if d < dim else 1 for d in range(3)]
    rng = np.random.default_rng(seed)
    F = np.zeros((9, ext[2], ext[1], ext[0]))
    F[:6] = rng.normal(size=(6, ext[2], ext[1], ext[0]))
    for comp in range(6):
        c = comp % 3
        for d in range(dim):
            stag = (d == c) if comp < 3 else (d != c)
            if stag:
                sl = [slice(None)] * 3
                sl[2 - d] = slice(n[d], None)
                F[(comp,) + tuple(sl)] = 0.0
    return F


@pytest.mark.parametrize("dim,shape", [(1, SHAPES[1]), (2, SHAPES[2]), (3, SHAPES[3]), (3, SHAPE_3D_ENDS)],
                         ids=["1d", "2d", "3d", "3d_node_planes"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_vacuum_field_solve_matches_oracle(P, orc, dim, shape, prec):
    make = {1: small_1d, 2: small_2d, 3: small_3d}[dim]
    w = make().with_(n=shape, ppc=0, precision=synth.FP32 if prec == "fp32" else synth.FP64)
    sim = P.Simulation(P.config_from(w))
    ref = orc.Sim(orc.config_from(w))
    F = noise_fields(shape, dim, seed=40 + dim)
    sim.set_fields(F)
    ref.set_fields(F)
    tol = 1e-5 if prec == "fp32" else 1e-12
    for k in (1, 24):
        sim.step(k)
        ref.step(k)
        G, H = sim.fields(), ref.fields()
        for comp in range(6):
            err = np.abs(G[comp] - H[comp]).max() / np.abs(H[comp]).max()
            assert err < tol, (k, comp, err)
