"""The oracle's 2D operators against the stencils printed in Sec. 5.1
(tests/golden/sec5_1_stencils_2d.txt): each operator applied to a unit
impulse reproduces the printed weights and scale exactly (up to rounding).
Array conventions of the oracle: shape (ny, nx), last axis x; vertex array
index v holds the corner shared by cells v and v + 1."""

import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    out = {}
    with open(os.path.join(HERE, "golden", "sec5_1_stencils_2d.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            name, scale, *entries = line.split()
            w = {}
            for e in entries:
                off, val = e.split(":")
                di, dj = (int(t) for t in off.split(","))
                w[(di, dj)] = float(val)
            out[name] = (scale, w)
    return out


GOLD = _load()
N, H = 8, 0.3


def _scale(tag):
    return {"1/h^2": 1 / H ** 2, "1/2h^2": 1 / (2 * H ** 2), "1/2h": 1 / (2 * H)}[tag]


def _impulse(i, j):
    u = np.zeros((N, N))
    u[j % N, i % N] = 1.0  # cell (i, j): x index i on the last axis
    return u


def _apply(oracle, name, u):
    if name == "laplacian":
        return oracle.lap(u, H)
    if name == "skew_laplacian":
        return oracle.skew_lap(u, H)
    if name == "vertex_dx":
        return oracle.vgrad(u, H)[1]  # array axis 1 is x
    if name == "vertex_dy":
        return oracle.vgrad(u, H)[0]
    if name == "cell_dx":
        return oracle.vdiv([np.zeros_like(u), u], H)
    if name == "cell_dy":
        return oracle.vdiv([u, np.zeros_like(u)], H)
    raise KeyError(name)


@pytest.mark.parametrize("name", sorted(GOLD))
def test_operator_matches_printed_stencil(oracle, name):
    scale, w = GOLD[name]
    s = _scale(scale)
    ci, cj = 3, 4  # target cell (or vertex (ci+1/2, cj+1/2))
    for di in range(-2, 3):
        for dj in range(-2, 3):
            if name.startswith("cell_"):
                # input on vertices: vertex (ci + di - 1/2, cj + dj - 1/2) is vertex index (ci + di - 1, cj + dj - 1)
                out = _apply(oracle, name, _impulse(ci + di - 1, cj + dj - 1))
            else:
                out = _apply(oracle, name, _impulse(ci + di, cj + dj))
            got = out[cj, ci]
            assert got == pytest.approx(s * w.get((di, dj), 0.0), abs=1e-12 * s), (name, di, dj)


def test_p2_plaplacian_is_the_skew_laplacian(oracle):
    """Sec. 5.1: for p = 2 the discrete p-Laplacian is Delta_h^v."""
    u = np.random.default_rng(3).standard_normal((N, N))
    assert np.allclose(oracle.plap(u, H, 2.0), oracle.skew_lap(u, H), rtol=0, atol=1e-12)
