"""Pins of the 3D oracle's diagnostics (Sec. 3: the Tr c admissibility
counts; mid-plane statistics; energy) on constructed fields whose values
follow in closed form or by direct evaluation on the grid, independent of
the oracle's transforms.  No GPU.

Fields (grid x_j = j Lx/nx, y_l = cos(pi l/(ny-1)), z_k = k Lz/nz):
  u = (1 - y^2) (1 + A cos(kx x) + B sin(kz z)),  v = 0,  w = C (2 y^2 - 1),
  c = I + diag(f, 0, 0),  f = 10 (y^2 - 0.31) (1 + cos(kx x)/2),
with kx = 2 pi/Lx, kz = 2 pi/Lz; every field is exactly representable, and
no grid point has Tr c = 3 + f within the tie band of 3 or of 0.
"""
import math

import numpy as np
import pytest

from oracle import ptt3d as O3

NX, NY, NZ, LX, LZ = 16, 17, 8, 10.0, 5.0
A, B, C = 0.3, 0.2, 0.1
KX, KZ = 2 * math.pi / LX, 2 * math.pi / LZ


def _grid():
    x = np.arange(NX) * LX / NX
    y = np.cos(np.pi * np.arange(NY) / (NY - 1))
    z = np.arange(NZ) * LZ / NZ
    return np.meshgrid(x, y, z, indexing="ij")


def _fields():
    X, Y, Z = _grid()
    u = (1 - Y ** 2) * (1 + A * np.cos(KX * X) + B * np.sin(KZ * Z))
    w = C * (2 * Y ** 2 - 1)
    f = 10.0 * (Y ** 2 - 0.31) * (1 + 0.5 * np.cos(KX * X))
    zero, one = np.zeros_like(u), np.ones_like(u)
    return [u, zero, w, one + f, zero, zero, one, zero, one], f


@pytest.fixture(scope="module")
def diag():
    ch = O3.Channel3D(O3.Params3(nx=NX, ny=NY, nz=NZ, lx=LX, lz=LZ))
    fields, f = _fields()
    ch.set_physical(fields)
    return ch.diagnostics(), f


def test_volume_counts_match_direct_evaluation(diag):
    d, f = diag
    tr = 3.0 + f
    tau = 1e-9 * np.max(np.abs(tr))
    assert d["n_lt3"] == int(np.sum(tr < 3.0)) > 0
    assert d["n_lt0"] == int(np.sum(tr < 0.0)) > 0
    assert d["n_band3"] == int(np.sum(np.abs(tr - 3.0) <= tau)) == 0
    assert d["n_band0"] == int(np.sum(np.abs(tr) <= tau)) == 0
    assert abs(d["min_trc"] - tr.min()) <= 1e-12 * np.max(np.abs(tr))
    assert abs(d["max_trc"] - tr.max()) <= 1e-12 * np.max(np.abs(tr))


def test_mean_trace_and_energy_closed_forms(diag):
    d, _ = diag
    # volume averages: <y^2> = 1/3, <(1 - y^2)^2> = 8/15, <(2 y^2 - 1)^2> = 7/15;
    # <(1 + A cos + B sin)^2>_xz = 1 + (A^2 + B^2)/2, <1 + cos/2>_x = 1
    assert abs(d["mean_trc"] - (3.0 + 10.0 * (1.0 / 3.0 - 0.31))) <= 1e-13
    e = 0.5 * (8.0 / 15.0 * (1 + (A * A + B * B) / 2) + C * C * 7.0 / 15.0)
    assert abs(d["energy"] - e) <= 1e-14


def test_midplane_counts_and_power_sums(diag):
    d, _ = diag
    x = np.arange(NX) * LX / NX
    z = np.arange(NZ) * LZ / NZ
    Xm, Zm = np.meshgrid(x, z, indexing="ij")
    # at y = 0: u = 1 + A cos + B sin, w = -C, Tr c = 3 - 3.1 (1 + cos(kx x)/2)
    trm = 3.0 - 3.1 * (1 + 0.5 * np.cos(KX * Xm))
    up = A * np.cos(KX * Xm) + B * np.sin(KZ * Zm)
    q = [trm, up, np.zeros_like(up), -A * KX * np.sin(KX * Xm), B * KZ * np.cos(KZ * Zm),
         np.zeros_like(up), np.zeros_like(up), np.zeros_like(up)]
    assert d["n_mid_lt3"] == int(np.sum(trm < 3.0)) == NX * NZ
    assert d["n_mid_lt0"] == int(np.sum(trm < 0.0)) == 9 * NZ
    want = np.array([[np.sum(qq ** k) for k in range(1, 5)] for qq in q])
    scale = np.maximum(np.abs(want), NX * NZ)
    assert np.all(np.abs(d["mid_sums"] - want) <= 1e-12 * scale), d["mid_sums"] - want
    # the second moments in closed form (discrete orthogonality on the grid)
    n = NX * NZ
    assert abs(d["mid_sums"][1][1] - n * (A * A + B * B) / 2) <= 1e-12 * n
    assert abs(d["mid_sums"][3][1] - n * (A * KX) ** 2 / 2) <= 1e-12 * n
    assert abs(d["mid_sums"][4][1] - n * (B * KZ) ** 2 / 2) <= 1e-12 * n
    assert abs(d["mid_sums"][0][0] - n * (3.0 - 3.1)) <= 1e-12 * n
