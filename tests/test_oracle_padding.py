"""Pins the oracle's padding convention to the one number the paper prints
for its FFT grid: the all-to-all volume at N = 400 (Results, Performance)."""

import json
import os

import numpy as np

from oracle import micromag

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_transpose_volume.json")


def test_padding_matches_paper_transpose_volume():
    g = json.load(open(GOLDEN))
    n = g["mesh_n"]
    p = micromag.Problem((n, n, n), (1e-9, 1e-9, 1e-9))
    Px, Py, Pz = p.padded
    assert Px == Py == Pz == g["padded_len"]
    # numpy's real FFT keeps P/2 + 1 values along the last transformed axis
    assert np.fft.rfftfreq(Pz).size == g["rfft_len"]
    assert n // g["ranks"] == g["slab_rows"]
    vol = g["slab_rows"] * Px * (Pz // 2 + 1) * g["components"] * g["bytes_per_complex"]
    assert abs(vol - g["approx_bytes"]) / g["approx_bytes"] < 0.001


def test_single_cell_axis_is_not_padded():
    p = micromag.Problem((8, 4, 1), (1e-9, 1e-9, 1e-9))
    assert p.padded == (16, 8, 1)
