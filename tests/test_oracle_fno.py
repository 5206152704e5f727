"""Pins for the oracle FNO: the FFT-based spectral layer against the direct
double sums of its definition, band-limited inputs passing unchanged through
identity mixing while modes outside the retained set vanish, and autograd
gradients passing a float64 finite-difference check (gradcheck)."""

import numpy as np
import torch

from oracle import fno


def test_spectral_layer_against_direct_dft_sums():
    """The spectral term written out as plain double sums over the grid and
    the retained modes: S(ky, kx) = sum_{y,x} v e^{-2 pi i (kx x / NX + ky y / NY)},
    T = R S, out = Re(sum c_kx T e^{+2 pi i (...)}) / (NX NY), c_0 = 1, c_kx = 2."""
    rng = np.random.default_rng(0)
    B, W, NY, NX, M = 2, 2, 6, 8, 2
    v = rng.standard_normal((B, W, NY, NX))
    R = rng.standard_normal((W, W, 2 * M, M)) + 1j * rng.standard_normal((W, W, 2 * M, M))
    kys = list(range(M)) + list(range(-M, 0))
    out = np.zeros((B, W, NY, NX))
    for b in range(B):
        S = np.zeros((W, 2 * M, M), dtype=complex)
        for i in range(W):
            for r, ky in enumerate(kys):
                for kx in range(M):
                    for y in range(NY):
                        for x in range(NX):
                            S[i, r, kx] += v[b, i, y, x] * np.exp(-2j * np.pi * (kx * x / NX + ky * y / NY))
        for o in range(W):
            for y in range(NY):
                for x in range(NX):
                    z = 0.0
                    for r, ky in enumerate(kys):
                        for kx in range(M):
                            t = sum(R[o, i, r, kx] * S[i, r, kx] for i in range(W))
                            z += (1 if kx == 0 else 2) * (t * np.exp(2j * np.pi * (kx * x / NX + ky * y / NY))).real
                    out[b, o, y, x] = z / (NX * NY)
    got = fno.spectral(torch.tensor(v), torch.tensor(R), M).numpy()
    np.testing.assert_allclose(got, out, atol=1e-12)


def test_band_limited_inputs_pass_and_outside_modes_vanish():
    NY, NX, M, W = 16, 16, 3, 2
    R = torch.zeros((W, W, 2 * M, M), dtype=torch.complex128)
    for i in range(W):
        R[i, i] = 1.0
    y, x = np.meshgrid(np.arange(NY), np.arange(NX), indexing="ij")
    band = np.cos(2 * np.pi * (2 * x / NX + 1 * y / NY)) + 0.5 * np.sin(2 * np.pi * (1 * x / NX - 2 * y / NY)) + 0.3
    vb = torch.tensor(np.broadcast_to(band, (1, W, NY, NX)).copy())
    assert torch.allclose(fno.spectral(vb, R, M), vb, atol=1e-12)
    outside = np.cos(2 * np.pi * (M * x / NX)) + np.sin(2 * np.pi * (1 * x / NX + (M + 1) * y / NY))
    vo = torch.tensor(np.broadcast_to(outside, (1, W, NY, NX)).copy())
    assert float(fno.spectral(vo, R, M).abs().max()) < 1e-12


def test_autograd_gradients_pass_finite_difference_check():
    W, M, L, NY, NX = 3, 2, 2, 8, 8
    rng = np.random.default_rng(1)
    n = 3 * W + W + L * (W * W + W + 2 * W * W * 2 * M * M) + 3 * W + 3
    params = torch.tensor(rng.standard_normal(n) * 0.3, requires_grad=True)
    m = torch.tensor(rng.standard_normal((2, 3, NY, NX)))
    t = torch.tensor(rng.standard_normal((2, 3, NY, NX)))

    def f(pp):
        P, p, layers, Q, q = fno.unpack_t(pp, W, M, L)
        return fno.loss(fno.forward_t(m, P, p, layers, Q, q, M), t)
    assert torch.autograd.gradcheck(f, (params,), eps=1e-6, atol=1e-8, rtol=1e-6)
