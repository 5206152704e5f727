"""Fourier neural operator, CPU oracle (test infrastructure only).

Plain float64 PyTorch (CPU) restatement of the surrogate network, for
checking the GPU kernels' outputs and gradients:
    v0 = P m + p;  a_l = W_l v_l + b_l + irfft2(keep(R_l . keep(rfft2(v_l))));
    v_{l+1} = GELU(a_l) for l < L-1, v_L = a_{L-1};  h = Q v_L + q,
where keep() retains kx < M and ky in [0, M) U [NY - M, NY) of the
half-spectrum (everything else zero) and GELU is the exact erf form.
Gradients come from torch.autograd on this forward.

The flat parameter vector has the GPU's layout: P [W][3], p [W], then per
layer W_l [W][W], b_l [W], R_l [W][W][2M][M] complex (re, im interleaved),
then Q [3][W], q [3].
"""

import numpy as np
import torch


def unpack(params, W, M, L):
    t = torch.as_tensor(np.asarray(params, dtype=np.float64))
    o = 0

    def take(n):
        nonlocal o
        v = t[o:o + n]
        o += n
        return v
    P = take(3 * W).reshape(W, 3)
    p = take(W)
    layers = []
    for _ in range(L):
        Wl = take(W * W).reshape(W, W)
        bl = take(W)
        R = take(2 * W * W * 2 * M * M).reshape(W, W, 2 * M, M, 2)
        layers.append((Wl, bl, torch.complex(R[..., 0], R[..., 1])))
    Q = take(3 * W).reshape(3, W)
    q = take(3)
    assert o == t.numel()
    return P, p, layers, Q, q


def retained_rows(M, NY):
    return list(range(M)) + list(range(NY - M, NY))


def spectral(v, R, M):
    """irfft2 of R . (retained rfft2(v)) with zeros elsewhere; v [B, W, NY, NX]."""
    B, W, NY, NX = v.shape
    V = torch.fft.rfft2(v)                         # [B, W, NY, NX/2+1]
    rows = retained_rows(M, NY)
    S = V[:, :, rows, :M]                          # [B, W, 2M, M]
    T = torch.einsum("oiyk,biyk->boyk", R, S)
    Z = torch.zeros((B, W, NY, NX // 2 + 1), dtype=V.dtype)
    Z[:, :, rows, :M] = T
    return torch.fft.irfft2(Z, s=(NY, NX))


def gelu(x):
    return 0.5 * x * (1 + torch.erf(x / np.sqrt(2.0)))


def forward(params, m, W, M, L):
    """m: array [B, 3, NY, NX] -> h [B, 3, NY, NX] (torch float64)."""
    P, p, layers, Q, q = unpack(params, W, M, L)
    return forward_t(torch.as_tensor(np.asarray(m, dtype=np.float64)), P, p, layers, Q, q, M)


def forward_t(m, P, p, layers, Q, q, M):
    v = torch.einsum("wc,bcyx->bwyx", P, m) + p[None, :, None, None]
    for l, (Wl, bl, R) in enumerate(layers):
        a = torch.einsum("oi,biyx->boyx", Wl, v) + bl[None, :, None, None] + spectral(v, R, M)
        v = gelu(a) if l < len(layers) - 1 else a
    return torch.einsum("cw,bwyx->bcyx", Q, v) + q[None, :, None, None]


def loss(h, target):
    """Mean over samples of |h - t|^2 / |t|^2."""
    d = ((h - target) ** 2).sum(dim=(1, 2, 3))
    n = (target ** 2).sum(dim=(1, 2, 3))
    return (d / n).mean()


def loss_and_grad(params, m, target, W, M, L):
    """(loss, dloss/dparams as a flat float64 numpy array)."""
    t = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    P, p, layers, Q, q = unpack_t(t, W, M, L)
    h = forward_t(torch.as_tensor(np.asarray(m, dtype=np.float64)), P, p, layers, Q, q, M)
    Lv = loss(h, torch.as_tensor(np.asarray(target, dtype=np.float64)))
    Lv.backward()
    return float(Lv.detach()), t.grad.numpy().copy()


def unpack_t(t, W, M, L):
    o = 0

    def take(n):
        nonlocal o
        v = t[o:o + n]
        o += n
        return v
    P = take(3 * W).reshape(W, 3)
    p = take(W)
    layers = []
    for _ in range(L):
        Wl = take(W * W).reshape(W, W)
        bl = take(W)
        R = take(2 * W * W * 2 * M * M).reshape(W, W, 2 * M, M, 2)
        layers.append((Wl, bl, torch.complex(R[..., 0], R[..., 1])))
    Q = take(3 * W).reshape(3, W)
    q = take(3)
    return P, p, layers, Q, q
