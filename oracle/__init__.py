"""CPU oracle for the micromagnetic hot path (test infrastructure only).

This package is a plain, slow, obviously-correct CPU restatement of what the
GPU library computes, written from the paper's equations:

* ``newell``   - the cell-averaged demagnetisation tensor of Newell (cited at
                 Eq. 4 of the paper), exact near field in extended precision and
                 a convergent Taylor series of the cell-averaged dipole field far
                 away (error bound stated and pinned by the tests).
* ``micromag`` - demag field as the zero-padded (linear, non-periodic)
                 convolution of Eq. 4 (FFT and O(N^2) direct sum), the exchange
                 field of Eq. 2, uniaxial anisotropy, Zeeman, the LLG right-hand
                 side of Eq. 1, classic RK4 and Fehlberg RKF45 steps (the paper's
                 integrator), energies, torque and relax().
* ``adjoint``  - gradients of a trajectory loss with respect to the per-cell
                 Ms by their definition (central differences, Richardson).
* ``fno``      - the demag surrogate network in float64 PyTorch (CPU), with
                 gradients by autograd, for checking the GPU kernels.

It is NOT part of the product.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import it.  It imports nothing from the GPU
package and the GPU package imports nothing from it.  Arrays are float64
(Newell near field: numpy ``longdouble``), laid out component-planar
``[3][nz][ny][nx]`` with x fastest, SI units throughout.
"""

from . import newell, micromag, adjoint, fno  # noqa: F401
