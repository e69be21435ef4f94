"""Writes the stored expected values under tests/golden/ (run: python tests/golden/make_golden.py).

Every value comes from the FP64 oracle (``oracle/``) on a small seeded input; the
paper prints no worked numerical example, so these fixtures are regression pins
of the oracle (tests/test_golden.py checks the oracle still reproduces them and
the GPU path matches them).  Format: one header line, then one line per grid
point in C order: "jx jy jz re(input) im(input) re(output) im(output)", the
complex64 input written exactly (float32 values printed with 9 significant
digits) and the output with 17.
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def _write(path, header, x, y):
    with open(path, "w") as f:
        f.write(header.rstrip() + "\n")
        for idx in np.ndindex(*x.shape):
            a, b = x[idx], y[idx]
            f.write(f"{idx[0]} {idx[1]} {idx[2]} {a.real:.9g} {a.imag:.9g} {b.real:.17g} {b.imag:.17g}\n")


def inputs():
    """The fixtures' inputs (seeded): complex64 grids and a float32 influence function."""
    rng = np.random.default_rng(2002)
    x = (rng.uniform(-1, 1, (2, 3, 5)) + 1j * rng.uniform(-1, 1, (2, 3, 5))).astype(np.complex64)
    xc = (rng.uniform(-1, 1, (3, 4, 5)) + 1j * rng.uniform(-1, 1, (3, 4, 5))).astype(np.complex64)
    g = rng.uniform(0, 1, (3, 4, 5)).astype(np.float32)
    return x, xc, g


def main():
    x, xc, g = inputs()
    _write(os.path.join(HERE, "dft3_forward_2x3x5.txt"),
           "# Eq. (1) forward DFT of a seeded 2x3x5 complex64 grid (oracle.forward, float64)", x, oracle.forward(x))
    _write(os.path.join(HERE, "dft3_backward_2x3x5.txt"),
           "# Eq. (2) backward DFT, unnormalised, of the same grid (oracle.backward, float64)", x, oracle.backward(x))
    _write(os.path.join(HERE, "convolve_3x4x5.txt"),
           "# B(G * F(x)) of a seeded 3x4x5 grid with the influence function in convolve_3x4x5_g.txt (oracle.convolve)",
           xc, oracle.convolve(xc, g))
    with open(os.path.join(HERE, "convolve_3x4x5_g.txt"), "w") as f:
        f.write("# influence function G(kx, ky, kz) of convolve_3x4x5.txt, float32, C order\n")
        for idx in np.ndindex(*g.shape):
            f.write(f"{idx[0]} {idx[1]} {idx[2]} {g[idx]:.9g}\n")


if __name__ == "__main__":
    main()
