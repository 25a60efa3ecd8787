"""Oracle of robust phase estimation (test infrastructure, not product code).

Plain Python, FP64, written from the method (Methods, "Data analysis": RPE
after Kimmel et al. 2015 recovers the dominant frequency of the signal
Z_m = g(delta 2^m), m = 0..M):
  * round 0 reads the phase theta_0 = arg Z_0 in (-pi, pi];
  * round m reads arg Z_m, which is 2^m theta modulo 2 pi: of the 2^m
    candidate angles (arg Z_m + 2 pi k) / 2^m it keeps the one nearest the
    previous round's estimate;
  * the energy is the last estimate divided by delta.
``signal`` evaluates Z_m with this package's own product formula (2^m
first-order Trotter steps of size delta).  Only ``tests/`` may import this
module.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

from . import overlap, trotter


def rpe_estimate(Z, delta: float) -> tuple[float, list[float]]:
    """(energy, [theta_0, ..., theta_M]) for the complex signal Z_0..Z_M."""
    thetas = []
    theta = None
    for m, zm in enumerate(Z):
        phase = cmath.phase(complex(zm))  # in (-pi, pi]
        if m == 0:
            theta = phase
        else:
            scale = 2.0 ** m
            # candidates (phase + 2 pi k) / scale; the nearest to theta is the k
            # that rounds (scale theta - phase) / (2 pi)
            k = math.floor((scale * theta - phase) / (2.0 * math.pi) + 0.5)
            theta = (phase + 2.0 * math.pi * k) / scale
        thetas.append(theta)
    return theta / delta, thetas


def signal(psi0, x, z, h, delta: float, M: int) -> np.ndarray:
    """Z_m = <psi0| U(delta)^(2^m) |psi0> for m = 0..M, U one first-order
    Trotter step exp(i delta h_L P_L) ... exp(i delta h_1 P_1)."""
    out = []
    for m in range(M + 1):
        steps = 1 << m
        psi = trotter(psi0, x, z, h, delta * steps, steps)
        out.append(overlap(psi0, psi))
    return np.array(out, dtype=np.complex128)
