"""Discrete-variable-representation levels (test infrastructure only).

The paper computes the internal energies E_vj with the DVR of Colbert and
Miller ("A novel discrete variable representation for quantum mechanical
reactive scattering via the S-matrix Kohn method", J. Chem. Phys. 96 (1992)
1982), particle-in-a-box basis on an interval (a, b) with N - 1 interior
grid points (Sec. 2.1 and Sec. 3.1: npts, xmin, xmax).  Here it serves as an
independent cross-check of the Bohr-Sommerfeld levels: for a Morse pair
with j = 0 both reproduce the exact Morse spectrum; for j > 0 the quantum
(DVR) and semiclassical (Bohr-Sommerfeld) levels differ by small
higher-order terms in hbar.

Hamiltonian on the grid x_i = a + i (b - a)/N, i = 1..N-1 (hbar = 1):
  T_ii  = K [ (2N^2 + 1)/3 - 1/sin^2(pi i / N) ]
  T_ik  = K (-1)^(i-k) [ 1/sin^2(pi (i-k)/(2N)) - 1/sin^2(pi (i+k)/(2N)) ]
  K     = pi^2 / (2 mu 2 (b - a)^2)
  H     = T + diag(V(x_i) + j(j+1)/(2 mu x_i^2)),
diagonalised with numpy's symmetric eigensolver.
"""
from __future__ import annotations

import numpy as np

from . import pair_potential


def dvr_levels(pair, mu: float, j: int, a: float, b: float, npts: int):
    """Sorted eigenvalues of the radial Hamiltonian of `pair` (oracle OPair)
    with centrifugal term j(j+1)/(2 mu r^2) on (a, b) with npts intervals."""
    N = int(npts)
    i = np.arange(1, N)
    x = a + (b - a) * i / N
    V = np.array([pair_potential(pair, r)[0] for r in x]) + j * (j + 1) / (2.0 * mu * x * x)
    K = np.pi ** 2 / (2.0 * mu * 2.0 * (b - a) ** 2)
    I, Kk = np.meshgrid(i, i, indexing="ij")
    with np.errstate(divide="ignore"):
        off = (1.0 / np.sin(np.pi * (I - Kk) / (2 * N)) ** 2
               - 1.0 / np.sin(np.pi * (I + Kk) / (2 * N)) ** 2)
    T = K * np.where(((I - Kk) % 2) == 0, 1.0, -1.0) * off
    T[np.diag_indices_from(T)] = K * ((2.0 * N * N + 1.0) / 3.0 - 1.0 / np.sin(np.pi * i / N) ** 2)
    return np.linalg.eigvalsh(T + np.diag(V))


def bound_levels(pair, mu: float, j: int, a: float, b: float, npts: int, E_top: float = 0.0):
    """DVR eigenvalues below E_top (the bound part of the spectrum)."""
    E = dvr_levels(pair, mu, j, a, b, npts)
    return E[E < E_top]
