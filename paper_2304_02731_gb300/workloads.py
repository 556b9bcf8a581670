"""Seeded synthetic workloads for the QCT hot path.

This module is shared by the tests, the benchmark and the oracle harness.  It
holds NONE of the method's arithmetic: only the parameters of each workload
(masses in unified atomic mass units, pair-potential parameters in atomic
units, as the H2 + Ca study is specified) and seeded draws of the per-lane
inputs (collision energy, impact parameter, v, j, system index, cell index).
The random orientation / phase of each trajectory is NOT drawn here: each
implementation derives it from (seed, lane id) with its own Philox4x32-10.

Pair-spec kinds (converted to potential parameters by each implementation's
own set-up code):
  ("morse",  De, re, alpha)            V = De (1 - e^{-alpha (r-re)})^2 - De
  ("lj_fit", m, n, De, re)             V = Cm/r^m - Cn/r^n with the well (De, re)
  ("buck",   A, B, C6, r_max_guess)    V = A e^{-B r} - C6 / r^6
Pairs are ordered AB, BC, CA; atom C is the projectile.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# H2 + Ca, H-H Morse and Ca-H Morse parameters of the plain FP64 study.
MASS_H2_CA = (1.00784, 1.00784, 40.078)
HH_MORSE = ("morse", 0.1745, 1.40, 1.03)
CAH_MORSE = ("morse", 0.0630, 3.79, 0.60)
CAH_BUCK = ("buck", 25.0, 1.6, 40.0, 2.0)
CAH_LJ12_6 = ("lj_fit", 12, 6, 0.0630, 3.79)
CAH_LJ8_6 = ("lj_fit", 8, 6, 0.0630, 3.79)

SYS_H2_CA_MORSE = dict(mass_u=MASS_H2_CA, pairs=(HH_MORSE, CAH_MORSE, CAH_MORSE))
SYS_H2_CA_BUCK = dict(mass_u=MASS_H2_CA, pairs=(HH_MORSE, CAH_BUCK, CAH_BUCK))
SYS_H2_CA_LJ12 = dict(mass_u=MASS_H2_CA, pairs=(HH_MORSE, CAH_LJ12_6, CAH_LJ12_6))
SYS_H2_CA_LJ8 = dict(mass_u=MASS_H2_CA, pairs=(HH_MORSE, CAH_LJ8_6, CAH_LJ8_6))

# integration parameters of the FP64 study
INTEG_FP64 = dict(rtol=1e-10, atol=1e-12, r_stop=35.0, t_stop=15.0)
# FP32 study (FP32 cannot honour 1e-10)
INTEG_FP32 = dict(rtol=1e-6, atol=1e-8, r_stop=35.0, t_stop=15.0)
R0 = 30.0


@dataclass
class Workload:
    """Per-lane inputs plus the cell / group bookkeeping used by the reduction."""
    name: str
    systems: list
    E: np.ndarray           # collision energy per lane (hartree)
    b: np.ndarray           # impact parameter per lane (bohr)
    v: np.ndarray           # initial vibrational quantum number
    j: np.ndarray           # initial rotational quantum number
    sys_id: np.ndarray      # index into systems
    cell: np.ndarray        # histogram cell per lane
    cell_b: np.ndarray      # per cell: impact parameter (quadrature abscissa)
    cell_w: np.ndarray      # per cell: quadrature weight of sigma = 2 pi sum w b P
    cell_group: np.ndarray  # per cell: group (one cross section per group)
    n_groups: int
    R0: float = R0
    seed: int = 0
    id_offset: int = 0
    integ: dict = field(default_factory=lambda: dict(INTEG_FP64))

    @property
    def n(self) -> int:
        return int(self.E.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cell_b.shape[0])

    def slice(self, lo: int, hi: int) -> "Workload":
        """Lanes [lo, hi) with the same cells (global ids keep their offset)."""
        return Workload(self.name, self.systems, self.E[lo:hi], self.b[lo:hi], self.v[lo:hi],
                        self.j[lo:hi], self.sys_id[lo:hi], self.cell[lo:hi], self.cell_b,
                        self.cell_w, self.cell_group, self.n_groups, self.R0, self.seed,
                        self.id_offset + lo, dict(self.integ))

    def take(self, idx) -> "Workload":
        """Arbitrary subset of lanes; ids are NOT preserved (use for timing only)."""
        idx = np.asarray(idx)
        return Workload(self.name + "[sub]", self.systems, self.E[idx], self.b[idx],
                        self.v[idx], self.j[idx], self.sys_id[idx], self.cell[idx],
                        self.cell_b, self.cell_w, self.cell_group, self.n_groups, self.R0,
                        self.seed, self.id_offset, dict(self.integ))


def _trapezoid_weights(x: np.ndarray) -> np.ndarray:
    w = np.zeros_like(x)
    d = np.diff(x)
    w[:-1] += 0.5 * d
    w[1:] += 0.5 * d
    return w


def plain_h2_ca(per_b: int = 200, b_grid=(0.0, 1.5, 3.0, 4.5, 6.0), E: float = 0.10,
                v: int = 0, j: int = 0, seed: int = 0) -> Workload:
    """H2(v,j) + Ca, all-Morse, one collision energy, `per_b` lanes per impact
    parameter; lane id = b_index * per_b + k (1,000 lanes by default)."""
    bg = np.asarray(b_grid, np.float64)
    nb = len(bg)
    n = nb * per_b
    cell = np.repeat(np.arange(nb, dtype=np.int32), per_b)
    return Workload(
        name=f"h2ca_plain_E{E}_n{n}", systems=[SYS_H2_CA_MORSE],
        E=np.full(n, E), b=bg[cell].astype(np.float64), v=np.full(n, v, np.int32),
        j=np.full(n, j, np.int32), sys_id=np.zeros(n, np.int32), cell=cell,
        cell_b=bg.copy(), cell_w=_trapezoid_weights(bg), cell_group=np.zeros(nb, np.int32),
        n_groups=1, seed=seed)


def sweep_energies(n_E: int = 16):
    k = np.arange(n_E, dtype=np.float64)
    return 0.02 * 20.0 ** (k / (n_E - 1))


def sweep_h2_ca(per_cell: int = 8192, n_E: int = 16, n_b: int = 24, b_max: float = 10.0,
                seed: int = 0) -> Workload:
    """Batched sweep: n_E energies log-spaced 0.02-0.40 hartree x n_b impact
    parameters on [0, b_max] x per_cell lanes; lane id = (k n_b + l) per_cell + m.
    Defaults: 16 x 24 x 8,192 = 3,145,728 lanes."""
    Es = sweep_energies(n_E)
    bs = b_max * np.arange(n_b, dtype=np.float64) / (n_b - 1)
    n_cells = n_E * n_b
    cell = np.repeat(np.arange(n_cells, dtype=np.int32), per_cell)
    kE = cell // n_b
    lb = cell % n_b
    n = n_cells * per_cell
    cell_b = np.tile(bs, n_E)
    cell_w = np.tile(_trapezoid_weights(bs), n_E)
    group = np.repeat(np.arange(n_E, dtype=np.int32), n_b)
    return Workload(
        name=f"h2ca_sweep_{n_E}x{n_b}x{per_cell}", systems=[SYS_H2_CA_MORSE],
        E=Es[kE], b=bs[lb], v=np.zeros(n, np.int32), j=np.zeros(n, np.int32),
        sys_id=np.zeros(n, np.int32), cell=cell, cell_b=cell_b, cell_w=cell_w,
        cell_group=group, n_groups=n_E, seed=seed)


def stratified(w: Workload, per_cell: int, skip: int = 0) -> np.ndarray:
    """Sorted indices of lanes skip .. skip + per_cell - 1 (in lane order) of
    every cell: a bounded sample that spans every cell, whether or not the
    lanes of a cell are contiguous."""
    order = np.argsort(w.cell, kind="stable")
    c = w.cell[order]
    starts = np.flatnonzero(np.r_[True, c[1:] != c[:-1]])
    ends = np.r_[starts[1:], len(c)]
    idx = [order[min(s + skip, e):min(s + skip + per_cell, e)] for s, e in zip(starts, ends)]
    return np.sort(np.concatenate(idx)) if idx else np.zeros(0, np.int64)


def mixed_ca_h(n: int = 2_000_000, seed: int = 0, n_E_bins: int = 10) -> Workload:
    """Mixed potentials and states: Ca-H as Buckingham, LJ(12,6) or LJ(8,6) in
    equal thirds (lanes sorted by system), v uniform on 0..10, j uniform on
    0..20, E uniform on [0.05, 0.30] hartree, b^2 uniform on [0, 100] bohr^2.
    Cells = system x E-bin x v; groups = system x E-bin.  With b^2 uniform
    the cross section is pi b_max^2 P, i.e. w b = b_max^2 / 2 = 50."""
    rng = np.random.default_rng(seed)
    sys_id = np.sort(rng.integers(0, 3, n)).astype(np.int32)
    E = rng.uniform(0.05, 0.30, n)
    b = np.sqrt(rng.uniform(0.0, 100.0, n))
    v = rng.integers(0, 11, n).astype(np.int32)
    j = rng.integers(0, 21, n).astype(np.int32)
    ebin = np.minimum(((E - 0.05) / 0.25 * n_E_bins).astype(np.int32), n_E_bins - 1)
    cell = ((sys_id * n_E_bins + ebin) * 11 + v).astype(np.int32)
    n_cells = 3 * n_E_bins * 11
    cell_b = np.ones(n_cells)
    cell_w = np.full(n_cells, 50.0)
    group = (np.arange(n_cells) // 11).astype(np.int32)
    return Workload(
        name=f"cah_mixed_n{n}", systems=[SYS_H2_CA_BUCK, SYS_H2_CA_LJ12, SYS_H2_CA_LJ8],
        E=E, b=b, v=v, j=j, sys_id=sys_id, cell=cell, cell_b=cell_b, cell_w=cell_w,
        cell_group=group, n_groups=3 * n_E_bins, seed=seed)


def random_states(n: int, seed: int, v_max: int = 10, j_max: int = 20, E_lo: float = 0.05,
                  E_hi: float = 0.30, b_max: float = 8.0, sys_count: int = 1):
    """Small seeded lane sets for parity tests: (E, b, v, j, sys_id)."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(E_lo, E_hi, n), rng.uniform(0.0, b_max, n),
            rng.integers(0, v_max + 1, n).astype(np.int32),
            rng.integers(0, j_max + 1, n).astype(np.int32),
            np.sort(rng.integers(0, sys_count, n)).astype(np.int32))
