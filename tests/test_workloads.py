"""Host logic of the seeded workloads (no GPU, no oracle)."""
import numpy as np


def test_stratified_sample_with_scattered_cells():
    """The bounded samples the benchmark and tests take: per_cell lanes of
    every cell in lane order, also when a cell's lanes are not contiguous
    (mixed study), with an optional per-cell offset."""
    from paper_2304_02731_gb300 import workloads as W
    wl = W.mixed_ca_h(n=50_000, seed=3)
    for per, skip in [(1, 0), (7, 0), (5, 3)]:
        idx = W.stratified(wl, per, skip=skip)
        assert np.all(np.diff(idx) > 0)
        for c in range(wl.n_cells):
            lanes = np.flatnonzero(wl.cell == c)
            assert np.array_equal(idx[wl.cell[idx] == c], lanes[skip:skip + per])
    sw = W.sweep_h2_ca(per_cell=16, n_E=3, n_b=4)
    idx = W.stratified(sw, 5)
    assert np.array_equal(idx, np.concatenate([np.arange(16 * c, 16 * c + 5) for c in range(12)]))
