"""Pins of the oracle's sparse B0' (Sec. 3.3: the sparsity analysis of B and the drop-tolerance filter of
Eq. filtereq, reading R8) against the paper's numbers and closed form and against the dense operator."""

import os

import numpy as np

from oracle import grid, ib
from paper_2103_06415_gb300 import workloads as wl

from runners import oracle_history, oracle_sim

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sine_cosine_cross(n):
    """Discrete S_x C_x^T with orthonormal DST-I (Dirichlet points) and DCT-II without the constant vector
    (Neumann points at cell centres), as in the analysis of Sec. 3.3.1."""
    k = np.arange(1, n)
    s = np.sqrt(2.0 / n) * np.sin(np.pi * np.outer(np.arange(1, n), k) / n)
    c = np.sqrt(2.0 / n) * np.cos(np.pi * np.outer(np.arange(n) + 0.5, k) / n)
    return s @ c.T


def test_filter_keeps_entries_strictly_above_tolerance_times_column_diagonal():
    b = np.array([0.014, -0.014, 0.01400001, -0.0140001, 2.0, 1e-3, -0.5, 0.0])
    out = ib.drop_filter(b, 4, 0.007)                        # threshold 0.007 * |b_4| = 0.014
    assert np.array_equal(out, [0.0, 0.0, 0.01400001, -0.0140001, 2.0, 0.0, -0.5, 0.0])
    assert ib.drop_filter(b, 4, 0.0) is b                     # no tolerance: the column itself


def test_zero_drop_tolerance_reproduces_dense_b0_and_filter_only_removes_entries():
    lev = grid.Level(24, 20, 0.1, 0.0, 0.0)
    sd = ib.Subdomain(lev, 6, 13, 5, 12)
    dense = ib.b0_dense(sd, 100.0, 0.004)
    for col in (0, 17, sd.n_sd + 30, 2 * sd.n_sd - 1):
        assert np.array_equal(ib.b0_column(sd, col, 100.0, 0.004, 0.0), dense[:, col])
        f = ib.b0_column(sd, col, 100.0, 0.004, 0.007)
        kept = f != 0.0
        assert np.array_equal(f[kept], dense[kept, col])
        assert np.all(np.abs(dense[~kept, col]) <= 0.007 * abs(dense[col, col]))
        assert kept[col] and kept.sum() < kept.size


def test_paper_sixty_kept_entries_per_row_of_sine_cosine_cross_product():
    """Sec. 3.3.1: ~60 entries per row of S_x C_x^T above 1e-2, on 500 x 500 and irrespective of size."""
    vals = dict(l.split() for l in open(os.path.join(GOLDEN, "paper_sparsity_nnz.txt")) if l[0] != "#")
    n0, col, tol, nnz = int(vals["grid"]), int(vals["column"]), float(vals["tolerance"]), int(vals["nnz_per_row"])
    counts = []
    for n in (n0 // 2, n0, 2 * n0):
        m = _sine_cosine_cross(n)
        counts.append(int(np.sum(np.abs(m[:, col * n // n0]) > tol)))
    assert all(abs(c - nnz) <= 0.1 * nnz for c in counts), counts


def test_sine_cosine_cross_product_follows_the_closed_form_of_eq_offdiag():
    """Eq. offdiag: the continuous analogue of (S_x C_x^T)_(i, j+1), scaled by 1/(L/2), is
    (2/pi)(1/(2i - 2j - 1) + 1/(2i + 2j + 1)); the discrete column decays like it, as 1/|i - j|."""
    n, j = 500, 250
    m = _sine_cosine_cross(n)
    i = np.arange(1, n)
    cont = (2.0 / np.pi) * (1.0 / (2 * i - 2 * j - 1) + 1.0 / (2 * i + 2 * j + 1))
    assert np.max(np.abs(m[:, j] - cont)) < 5e-3 * np.max(np.abs(cont))


def test_kept_entries_per_column_stay_flat_as_the_grid_is_refined():
    """Sec. 3.3.1: at fixed alpha = dt/(2 Re h^2) = 1/8 a column of B0' keeps about as many entries on a
    finer grid (the decay is in grid units), once Omega_0 is larger than the kept region."""
    counts = []
    for n in (64, 128, 256):
        h = 1.0 / n
        lev = grid.Level(n, n, h, 0.0, 0.0)
        sd = ib.Subdomain.from_box(lev, 0.3, 0.7, 0.3, 0.7)
        p = (sd.nj // 2) * sd.ni + sd.ni // 2
        counts.append([int(np.sum(ib.b0_column(sd, c * sd.n_sd + p, 1.0 / h, h / 4.0, 0.007) != 0))
                       for c in (0, 1)])
    counts = np.array(counts, dtype=float)
    assert np.all(np.abs(counts[2] - counts[1]) < 0.05 * counts[2])
    assert np.all(np.abs(counts[1] - counts[0]) < 0.15 * counts[2])
    assert counts[2].max() < 0.1 * (2 * 101 ** 2)          # a small fraction of the dense column


def test_sparse_b0_forces_within_two_percent_of_dense():
    """With the paper's drop tolerance 0.007 the force and angle histories stay within 2 % of the dense
    operator's (cf. Sec. 5.1)."""
    w = wl.small_plate()
    hist = []
    for tol in (0.0, 0.007):
        sim = oracle_sim(w, drop_tol=tol)
        for _ in range(10):
            sim.step()
        hist.append(oracle_history(sim))
    for k in range(5):
        assert np.max(np.abs(hist[1][:, k] - hist[0][:, k])) < 0.02 * np.max(np.abs(hist[0][:, k])), k
