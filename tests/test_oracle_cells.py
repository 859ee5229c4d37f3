"""Oracle of the cell-based model map pinned to closed forms: constants are preserved, an
interior node sees the mean of its 2^D cells (exact for fields linear in the cell
centres), and the counts of adjacent cells are the textbook 8 / 4 / 2 / 1."""
import numpy as np

from paper_2609_14982_b300 import workloads as W


def test_cell_average_closed_forms(oracle_mod):
    n = (6, 5, 4)
    g = W.Grid(3, n, (1.0, 1.0, 1.0), np.zeros((int(np.prod(n)), 3)))
    A = oracle_mod.cell_average(g)
    assert A.shape == (120, 60)
    assert np.allclose(A @ np.ones(60), 1.0, atol=0, rtol=1e-15)
    nadj = np.diff(A.indptr).reshape(n)
    assert nadj[0, 0, 0] == 1 and nadj[0, 0, 1] == 2 and nadj[0, 1, 1] == 4 and nadj[2, 2, 2] == 8
    # a field linear in the cell centres (c + 1/2) is reproduced at interior nodes
    ci = np.meshgrid(*[np.arange(m - 1) + 0.5 for m in n], indexing="ij")
    f = (2.0 * ci[0] - 3.0 * ci[1] + 0.5 * ci[2]).ravel()
    ni = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    exact = (2.0 * ni[0] - 3.0 * ni[1] + 0.5 * ni[2])
    got = (A @ f).reshape(n)
    assert np.allclose(got[1:-1, 1:-1, 1:-1], exact[1:-1, 1:-1, 1:-1], rtol=0, atol=1e-13)


def test_cell_average_2d_counts(oracle_mod):
    n = (5, 4)
    g = W.Grid(2, n, (1.0, 1.0), np.zeros((20, 2)))
    A = oracle_mod.cell_average(g)
    assert A.shape == (20, 12)
    nadj = np.diff(A.indptr).reshape(n)
    assert nadj[0, 0] == 1 and nadj[0, 1] == 2 and nadj[2, 2] == 4
