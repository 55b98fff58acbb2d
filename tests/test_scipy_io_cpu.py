"""Host-side conversion between scipy.sparse matrices and the plan's CSR arrays (no GPU)."""
import numpy as np
import scipy.sparse as sp

import paper_1710_10899_gb300 as sm


def test_csr_arrays_sorts_sums_duplicates_and_keeps_stored_zeros():
    # COO with an unsorted row, a duplicate (summed) and an explicitly stored zero
    r = np.array([0, 0, 1, 1, 1, 2, 2, 0])
    c = np.array([2, 0, 1, 0, 1, 2, 0, 2])
    v = np.array([1.0, 4.0, 3.0, 1.0, 2.0, 5.0, 0.0, 0.5])
    coo = sp.coo_matrix((v, (r, c)), shape=(3, 3))
    rp, ci, vals = sm.csr_arrays(coo)
    assert rp.dtype == np.int32 and ci.dtype == np.int32 and vals.dtype == np.float64
    np.testing.assert_array_equal(rp, [0, 2, 4, 6])
    np.testing.assert_array_equal(ci, [0, 2, 0, 1, 0, 2])
    np.testing.assert_array_equal(vals, [4.0, 1.5, 1.0, 5.0, 0.0, 5.0])
    back = sm.scipy_csr(rp, ci, vals)
    np.testing.assert_array_equal(back.toarray(), coo.toarray())
    assert back.nnz == 6                       # the stored zero is still stored


def test_csr_arrays_rejects_non_square():
    import pytest
    with pytest.raises(ValueError):
        sm.csr_arrays(sp.random(3, 4, density=0.5, random_state=0))
