"""Host arithmetic of libgf that needs no GPU."""
import numpy as np
import pytest

from oracle import dmft
from paper_1111_2157_gb300 import gf as gfm


@pytest.mark.parametrize("U,J,l,n", [(8.0, 1.0, 2, 8.0), (6.0, 0.0, 3, 1.0), (6.0, 0.7, 0, 1.0),
                                     (5.5, 0.6, 3, 9.0)])
def test_double_counting_entry_matches_oracle(U, J, l, n):
    got = gfm.double_counting(U, J, l, n)
    assert np.allclose(got, dmft.double_counting(U, J, l, n), rtol=1e-15, atol=0)


def test_double_counting_rejects_bad_input():
    with pytest.raises(gfm.GFError, match="EINVAL"):
        gfm.double_counting(float("nan"), 0.0, 2, 1.0)
    with pytest.raises(gfm.GFError, match="EINVAL"):
        gfm.double_counting(1.0, 0.0, -1, 1.0)
