"""The 2-bit packed genotype layout of gls_solve_*_packed, on the CPU: packing
round-trips, padding bits are zero, numpy and torch agree, codes outside
0..2 are refused (0..3 with allow_code3)."""
import numpy as np
import pytest
import torch

from paper_1210_7325_gb300 import gls


def unpack(b, n):
    nb = b.shape[0]
    u = np.zeros((4 * nb, b.shape[1]), dtype=np.int8)
    for q in range(4):
        u[q::4] = (b >> (2 * q)) & 3
    return u[:n]


@pytest.mark.parametrize("n,k", [(1, 1), (3, 2), (4, 5), (5, 3), (1001, 7)])
def test_round_trip_and_layout(n, k):
    g = np.random.default_rng(n + k)
    X = np.asfortranarray(g.integers(0, 4, size=(n, k)).astype(np.int8))
    b = gls.pack_genotypes(X, allow_code3=True)
    assert b.shape == (gls.packed_rows(n), k) and b.dtype == np.uint8 and b.flags.f_contiguous
    assert np.array_equal(unpack(b, n), X)
    # genotype i sits in bits 2 (i mod 4) of byte i // 4; padding bits are zero
    i = n - 1
    assert ((b[i // 4, 0] >> (2 * (i % 4))) & 3) == X[i, 0]
    if n % 4:
        assert (b[-1, :] >> (2 * (n % 4))).max() == 0
    t = gls.pack_genotypes(torch.from_numpy(np.ascontiguousarray(X.T)).t(), allow_code3=True)
    assert t.stride(0) == 1 and np.array_equal(t.numpy(), b)


@pytest.mark.parametrize("bad,allow", [(-1, False), (3, False), (4, True), (127, True)])
def test_codes_outside_range_refused(bad, allow):
    X = np.zeros((6, 2), dtype=np.int8, order="F")
    X[3, 1] = bad
    with pytest.raises(ValueError):
        gls.pack_genotypes(X, allow_code3=allow)
    with pytest.raises(ValueError):
        gls.pack_genotypes(torch.from_numpy(np.ascontiguousarray(X.T)).t(), allow_code3=allow)
