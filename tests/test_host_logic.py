"""Arithmetic identities the CUDA kernels rely on, checked exhaustively on the
CPU over the ranges the library admits (no GPU needed)."""
import numpy as np


def test_tree_parent_reciprocal_is_exact():
    """The graph kernel finds a tree node's parent (v - 1) // k as the high 32
    bits of (v - 1) * kinv with kinv = floor((2^32 - 1) / k) + 1 = ceil(2^32 / k);
    exact for every arity 2 <= k <= 8191 and node v < 8192 (the template has at
    most 8192 nodes)."""
    x = np.arange(0, 8191, dtype=np.uint64)  # v - 1
    for k in range(2, 8192):
        kinv = np.uint64(0xFFFFFFFF // k + 1)
        assert np.array_equal((x * kinv) >> np.uint64(32), x // np.uint64(k)), k

