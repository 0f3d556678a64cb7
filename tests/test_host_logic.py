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



# ---------------------------------------------------------------------------
# the allocation-free entry point's binding checks its buffers before the C
# call (which trusts the pointers it is given); on the CPU every rejection is
# raised before the library is loaded
# ---------------------------------------------------------------------------
import pytest  # noqa: E402


def _noalloc_args(torch, **over):
    N, chains = 16, 4
    a = dict(couplings=torch.zeros((N, N), dtype=torch.float32),
             spins=torch.ones((chains, N), dtype=torch.int8),
             energy=torch.zeros(chains, dtype=torch.float64))
    a.update(over)
    return a


@pytest.mark.parametrize("over,exc,msg", [
    (dict(couplings="float64"), TypeError, "couplings must be int8"),
    (dict(couplings="int32"), TypeError, "couplings must be int8"),
    (dict(spins="int32"), TypeError, "spins must be int8"),
    (dict(energy="float32"), TypeError, "energy must be float64"),
    (dict(couplings="nonsquare"), ValueError, "square"),
    (dict(couplings="3d"), ValueError, "square"),
    (dict(spins="wrong_n"), ValueError, "shape (chains, 16)"),
    (dict(spins="1d"), ValueError, "shape (chains, 16)"),
    (dict(energy="short"), ValueError, "hold 4 values"),
    (dict(spins="noncontig"), ValueError, "spins must be contiguous"),
    (dict(couplings="noncontig"), ValueError, "couplings must be contiguous"),
    (dict(), ValueError, "one CUDA device"),
    (dict(couplings="numpy"), TypeError, "couplings must be a torch tensor"),
])
def test_run_noalloc_rejects_bad_buffers(over, exc, msg):
    torch = pytest.importorskip("torch")
    from paper_2102_05613_gb300 import sk
    N, chains = 16, 4
    make = {
        ("couplings", "float64"): lambda: torch.zeros((N, N), dtype=torch.float64),
        ("couplings", "int32"): lambda: torch.zeros((N, N), dtype=torch.int32),
        ("spins", "int32"): lambda: torch.ones((chains, N), dtype=torch.int32),
        ("energy", "float32"): lambda: torch.zeros(chains, dtype=torch.float32),
        ("couplings", "nonsquare"): lambda: torch.zeros((N, N + 1), dtype=torch.float32),
        ("couplings", "3d"): lambda: torch.zeros((2, N, N), dtype=torch.float32),
        ("spins", "wrong_n"): lambda: torch.ones((chains, N + 1), dtype=torch.int8),
        ("spins", "1d"): lambda: torch.ones(chains * N, dtype=torch.int8),
        ("energy", "short"): lambda: torch.zeros(chains - 1, dtype=torch.float64),
        ("spins", "noncontig"): lambda: torch.ones((N, chains), dtype=torch.int8).t(),
        ("couplings", "noncontig"): lambda: torch.zeros((N, N), dtype=torch.float32).t(),
        ("couplings", "numpy"): lambda: np.zeros((N, N), dtype=np.float32),
    }
    args = _noalloc_args(torch, **{k: make[(k, v)]() for k, v in over.items()})
    loaded = sk._lib
    with pytest.raises(exc) as e:
        sk.run_noalloc(args["couplings"], args["spins"], args["energy"], K=8, steps=1)
    assert msg in str(e.value)
    assert sk._lib is loaded  # rejected before the library was touched
