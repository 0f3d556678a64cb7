"""The kernels' bounded waits, made to run out without any fault: a run
created with a fault-injection bit withholds one copy (a row of J the step
kernel stages by TMA, or an operand tile of the tensor-core recompute), so
the wait for it expires after about two seconds; the kernel lets its other
copies and MMAs finish, returns, and the call reports SK_ERR_TIMEOUT.  The
context stays usable: a new run on the same instance then follows the
oracle bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _clean_run_matches_oracle(inst, J, init, staged):
    run = sk.Run(inst, chains=init.shape[0], K=8, beta=0.9, seed=3, init=init)
    b = sk.Batch([run])
    if staged:
        b.set_layout(32, 1)
    b.advance(300)
    b.close()
    s, _ = run.state()
    run.close()
    o = oracle.run(J, K=8, beta=0.9, seed=3, chains=init.shape[0], init=init, steps=300)
    assert np.array_equal(s, o["spins"])


def test_step_kernel_row_wait_expires_and_returns():
    need_gpu()
    N = 256
    J = inputs.couplings_pm1(N, 21)
    init = inputs.initial_spins(4, N, 22)
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=4, K=8, seed=3, init=init, fault_inject=sk.SK_FAULT_WITHHOLD_ROW)
    b = sk.Batch([run])
    b.set_layout(32, 1)   # rows staged by TMA
    b.advance(20)
    with pytest.raises(sk.SKError) as e:
        run.wait()
    assert e.value.status == sk.SK_ERR_TIMEOUT
    b.close()
    run.close()
    _clean_run_matches_oracle(inst, J, init, staged=True)
    inst.close()


def test_recompute_tile_wait_expires_and_returns():
    need_gpu()
    N = 256
    J = inputs.couplings_pm1(N, 23)
    init = inputs.initial_spins(130, N, 24)
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=130, K=8, seed=3, init=init, fault_inject=sk.SK_FAULT_WITHHOLD_TILE)
    run.advance(10)
    run.wait()
    with pytest.raises(sk.SKError) as e:
        run.recompute(sk.SK_RECOMPUTE_CHECK)
    assert e.value.status == sk.SK_ERR_TIMEOUT
    run.close()
    clean = sk.Run(inst, chains=130, K=8, seed=3, init=init)
    clean.advance(10)
    st, _ = clean.recompute(sk.SK_RECOMPUTE_CHECK)
    assert st["mismatches"] == 0 and st["max_field_drift"] == 0.0
    clean.close()
    _clean_run_matches_oracle(inst, J, init[:4], staged=False)
    inst.close()


def test_unknown_fault_bits_are_rejected():
    need_gpu()
    inst = sk.Instance(inputs.couplings_pm1(32, 1))
    with pytest.raises(sk.SKError) as e:
        sk.Run(inst, chains=2, K=4, fault_inject=4)
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    inst.close()
