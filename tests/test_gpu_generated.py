"""Instances whose couplings are drawn on the device from a seed
(sk_create_instance with couplings NULL) against the oracle's separate
implementation of the same generator (Philox domain 2): +-J couplings bit
for bit, Gaussian couplings within one float32 unit in the last place (the
Box-Muller transform's double-precision log and cos come from two different
math libraries), and a +-J trajectory on the drawn instance equal to the
oracle's on its own draw."""
import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [2, 33, 512, 2048])
@pytest.mark.parametrize("kind", [sk.SK_J_PM1, sk.SK_J_GAUSS])
def test_drawn_couplings_match_the_oracle(N, kind):
    need_gpu()
    seed = 1000 + N
    inst = sk.Instance(None, N=N, kind=kind, seed=seed)
    Jg = inst.couplings()
    inst.close()
    Jo = oracle.gen_couplings(N, kind, seed)
    if kind == sk.SK_J_PM1:
        assert np.array_equal(Jg, Jo)
    else:
        ulp = np.spacing(np.abs(Jo).astype(np.float32))
        assert np.all(np.abs(Jg - Jo) <= ulp)
        assert np.count_nonzero(Jg != Jo) <= max(2, N * N // 100000)


def test_trajectory_on_a_drawn_pm1_instance():
    need_gpu()
    N, K, chains, steps, R = 96, 16, 4, 500, 100
    inst = sk.Instance(None, N=N, kind=sk.SK_J_PM1, seed=5)
    init = inputs.initial_spins(chains, N, 6)
    run = sk.Run(inst, chains=chains, K=K, beta=0.8, seed=7, record_every=R, max_records=steps // R, init=init)
    run.advance(steps)
    E, q, acc = run.observables()
    spins, _ = run.state()
    run.close(); inst.close()
    o = oracle.run(oracle.gen_couplings(N, oracle.PM1, 5), K=K, beta=0.8, seed=7, chains=chains, init=init,
                   steps=steps, record_every=R)
    assert np.array_equal(spins, o["spins"]) and np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"])


def test_drawn_instance_rejects_bad_sizes():
    need_gpu()
    with pytest.raises(ValueError):
        sk.Instance(None, N=1, kind=sk.SK_J_PM1, seed=1)
    with pytest.raises(ValueError):
        sk.Instance(None, N=sk.SK_MAX_N + 1, kind=sk.SK_J_GAUSS, seed=1)
