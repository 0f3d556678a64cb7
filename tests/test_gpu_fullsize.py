"""Parity at the benchmark's full size and in the launch configuration it
times: Gaussian SK N = 512, 64 instances x 4096 chains, MCMCMC K = 128,
beta = 1, one autotuned batch.  The oracle recomputes sampled chains one by
one: decision replay on their slot logs (Gaussian) and bit-exact
trajectories for a +-J twin of the workload."""
import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

N, INSTANCES, CHAINS, K, BETA, STEPS, R = 512, 64, 4096, 128, 1.0, 200, 100
SAMPLED = [(0, 0), (0, 4095), (17, 1234), (63, 2049)]  # (instance, chain)
TRACE = 4096  # every chain of an instance logs its slots (the sampled ones are checked)


@pytest.mark.parametrize("kind", [sk.SK_J_GAUSS, sk.SK_J_PM1])
def test_full_size_sampled_chains(kind):
    torch = need_gpu()
    st = torch.cuda.Stream()
    Js = [inputs.couplings(N, kind, i) for i in range(INSTANCES)]
    insts = [sk.Instance(J, stream=st) for J in Js]
    runs = [sk.Run(x, chains=CHAINS, K=K, beta=BETA, seed=1, stream_id=i, record_every=R,
                   max_records=STEPS // R, trace_chains=TRACE if i in (0, 17, 63) else 0,
                   trace_steps=STEPS if i in (0, 17, 63) else 0)
            for i, x in enumerate(insts)]
    b = sk.Batch(runs)
    b.autotune(trial_steps=10)
    b.advance(R)
    b.advance(STEPS - R)
    for inst_i, chain in SAMPLED:
        run = runs[inst_i]
        J = Js[inst_i]
        E, q, acc = run.observables()
        spins, h, _ = run.state(fields=True)
        tr = run.trace()[chain]
        init = oracle.init_spins(1, inst_i, chain, N)
        if kind == sk.SK_J_PM1:
            o = oracle.run(J, K=K, beta=BETA, seed=1, stream=inst_i, chain0=chain, chains=1,
                           steps=STEPS, record_every=R, trace=True, want_q=False)
            assert np.array_equal(tr, o["trace"][0])
            assert np.array_equal(E[:, chain], o["E"][:, 0])
            assert np.array_equal(acc[:, chain], o["acc"][:, 0])
            assert np.array_equal(spins[chain], o["spins"][0])
            assert np.array_equal(h[chain], J.astype(np.int64) @ spins[chain].astype(np.int64))
        else:
            r = oracle.replay(J, tr, K=K, beta=BETA, seed=1, stream=inst_i, chain=chain, init=init,
                              tol=1e-4)
            assert r["bad"] == 0 and r["disagree"] <= 2, r
            assert np.array_equal(r["spins"], spins[chain])
            assert abs(E[-1, chain] - oracle.energy(J, spins[chain])) / N <= 1e-5
    b.close()
    for r in runs:
        r.close()
    for x in insts:
        x.close()
