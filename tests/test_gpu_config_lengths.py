"""Parity at the lengths and parameters the workloads run.

The fp32 field drift that the Gaussian replay tolerance is derived for grows
with the number of steps (as sqrt(f T) 2^-24 |h|), so the tolerance is checked
here at the longest configured runs, and the ensemble test at configured
(N, K, beta):
  - Gaussian SK N = 512, J ~ N(0, 1/N) fp32, records every 100 steps, 1e4 steps
    without resynchronisation: decision replay of every step of 4 chains for
    K = 128 at beta = 1 and 3, K = 32 at beta = 2 and Metropolis at beta = 1;
    final energy per spin within 1e-5 of the FP64 energy, fields within 1e-4;
  - N = 2048, K = 64, beta = 2, 4096 steps with the tensor-core field
    recompute every 256 steps: +-J with the FP8 check (trajectory bit-exact,
    0 mismatches), Gaussian with the split-bf16 resync (decision replay);
  - independent GPU (4096 chains) and oracle (512 chains) ensembles at N = 512:
    E/N, |q| and acceptance per record within 3 sigma (at most 10 % of the
    points beyond 3 sigma, none beyond 4.5).
"""
import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

REPLAY_TOL = 1e-4
E_PER_SPIN_TOL = 1e-5


@pytest.mark.parametrize("rule,K,beta", [
    (sk.SK_RULE_MCMCMC, 128, 1.0),
    (sk.SK_RULE_MCMCMC, 128, 3.0),
    (sk.SK_RULE_MCMCMC, 32, 2.0),
    (sk.SK_RULE_METROPOLIS, 1, 1.0),
])
def test_gauss_n512_replay_over_1e4_steps(rule, K, beta):
    need_gpu()
    N, chains, steps, R = 512, 4, 10_000, 100
    J = inputs.couplings_gauss(N, 0)
    init = inputs.initial_spins(chains, N, 5)
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=beta, seed=1, stream_id=0, record_every=R,
                 max_records=steps // R, init=init, trace_chains=chains, trace_steps=steps)
    run.advance(steps)
    E, _, _ = run.observables()
    spins, h, _ = run.state(fields=True)
    tr = run.trace()
    run.close(); inst.close()
    orule = oracle.METROPOLIS if rule == sk.SK_RULE_METROPOLIS else oracle.MCMCMC
    for c in range(chains):
        r = oracle.replay(J, tr[c], rule=orule, K=K, beta=beta, seed=1, stream=0, chain=c, init=init[c],
                          tol=REPLAY_TOL)
        assert r["bad"] == 0, (c, r)
        assert r["disagree"] <= 10, (c, r)
        assert np.array_equal(r["spins"], spins[c])
        assert abs(E[-1, c] - oracle.energy(J, spins[c])) / N <= E_PER_SPIN_TOL
        hx = J.astype(np.float64) @ spins[c].astype(np.float64)
        assert np.abs(h[c] - hx).max() < 1e-4


def test_pm1_n2048_fp8_check_every_256_steps_bit_exact():
    need_gpu()
    N, chains, K, beta, steps, R = 2048, 8, 64, 2.0, 4096, 256
    J = inputs.couplings_pm1(N, 2048)
    init = inputs.initial_spins(chains, N, 6)
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=chains, K=K, beta=beta, seed=5, init=init, recompute_every=256,
                 record_every=R, max_records=steps // R)
    run.advance(steps)
    E, q, acc = run.observables()
    spins, h, _ = run.state(fields=True)
    st = run.recompute_stats()
    run.close(); inst.close()
    assert st["recomputes"] == steps // 256 and st["mismatches"] == 0 and st["max_field_drift"] == 0.0
    o = oracle.run(J, K=K, beta=beta, seed=5, chains=chains, init=init, steps=steps, record_every=R)
    assert np.array_equal(spins, o["spins"])
    assert np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"]) and np.array_equal(q, o["q"])
    assert np.array_equal(h, (J.astype(np.int64) @ spins.T.astype(np.int64)).T)


def test_gauss_n2048_bf16_resync_every_256_steps_replay():
    need_gpu()
    N, chains, K, beta, steps, R = 2048, 2, 64, 2.0, 4096, 256
    J = inputs.couplings_gauss(N, 2049)
    init = inputs.initial_spins(chains, N, 7)
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=chains, K=K, beta=beta, seed=5, init=init, recompute_every=256,
                 recompute_terms=3, record_every=R, max_records=steps // R, trace_chains=chains,
                 trace_steps=steps)
    run.advance(steps)
    E, _, _ = run.observables()
    spins, h, _ = run.state(fields=True)
    tr = run.trace()
    st = run.recompute_stats()
    run.close(); inst.close()
    assert st["recomputes"] == steps // 256 and st["max_field_drift"] < 1e-4
    for c in range(chains):
        r = oracle.replay(J, tr[c], K=K, beta=beta, seed=5, chain=c, init=init[c], tol=REPLAY_TOL)
        assert r["bad"] == 0, (c, r)
        assert np.array_equal(r["spins"], spins[c])
        assert abs(E[-1, c] - oracle.energy(J, spins[c])) / N <= E_PER_SPIN_TOL
        hx = J.astype(np.float64) @ spins[c].astype(np.float64)
        assert np.abs(h[c] - hx).max() < 1e-4


@pytest.mark.parametrize("K,beta", [(128, 1.0), (32, 3.0)])
def test_gauss_n512_ensembles_within_3_sigma(K, beta):
    need_gpu()
    N, steps, R = 512, 1000, 100
    J = inputs.couplings_gauss(N, 1)
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=4096, K=K, beta=beta, seed=100, record_every=R, max_records=steps // R)
    run.advance(steps)
    gE, gq, gacc = run.observables()
    run.close(); inst.close()
    o = oracle.run(J, K=K, beta=beta, seed=200, chains=512, steps=steps, record_every=R)
    zs = []
    for a, b in ((gE / N, o["E"] / N), (np.abs(gq), np.abs(o["q"])),
                 (gacc.astype(float), o["acc"].astype(float))):
        se = np.sqrt(a.var(axis=1, ddof=1) / a.shape[1] + b.var(axis=1, ddof=1) / b.shape[1])
        zs.append((a.mean(axis=1) - b.mean(axis=1)) / np.maximum(se, 1e-12))
    zs = np.concatenate(zs)
    assert np.mean(np.abs(zs) > 3) <= 0.1 and np.abs(zs).max() < 4.5, zs
