"""The continuous-batching request server: jobs of different N, couplings,
K, beta, rule and length that arrive while others run are admitted by device
footprint, share launches, and each result equals the same job run alone
(bit for bit: the draws are counter-based and every kernel is deterministic).
The +-J jobs' results also equal the FP64 oracle's trajectories bit for bit,
and every job's energies equal the oracle's energies of its final spins."""
import time

import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

JOBS = [  # N, kind, chains, K, rule, beta, steps, seed
    (64, sk.SK_J_PM1, 4, 8, sk.SK_RULE_MCMCMC, 1.0, 1500, 1),
    (200, sk.SK_J_GAUSS, 10, 40, sk.SK_RULE_MCMCMC, 0.7, 700, 2),
    (513, sk.SK_J_PM1, 3, 256, sk.SK_RULE_MCMCMC, 2.0, 400, 3),
    (128, sk.SK_J_GAUSS, 6, 1, sk.SK_RULE_METROPOLIS, 1.0, 3000, 4),
    (96, sk.SK_J_PM1, 1, 16, sk.SK_RULE_MCMCMC, 0.5, 2200, 5),
    (300, sk.SK_J_GAUSS, 7, 100, sk.SK_RULE_MCMCMC, 1.5, 900, 6),
]
P_CENTER = {1: 0.1, 4: 0.4}  # jobs with a non-uniform root of the star


def _alone(J, N, chains, K, rule, beta, steps, seed, stream_id, init, p_center=0.0):
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=beta, seed=seed, stream_id=stream_id,
                 init=init, p_center=p_center)
    run.advance(steps)
    spins, _ = run.state()
    E = inst.energy(spins)
    run.close(); inst.close()
    return E, spins


def test_results_in_the_mix_equal_results_alone():
    need_gpu()
    srv = sk.Server(budget_bytes=2 << 30, quantum_steps=64)
    data = []
    tickets = []
    for i, (N, kind, chains, K, rule, beta, steps, seed) in enumerate(JOBS):
        J = inputs.couplings(N, kind, 500 + i)
        init = inputs.initial_spins(chains, N, 600 + i) if i % 2 == 0 else None
        data.append((J, init))
        if i == 3:
            time.sleep(0.05)  # later arrivals join while the first jobs run
        tickets.append(srv.submit(N=N, kind=kind, chains=chains, steps=steps, K=K, rule=rule,
                                  beta=beta, seed=seed, stream_id=i, J=J, init=init,
                                  p_center=P_CENTER.get(i, 0.0)))
    srv.wait_all(timeout_ns=120 * 10**9)
    status = [srv.poll(t) for t in tickets]
    assert all(s["state"] == sk.SK_JOB_DONE for s in status), status
    for i, (t, (N, kind, chains, K, rule, beta, steps, seed)) in enumerate(zip(tickets, JOBS)):
        E, S, _ = srv.result(t, chains, N)
        J, init = data[i]
        E0, S0 = _alone(J, N, chains, K, rule, beta, steps, seed, i, init, P_CENTER.get(i, 0.0))
        assert np.array_equal(S, S0), i
        assert np.array_equal(E, E0), i
        # the job's energies are the FP64 energies of its spins (exact for +-J)
        Eo = np.array([oracle.energy(J, S[c]) for c in range(chains)])
        assert np.abs(E - Eo).max() <= (0.0 if kind == sk.SK_J_PM1 else 1e-9 * N), i
        if kind == sk.SK_J_PM1:  # the oracle's trajectory, bit for bit
            orule = oracle.METROPOLIS if rule == sk.SK_RULE_METROPOLIS else oracle.MCMCMC
            o = oracle.run(J, rule=orule, K=K, beta=beta, seed=seed, stream=i, chains=chains,
                           init=init, steps=steps, p_center=P_CENTER.get(i, 0.0))
            assert np.array_equal(S, o["spins"]), i
    st = srv.stats()
    assert st["completed"] == len(JOBS) and st["chain_steps"] > 0
    # the worker's host time between quanta, by phase, within the wall time
    phases = st["admit_seconds"] + st["retire_seconds"] + st["plan_seconds"]
    assert min(st["admit_seconds"], st["retire_seconds"], st["plan_seconds"]) > 0
    assert phases + st["busy_seconds"] <= st["elapsed_seconds"]
    # work overlapped: some job was admitted before another one finished
    starts = sorted((s["t_admit"], s["t_done"]) for s in status)
    assert any(b[0] < a[1] for a, b in zip(starts, starts[1:]))
    srv.close()


def test_admission_by_footprint_and_oversized_jobs():
    need_gpu()
    N, chains = 1024, 64
    J = inputs.couplings_gauss(N, 9)
    # each job needs ~10 MB of couplings and their tensor-core operand + ~0.5 MB
    # of state: two fit, not three
    srv = sk.Server(budget_bytes=24 << 20, quantum_steps=128)
    ts = [srv.submit(N=N, kind=sk.SK_J_GAUSS, chains=chains, steps=1024, K=32, seed=k,
                     stream_id=k, J=J) for k in range(4)]
    big = srv.submit(N=2048, kind=sk.SK_J_GAUSS, chains=8, steps=10, K=8,
                     J=inputs.couplings_gauss(2048, 1))
    srv.wait_all(timeout_ns=120 * 10**9)
    st = [srv.poll(t) for t in ts]
    assert all(s["state"] == sk.SK_JOB_DONE for s in st)
    # the third job had to wait for one of the first two to finish
    admits = sorted(s["t_admit"] for s in st)
    dones = sorted(s["t_done"] for s in st)
    assert admits[2] >= dones[0]
    b = srv.poll(big)
    assert b["state"] == sk.SK_JOB_FAILED and b["error"] == sk.SK_ERR_OOM
    for k, t in enumerate(ts):
        E, S, _ = srv.result(t, chains, N)
        E0, S0 = _alone(J, N, chains, 32, sk.SK_RULE_MCMCMC, 1.0, 1024, k, k, None)
        assert np.array_equal(S, S0)
    srv.close()


def test_shared_couplings_stay_resident():
    need_gpu()
    N = 256
    J = inputs.couplings_pm1(N, 4)
    srv = sk.Server(budget_bytes=1 << 30, quantum_steps=100)
    srv.add_couplings(7, J)
    ts = [srv.submit(N=N, kind=sk.SK_J_PM1, chains=5, steps=500 + 100 * k, K=24, seed=k,
                     stream_id=k, couplings_id=7) for k in range(5)]
    srv.wait_all(timeout_ns=60 * 10**9)
    for k, t in enumerate(ts):
        E, S, _ = srv.result(t, 5, N)
        E0, S0 = _alone(J, N, 5, 24, sk.SK_RULE_MCMCMC, 1.0, 500 + 100 * k, k, k, None)
        assert np.array_equal(S, S0) and np.array_equal(E, E0)
    srv.close()
