"""Object lifetimes, cancellation and time-outs through the C ABI (host-side
failure handling: nothing here faults or stalls the GPU).

  - an instance with live runs, and a run inside a live batch, refuse to be
    released (SK_ERR_BUSY) and stay usable; released in order they go;
  - mcmcmc_wait with a 1 ns limit on a long advance returns SK_ERR_TIMEOUT,
    and a later unlimited wait returns SK_OK with the same results as a run
    that was never polled;
  - the request server cancels a queued job at once and a running job at the
    next quantum (SK_JOB_CANCELLED, SK_ERR_CANCELLED from its result), and the
    other jobs' results equal those of the same jobs run alone."""
import time

import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_busy_instance_and_run():
    need_gpu()
    J = inputs.couplings_pm1(64, 1)
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=4, K=8, seed=3)
    with pytest.raises(sk.SKError) as e:
        inst.close()
    assert e.value.status == sk.SK_ERR_BUSY
    b = sk.Batch([run])
    with pytest.raises(sk.SKError) as e:
        run.close()
    assert e.value.status == sk.SK_ERR_BUSY
    b.advance(100)           # everything still works
    run.advance(50)
    s, step = run.state()
    assert step == 150
    b.close()
    run.close()
    inst.close()


def test_wait_times_out_then_completes_unchanged():
    need_gpu()
    J = inputs.couplings_gauss(1024, 2)
    init = inputs.initial_spins(2, 1024, 3)
    steps = 400_000   # a few tenths of a second on one GPU

    def one(poll):
        inst = sk.Instance(J)
        run = sk.Run(inst, chains=2, K=32, seed=4, init=init)
        run.advance(steps)
        if poll:
            with pytest.raises(sk.SKError) as e:
                run.wait(1)
            assert e.value.status == sk.SK_ERR_TIMEOUT
        run.wait(0)
        s, step = run.state()
        run.close(); inst.close()
        return s, step

    s1, t1 = one(True)
    s0, t0 = one(False)
    assert t1 == t0 == steps and np.array_equal(s1, s0)


def _alone(J, N, chains, K, beta, steps, seed, stream_id):
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=chains, K=K, beta=beta, seed=seed, stream_id=stream_id)
    run.advance(steps)
    spins, _ = run.state()
    E = inst.energy(spins)
    run.close(); inst.close()
    return E, spins


def test_server_cancels_queued_and_running_jobs():
    need_gpu()
    N = 256
    J = inputs.couplings_pm1(N, 5)
    srv = sk.Server(budget_bytes=1 << 30, quantum_steps=64)
    srv.add_couplings(1, J)
    long_job = srv.submit(N=N, kind=sk.SK_J_PM1, chains=64, steps=2_000_000, K=32, seed=1, stream_id=1,
                          couplings_id=1)
    keep = srv.submit(N=N, kind=sk.SK_J_PM1, chains=6, steps=3000, K=16, seed=2, stream_id=2, couplings_id=1)
    # wait until the long job runs, then cancel it
    t0 = time.time()
    while srv.poll(long_job)["state"] != sk.SK_JOB_RUNNING:
        assert time.time() - t0 < 30
        time.sleep(0.01)
    srv.cancel(long_job)
    srv.cancel(long_job)   # a second cancel is a no-op
    srv.wait_all(timeout_ns=120 * 10**9)
    st = srv.poll(long_job)
    assert st["state"] == sk.SK_JOB_CANCELLED and st["error"] == sk.SK_ERR_CANCELLED
    with pytest.raises(sk.SKError) as e:
        srv.result(long_job, 64, N)
    assert e.value.status == sk.SK_ERR_CANCELLED
    E, S, _ = srv.result(keep, 6, N)
    E0, S0 = _alone(J, N, 6, 16, 1.0, 3000, 2, 2)
    assert np.array_equal(S, S0) and np.array_equal(E, E0)
    o = oracle.run(J, K=16, beta=1.0, seed=2, stream=2, chains=6, steps=3000)
    assert np.array_equal(S, o["spins"])
    srv.close()
    # a queued job: a budget that holds one of the two jobs at a time
    srv = sk.Server(budget_bytes=sk_footprint_bytes(N, 512) + (1 << 20), quantum_steps=64)
    first = srv.submit(N=N, kind=sk.SK_J_PM1, chains=512, steps=20_000, K=8, seed=3, stream_id=3, J=J)
    queued = srv.submit(N=N, kind=sk.SK_J_PM1, chains=512, steps=100, K=8, seed=4, stream_id=4, J=J)
    assert srv.poll(queued)["state"] == sk.SK_JOB_QUEUED
    srv.cancel(queued)
    assert srv.poll(queued)["state"] == sk.SK_JOB_CANCELLED
    srv.wait_all(timeout_ns=120 * 10**9)
    assert srv.poll(first)["state"] == sk.SK_JOB_DONE
    with pytest.raises(sk.SKError) as e:
        srv.cancel(first)   # finished: nothing to cancel
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    E, S, _ = srv.result(first, 512, N)
    E0, S0 = _alone(J, N, 512, 8, 1.0, 20_000, 3, 3)
    assert np.array_equal(S, S0)
    srv.close()


def sk_footprint_bytes(N, chains):
    """Device bytes one +-J job of N spins and `chains` chains is charged: its
    couplings (and their tensor-core operand) and its chains' state, as the
    server's admission counts them (read back from a submitted job)."""
    srv = sk.Server(budget_bytes=1 << 40, quantum_steps=64)
    t = srv.submit(N=N, kind=sk.SK_J_PM1, chains=chains, steps=1, K=8, seed=0, J=np.zeros((N, N), np.int8))
    fp = srv.poll(t)["footprint_bytes"]
    srv.wait_all(timeout_ns=60 * 10**9)
    srv.close()
    return fp
