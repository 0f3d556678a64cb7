"""The cluster-per-chain layout (mcmcmc_batch_set_cluster): a chain's spins,
fields and columns of J spread over the CTAs of a thread-block cluster.
+-J runs follow the oracle bit for bit at every cluster size (trajectory,
trace, records, final spins and fields), Gaussian runs equal the whole-warp
layout bit for bit (the same arithmetic in every CTA, records included), the
autotuner may pick the layout without changing results, and the slice copy's
bounded wait expires cleanly."""
import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

# N, K, rule, chains, beta: +-J runs whose Npad = 256 splits into whole
# 16-byte rows of J at every cluster size up to 16; K = 130 takes two Philox
# blocks per lane, odd chain counts leave shadow warps, N = 230 pads.
PM1_SPECS = [(250, 8, 0, 3, 0.8), (250, 130, 0, 2, 1.1), (230, 13, 0, 5, 0.6),
             (250, 1, 1, 1, 1.0)]


def _pm1_runs(st, specs, steps, R, seed0=90):
    made = []
    for i, (N, K, rule, chains, beta) in enumerate(specs):
        J = inputs.couplings_pm1(N, seed0 + i)
        inst = sk.Instance(J, stream=st)
        init = inputs.initial_spins(chains, N, 40 + i)
        run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=beta, seed=5, stream_id=i,
                     record_every=R, max_records=steps // R, init=init, trace_chains=chains,
                     trace_steps=steps)
        made.append((J, init, inst, run))
    return made


def _close(b, made):
    b.close()
    for m in made:
        m[-1].close()
        m[-2].close()


@pytest.mark.parametrize("chains_per_cluster", [0, 4])
@pytest.mark.parametrize("ctas", [1, 2, 4, 8, 16])
def test_pm1_cluster_layout_follows_the_oracle(ctas, chains_per_cluster):
    torch = need_gpu()
    steps, R = 700, 100
    st = torch.cuda.Stream()
    made = _pm1_runs(st, PM1_SPECS, steps, R)
    b = sk.Batch([m[3] for m in made])
    b.set_cluster(ctas, chains_per_cluster)
    cls = b.classes()
    assert len(cls) == len(PM1_SPECS)
    assert all(c[0] >= 1024 and c[1] == 32 * ctas for c in cls), cls
    b.advance(300)
    b.advance(steps - 300)
    for i, ((N, K, rule, chains, beta), (J, init, inst, run)) in enumerate(zip(PM1_SPECS, made)):
        E, q, acc = run.observables()
        spins, h, step = run.state(fields=True)
        o = oracle.run(J, rule=rule, K=K, beta=beta, seed=5, stream=i, chains=chains, init=init,
                       steps=steps, record_every=R, trace=True)
        assert step == steps
        assert np.array_equal(run.trace(), o["trace"]), i
        assert np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"]), i
        if chains > 1:
            assert np.array_equal(q, o["q"]), i
        assert np.array_equal(spins, o["spins"]), i
        assert np.array_equal(h, (J.astype(np.int64) @ spins.T.astype(np.int64)).T), i
    _close(b, made)


def test_pm1_config1_one_chain_in_one_cta():
    # N = 64, K = 8, beta = 1, one chain: the whole of J (4 KB) in one CTA's
    # shared memory and in a 2- and 4-CTA cluster; 10^4 steps bit-exact
    torch = need_gpu()
    N, K, steps = 64, 8, 10_000
    J = inputs.couplings_pm1(N, 0)
    init = inputs.initial_spins(1, N, 1)
    o = oracle.run(J, K=K, beta=1.0, seed=1, chains=1, init=init, steps=steps, record_every=1000)
    st = torch.cuda.Stream()
    for ctas in (1, 2, 4):
        inst = sk.Instance(J, stream=st)
        run = sk.Run(inst, chains=1, K=K, beta=1.0, seed=1, init=init, record_every=1000,
                     max_records=steps // 1000)
        b = sk.Batch([run])
        b.set_cluster(ctas)
        assert b.classes()[0][3] == 1  # one chain per cluster
        b.advance(steps)
        E, _, acc = run.observables()
        spins, _ = run.state()
        assert np.array_equal(spins, o["spins"]) and np.array_equal(E, o["E"]), ctas
        assert np.array_equal(acc, o["acc"]), ctas
        b.close(); run.close(); inst.close()


def _gauss_runs(st, N, specs, steps, R):
    J = inputs.couplings_gauss(N, 7)
    made = []
    for i, (K, rule, chains, beta) in enumerate(specs):
        inst = sk.Instance(J, stream=st)
        init = inputs.initial_spins(chains, N, 60 + i)
        run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=beta, seed=11, stream_id=i,
                     record_every=R, max_records=steps // R, init=init, trace_chains=chains,
                     trace_steps=steps)
        made.append((J, init, inst, run))
    return made


@pytest.mark.parametrize("N,ctas", [(96, 1), (128, 2), (200, 4), (512, 8), (512, 16)])
def test_gauss_cluster_layout_equals_whole_warp_chains(N, ctas):
    # Gaussian couplings: every CTA computes the candidate energies, weights
    # and scan with the 32-lane arithmetic and updates its slice element by
    # element as the warp layout does, and rank 0 sums the energy records in
    # that layout's order, so trajectories, fields and records are equal bit
    # for bit (sizes whose columns of fp32 J fit a CTA at each cluster size)
    torch = need_gpu()
    steps, R = 600, 100
    specs = [(32, 0, 2, 1.0), (128, 0, 3, 2.0), (200, 0, 1, 0.5), (1, 1, 2, 1.0)]
    st = torch.cuda.Stream()
    res = []
    for mode in ("warp", "cluster"):
        made = _gauss_runs(st, N, specs, steps, R)
        b = sk.Batch([m[3] for m in made])
        if mode == "warp":
            b.set_layout(32, 2)
        else:
            b.set_cluster(ctas)
            assert all(c[0] >= 1024 for c in b.classes()), b.classes()
        b.advance(250)
        b.advance(steps - 250)
        res.append([(m[3].observables(), m[3].state(fields=True), m[3].trace()) for m in made])
        _close(b, made)
    for i, ((oa, sa, ta), (ob, sb, tb)) in enumerate(zip(*res)):
        assert np.array_equal(ta, tb), i
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1]), i
        for x, y in zip(oa, ob):  # energies, overlaps, accepted counts
            assert np.array_equal(x, y), i


def test_gauss_cluster_layout_decisions_replay_in_the_oracle():
    # one Gaussian chain at N = 512 in a 16-CTA cluster: the oracle replays its
    # trace (the same draws, each decision within the tolerance of the
    # weights' rounding) and the final spins agree
    torch = need_gpu()
    N, K, steps = 512, 64, 400
    J = inputs.couplings_gauss(N, 3)
    init = inputs.initial_spins(1, N, 4)
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=1, K=K, beta=2.0, seed=8, init=init, trace_chains=1, trace_steps=steps)
    b = sk.Batch([run])
    b.set_cluster(16)
    b.advance(steps)
    tr = run.trace()
    spins, _ = run.state()
    rep = oracle.replay(J, tr[0], K=K, beta=2.0, seed=8, chain=0, init=init[0], tol=1e-4)
    assert rep["bad"] == 0, rep
    assert np.array_equal(rep["spins"], spins[0])
    b.close(); run.close(); inst.close()


def test_shapes_the_cluster_layout_cannot_take_keep_the_warp_layout():
    torch = need_gpu()
    st = torch.cuda.Stream()
    # Npad = 96: 16 CTAs would hold 6 spins each, not a whole 16-byte row of int8 J
    inst = sk.Instance(inputs.couplings_pm1(90, 1), stream=st)
    run = sk.Run(inst, chains=2, K=8, seed=1)
    b = sk.Batch([run])
    b.set_cluster(16)
    assert b.classes()[0][0] < 1024
    b.set_cluster(2)
    assert b.classes()[0][0] >= 1024
    b.set_cluster(0)
    assert b.classes()[0][0] < 1024
    with pytest.raises(sk.SKError) as e:
        b.set_cluster(3)
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    b.close(); run.close(); inst.close()


def test_autotuner_may_choose_the_cluster_layout_without_changing_results():
    torch = need_gpu()
    steps = 400
    st = torch.cuda.Stream()
    spec = [(250, 64, 0, 1, 1.0)]
    a = _pm1_runs(st, spec, steps, 100)
    ba = sk.Batch([m[3] for m in a])
    ba.advance(steps)
    ref = (a[0][3].observables(), a[0][3].state(fields=True), a[0][3].trace())
    b = _pm1_runs(st, spec, steps, 100)
    bb = sk.Batch([m[3] for m in b])
    bb.autotune(trial_steps=50)
    bb.advance(steps)
    got = (b[0][3].observables(), b[0][3].state(fields=True), b[0][3].trace())
    for x, y in zip(ref[0], got[0]):
        assert np.array_equal(x, y)
    assert np.array_equal(ref[1][0], got[1][0]) and np.array_equal(ref[1][1], got[1][1])
    assert np.array_equal(ref[2], got[2])
    _close(ba, a)
    _close(bb, b)


def test_cluster_slice_wait_expires_and_returns():
    # a withheld row of the slice copy: the wait expires, the cluster skips
    # the item, the call reports SK_ERR_TIMEOUT; a clean run afterwards on the
    # same instance follows the oracle
    need_gpu()
    N = 256
    J = inputs.couplings_pm1(N, 31)
    init = inputs.initial_spins(2, N, 32)
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=2, K=8, seed=3, init=init, fault_inject=sk.SK_FAULT_WITHHOLD_ROW)
    b = sk.Batch([run])
    b.set_cluster(4)
    b.advance(20)
    with pytest.raises(sk.SKError) as e:
        run.wait()
    assert e.value.status == sk.SK_ERR_TIMEOUT
    b.close(); run.close()
    clean = sk.Run(inst, chains=2, K=8, beta=0.9, seed=3, init=init)
    b = sk.Batch([clean])
    b.set_cluster(4)
    b.advance(300)
    s, _ = clean.state()
    o = oracle.run(J, K=8, beta=0.9, seed=3, chains=2, init=init, steps=300)
    assert np.array_equal(s, o["spins"])
    b.close(); clean.close(); inst.close()
