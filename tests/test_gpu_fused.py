"""The fused launch (mcmcmc_batch_set_fused): every star run of a batch in one
persistent kernel, each work item dispatched to its run's variant.  +-J runs
of mixed N, K and rule follow the oracle bit for bit; every run, +-J and
Gaussian, equals the whole-warp per-class launches bit for bit (trajectory,
records, fields); graph runs and runs with node-weighted records keep their
own launches beside it."""
import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

# kind, N, K, rule, chains, beta: both coupling kinds, ragged N, K of one and
# two Philox blocks per lane, Metropolis with the unrolled (Npad = 1024) and
# the chunked (other Npad) field update, odd chain counts
SPECS = [(sk.SK_J_PM1, 100, 8, 0, 5, 0.8), (sk.SK_J_PM1, 333, 200, 0, 4, 1.5),
         (sk.SK_J_PM1, 1000, 1, 1, 3, 1.0), (sk.SK_J_PM1, 150, 1, 1, 2, 0.5),
         (sk.SK_J_GAUSS, 300, 64, 0, 3, 1.0), (sk.SK_J_GAUSS, 200, 130, 0, 2, 2.0),
         (sk.SK_J_GAUSS, 1024, 1, 1, 2, 1.0), (sk.SK_J_GAUSS, 96, 1, 1, 1, 0.7)]


def _runs(st, steps, R):
    made = []
    for i, (kind, N, K, rule, chains, beta) in enumerate(SPECS):
        J = inputs.couplings(N, kind, 300 + i)
        inst = sk.Instance(J, stream=st)
        init = inputs.initial_spins(chains, N, 400 + i)
        run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=beta, seed=13, stream_id=i,
                     record_every=R, max_records=steps // R, init=init, trace_chains=chains,
                     trace_steps=steps)
        made.append((J, init, inst, run))
    return made


def _results(made):
    return [(m[3].observables(), m[3].state(fields=True), m[3].trace()) for m in made]


def _close(b, made):
    b.close()
    for m in made:
        m[3].close()
        m[2].close()


@pytest.mark.parametrize("W", [2, 4, 16])
def test_fused_launch_equals_per_class_launches(W):
    torch = need_gpu()
    steps, R = 600, 100
    st = torch.cuda.Stream()
    res = []
    for mode in ("classes", "fused"):
        made = _runs(st, steps, R)
        b = sk.Batch([m[3] for m in made])
        if mode == "classes":
            b.set_layout(32, 2)
            assert len(b.classes()) > 1
        else:
            b.set_fused(W)
            cls = b.classes()
            assert len(cls) == 1 and cls[0][0] == 2048 and cls[0][3] == W, cls
        b.advance(250)
        b.advance(steps - 250)
        res.append(_results(made))
        if mode == "fused":  # +-J runs against the oracle
            for i, ((kind, N, K, rule, chains, beta), (J, init, _, run)) in enumerate(zip(SPECS, made)):
                if kind != sk.SK_J_PM1:
                    continue
                o = oracle.run(J, rule=rule, K=K, beta=beta, seed=13, stream=i, chains=chains, init=init,
                               steps=steps, record_every=R, trace=True)
                E, q, acc = run.observables()
                spins, h, step = run.state(fields=True)
                assert step == steps
                assert np.array_equal(run.trace(), o["trace"]), i
                assert np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"]), i
                if chains > 1:
                    assert np.array_equal(q, o["q"]), i
                assert np.array_equal(spins, o["spins"]), i
                assert np.array_equal(h, (J.astype(np.int64) @ spins.T.astype(np.int64)).T), i
        _close(b, made)
    for i, ((oa, sa, ta), (ob, sb, tb)) in enumerate(zip(*res)):
        assert np.array_equal(ta, tb), i
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1]) and sa[2] == sb[2], i
        for x, y in zip(oa, ob):
            assert np.array_equal(x, y), i


def test_fused_launch_beside_graph_and_node_weighted_runs():
    # a graph run and a run with node-weighted records keep their own launch
    # classes next to the fused one; the star runs stay bit-exact
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, steps, R = 128, 300, 100
    J = inputs.couplings_pm1(N, 31)
    init = inputs.initial_spins(4, N, 32)
    inst = sk.Instance(J, stream=st)
    star = sk.Run(inst, chains=4, K=16, beta=1.0, seed=2, init=init, record_every=R, max_records=steps // R)
    nw = sk.Run(inst, chains=2, K=8, beta=1.0, seed=3, init=init[:2], record_every=R,
                max_records=steps // R, node_weighted=True)
    tree = sk.Run(inst, chains=2, K=1, beta=1.0, seed=4, graph=sk.SK_GRAPH_TREE, arity=2, depth=2)
    b = sk.Batch([star, nw, tree])
    b.set_fused(4)
    cls = [c[0] for c in b.classes()]
    assert cls.count(2048) == 1 and len(cls) == 3, cls
    b.advance(steps)
    o = oracle.run(J, K=16, beta=1.0, seed=2, chains=4, init=init, steps=steps, record_every=R)
    spins, _ = star.state()
    E, q, acc = star.observables()
    assert np.array_equal(spins, o["spins"]) and np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"])
    o2 = oracle.run(J, K=8, beta=1.0, seed=3, chains=2, init=init[:2], steps=steps, record_every=R)
    s2, _ = nw.state()
    assert np.array_equal(s2, o2["spins"])
    b.set_fused(0)
    assert 2048 not in [c[0] for c in b.classes()]
    with pytest.raises(sk.SKError) as e:
        b.set_fused(3)
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    b.close()
    for r in (star, nw, tree):
        r.close()
    inst.close()


def test_fused_launch_in_a_captured_graph_with_recompute():
    # CUDA-graph replay of the fused launch with periodic recomputes (the
    # step kernel keeps the spins' operands): the same as plain advances
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, chains, steps = 256, 6, 512
    J = inputs.couplings_pm1(N, 41)
    init = inputs.initial_spins(chains, N, 42)
    out = []
    for mode in ("advance", "graph"):
        inst = sk.Instance(J, stream=st)
        run = sk.Run(inst, chains=chains, K=32, beta=1.2, seed=5, init=init, recompute_every=128)
        b = sk.Batch([run])
        b.set_fused(4)
        if mode == "advance":
            b.advance(steps)
        else:
            b.capture(128)
            b.replay(steps // 128)
        spins, h, step = run.state(fields=True)
        stt = run.recompute_stats()
        out.append((spins, h, step))
        assert stt["mismatches"] == 0 and stt["recomputes"] == steps // 128, stt
        b.close(); run.close(); inst.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    o = oracle.run(J, K=32, beta=1.2, seed=5, chains=chains, init=init, steps=steps)
    assert np.array_equal(out[0][0], o["spins"])


def test_fused_items_with_idle_warps_at_record_points():
    # large-N runs: an item holds fewer chains than the CTA has warps (the
    # launch's shared memory is sized for its items, not for W slices of the
    # largest run), so some warps only meet the record barriers and must not
    # touch slices they do not have; +-J bit-exact against the oracle
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, chains, steps, R = 4000, 6, 200, 50
    J = inputs.couplings_pm1(N, 51)
    init = inputs.initial_spins(chains, N, 52)
    inst = sk.Instance(J, stream=st)
    run = sk.Run(inst, chains=chains, K=16, beta=0.05, seed=9, init=init, record_every=R,
                 max_records=steps // R)
    small = sk.Run(inst, chains=2, K=8, beta=0.05, seed=10, init=init[:2], record_every=R,
                   max_records=steps // R)
    b = sk.Batch([run, small])
    b.set_fused(16)
    cls = b.classes()
    assert len(cls) == 1 and cls[0][4] >= 2, cls  # items of at most 10 chains of 16 warps
    b.advance(steps)
    o = oracle.run(J, K=16, beta=0.05, seed=9, chains=chains, init=init, steps=steps, record_every=R)
    E, q, acc = run.observables()
    spins, _ = run.state()
    assert np.array_equal(spins, o["spins"]) and np.array_equal(E, o["E"])
    assert np.array_equal(acc, o["acc"]) and np.array_equal(q, o["q"])
    b.close(); run.close(); small.close(); inst.close()


def test_fused_untraced_runs_bit_exact():
    # untraced uniform-root +-J runs (the loop compiled for that case; K <= 8
    # with two-lane scans and batched site draws) beside Gaussian ones in one
    # fused launch: +-J bit-exact against the oracle
    torch = need_gpu()
    st = torch.cuda.Stream()
    steps, R = 500, 100
    specs = [(sk.SK_J_PM1, 64, 8, 1), (sk.SK_J_PM1, 150, 3, 4), (sk.SK_J_PM1, 333, 1, 3),
             (sk.SK_J_PM1, 100, 24, 2), (sk.SK_J_GAUSS, 128, 8, 2)]
    made = []
    for i, (kind, N, K, chains) in enumerate(specs):
        J = inputs.couplings(N, kind, 900 + i)
        init = inputs.initial_spins(chains, N, 950 + i)
        inst = sk.Instance(J, stream=st)
        run = sk.Run(inst, chains=chains, K=K, beta=1.1, seed=8, stream_id=i, record_every=R,
                     max_records=steps // R, init=init)
        made.append((J, init, inst, run))
    b = sk.Batch([m[3] for m in made])
    b.set_fused(8)
    b.advance(123)
    b.advance(steps - 123)
    for i, ((kind, N, K, chains), (J, init, _, run)) in enumerate(zip(specs, made)):
        if kind != sk.SK_J_PM1:
            continue
        o = oracle.run(J, K=K, beta=1.1, seed=8, stream=i, chains=chains, init=init, steps=steps, record_every=R)
        E, q, acc = run.observables()
        spins, h, _ = run.state(fields=True)
        assert np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"]), i
        if chains > 1:
            assert np.array_equal(q, o["q"]), i
        assert np.array_equal(spins, o["spins"]), i
        assert np.array_equal(h, (J.astype(np.int64) @ spins.T.astype(np.int64)).T), i
    _close(b, made)


def test_autotuner_compares_fused_and_per_class_launches():
    # the autotuner may keep the fused launch or the per-class ones; either
    # way the runs' results equal a plain advance's (+-J: bit-exact)
    torch = need_gpu()
    st = torch.cuda.Stream()
    steps, R = 400, 100
    specs = [(100, 8, 0, 5), (333, 200, 0, 4), (1000, 1, 1, 3), (64, 32, 0, 2)]
    out = []
    for tune in (False, True):
        made = []
        for i, (N, K, rule, chains) in enumerate(specs):
            J = inputs.couplings_pm1(N, 500 + i)
            inst = sk.Instance(J, stream=st)
            run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=0.9, seed=6, stream_id=i, record_every=R,
                         max_records=steps // R)
            made.append((inst, run))
        b = sk.Batch([r for _, r in made])
        if tune:
            b.autotune(trial_steps=20)
        b.advance(steps)
        out.append([(r.observables(), r.state(fields=True)) for _, r in made])
        b.close()
        for inst, r in made:
            r.close()
            inst.close()
    for (oa, sa), (ob, sb) in zip(*out):
        for x, y in zip(oa, ob):
            assert np.array_equal(x, y)
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1]) and sa[2] == sb[2]
