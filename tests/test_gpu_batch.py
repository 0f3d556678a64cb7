"""Batched launches: CUDA-graph replay and the autotuner leave every chain's
trajectory exactly as a plain advance would (the draws are counter-based, so
launch geometry and capture cannot change results)."""
import numpy as np
import pytest

from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

SPECS = [(64, sk.SK_J_PM1, 8, 1.0, sk.SK_RULE_MCMCMC, 6),
         (200, sk.SK_J_GAUSS, 40, 0.7, sk.SK_RULE_MCMCMC, 10),
         (333, sk.SK_J_PM1, 150, 2.0, sk.SK_RULE_MCMCMC, 5),
         (128, sk.SK_J_PM1, 1, 1.0, sk.SK_RULE_METROPOLIS, 4)]


def _make(stream, recompute_every=0, R=100, cap=20):
    made = []
    for i, (N, kind, K, beta, rule, chains) in enumerate(SPECS):
        inst = sk.Instance(inputs.couplings(N, kind, 70 + i), stream=stream)
        run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=beta, seed=9, stream_id=i,
                     record_every=R, max_records=cap, recompute_every=recompute_every)
        made.append((inst, run))
    return made


def _results(made):
    return [(r.observables(), r.state(fields=True)) for _, r in made]


def _same(a, b):
    for (oa, sa), (ob, sb) in zip(a, b):
        for x, y in zip(oa, ob):
            assert np.array_equal(x, y)
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1]) and sa[2] == sb[2]


def _close(made, batch):
    batch.close()
    for inst, run in made:
        run.close(); inst.close()


@pytest.mark.parametrize("recompute_every", [0, 100])
def test_graph_replay_equals_advance(recompute_every):
    torch = need_gpu()
    st = torch.cuda.Stream()
    a = _make(st, recompute_every)
    ba = sk.Batch([r for _, r in a])
    ba.advance(600)
    ra = _results(a)
    b = _make(st, recompute_every)
    bb = sk.Batch([r for _, r in b])
    bb.capture(200)
    bb.replay(3)
    rb = _results(b)
    _same(ra, rb)
    if recompute_every:
        for _, r in b:
            st_ = r.recompute_stats()
            assert st_["recomputes"] == 6
            if r.inst.kind == sk.SK_J_PM1:
                assert st_["mismatches"] == 0
    _close(a, ba)
    _close(b, bb)


def test_autotune_has_no_side_effects():
    torch = need_gpu()
    st = torch.cuda.Stream()
    a = _make(st)
    ba = sk.Batch([r for _, r in a])
    ba.advance(300)
    ra = _results(a)
    b = _make(st)
    bb = sk.Batch([r for _, r in b])
    bb.advance(150)
    w = bb.autotune(trial_steps=20)
    assert w in (32, 28, 24, 20, 16, 12, 8, 6, 4, 2)
    assert bb.info()["warps_per_cta"] == w
    bb.advance(150)
    rb = _results(b)
    _same(ra, rb)
    _close(a, ba)
    _close(b, bb)


def test_capture_rejects_default_stream_and_misaligned_recompute():
    torch = need_gpu()
    a = _make(None)
    ba = sk.Batch([r for _, r in a])
    with pytest.raises(sk.SKError):
        ba.capture(100)
    _close(a, ba)
    st = torch.cuda.Stream()
    b = _make(st, recompute_every=100)
    bb = sk.Batch([r for _, r in b])
    with pytest.raises(sk.SKError):
        bb.capture(150)
    _close(b, bb)


@pytest.mark.parametrize("staging", [1, 2])
@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_blocks_per_lane_do_not_change_results(lanes, staging):
    # several Philox blocks (4 proposals each) per lane: 2 or 4 blocks on 8
    # or 16 lanes, 2 on 32; ragged K and chain counts; +-J bit-exact and a
    # Gaussian run replayed by the oracle
    torch = need_gpu()
    import oracle
    specs = [(100, 40, 7, 0.8, "pm1"), (130, 100, 5, 1.1, "pm1"), (96, 128, 6, 0.5, "pm1"),
             (70, 200, 3, 1.0, "pm1"), (120, 128, 4, 1.0, "gauss")]  # N, K, chains, beta, J
    steps, R = 600, 100
    st = torch.cuda.Stream()
    made = []
    for i, (N, K, chains, beta, kind) in enumerate(specs):
        J = inputs.couplings_pm1(N, 70 + i) if kind == "pm1" else inputs.couplings_gauss(N, 70 + i)
        inst = sk.Instance(J, stream=st)
        init = inputs.initial_spins(chains, N, 20 + i)
        run = sk.Run(inst, chains=chains, K=K, beta=beta, seed=8, stream_id=i, record_every=R,
                     max_records=steps // R, init=init, trace_chains=chains, trace_steps=steps)
        made.append((J, init, inst, run))
    b = sk.Batch([m[3] for m in made])
    b.set_layout(lanes, staging)
    # K > 128 needs 16 lanes at least, K > 16 needs 8
    assert {c[1] for c in b.classes()} == {max(lanes, 16 if K > 128 else 8) for (_, K, _, _, _) in specs}
    b.advance(250)
    b.advance(steps - 250)
    for i, ((N, K, chains, beta, kind), (J, init, inst, run)) in enumerate(zip(specs, made)):
        spins, h, _ = run.state(fields=True)
        tr = run.trace()
        if kind == "pm1":
            E, q, acc = run.observables()
            o = oracle.run(J, K=K, beta=beta, seed=8, stream=i, chains=chains, init=init,
                           steps=steps, record_every=R, trace=True)
            assert np.array_equal(tr, o["trace"]), i
            assert np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"]), i
            assert np.array_equal(spins, o["spins"]), i
            assert np.array_equal(h, (J.astype(np.int64) @ spins.T.astype(np.int64)).T), i
        else:
            for c in range(chains):
                r = oracle.replay(J, tr[c], K=K, beta=beta, seed=8, stream=i, chain=c,
                                  init=init[c], tol=1e-4)
                assert r["bad"] == 0 and np.array_equal(r["spins"], spins[c]), (i, c, r)
    b.close()
    for _, _, inst, run in made:
        run.close()
        inst.close()


@pytest.mark.parametrize("staging", [1, 2])
@pytest.mark.parametrize("lanes", [4, 8, 16, 32])
def test_lanes_per_chain_do_not_change_results(lanes, staging):
    # sub-warp chains (32/lanes chains per warp), ragged chain counts (groups
    # without a chain run as shadows): bit-exact against the oracle
    torch = need_gpu()
    import oracle
    specs = [(100, 8, 0, 7, 0.8), (130, 13, 0, 13, 1.1), (90, 16, 0, 5, 0.5),
             (64, 1, 1, 9, 1.0)]   # N, K, rule, chains, beta
    steps, R = 800, 100
    st = torch.cuda.Stream()
    made = []
    for i, (N, K, rule, chains, beta) in enumerate(specs):
        J = inputs.couplings_pm1(N, 90 + i)
        inst = sk.Instance(J, stream=st)
        init = inputs.initial_spins(chains, N, 40 + i)
        run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=beta, seed=5, stream_id=i,
                     record_every=R, max_records=steps // R, init=init, trace_chains=chains,
                     trace_steps=steps)
        made.append((J, init, inst, run))
    b = sk.Batch([m[3] for m in made])
    b.set_layout(lanes, staging)
    assert all(c[1] == lanes for c in b.classes())
    b.advance(300)
    b.advance(steps - 300)
    for i, ((N, K, rule, chains, beta), (J, init, inst, run)) in enumerate(zip(specs, made)):
        E, q, acc = run.observables()
        spins, h, _ = run.state(fields=True)
        tr = run.trace()
        o = oracle.run(J, rule=rule, K=K, beta=beta, seed=5, stream=i, chains=chains, init=init,
                       steps=steps, record_every=R, trace=True)
        assert np.array_equal(tr, o["trace"]), i
        assert np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"]), i
        assert np.array_equal(q, o["q"]), i
        assert np.array_equal(spins, o["spins"]), i
        assert np.array_equal(h, (J.astype(np.int64) @ spins.T.astype(np.int64)).T), i
    b.close()
    for _, _, inst, run in made:
        run.close(); inst.close()


def test_node_weighted_runs_share_a_batch_with_plain_runs():
    # a run with node-weighted records gets its own launch class (rows through
    # L1); both kinds stay bit-exact, autotuned or not, and the node-weighted
    # records equal the oracle's
    torch = need_gpu()
    import oracle
    N, K, chains, steps, R = 120, 24, 6, 400, 100
    st = torch.cuda.Stream()
    J = inputs.couplings_pm1(N, 55)
    init = inputs.initial_spins(chains, N, 56)
    made = []
    for i, nw in enumerate((False, True)):
        inst = sk.Instance(J, stream=st)
        run = sk.Run(inst, chains=chains, K=K, beta=0.9, seed=4, stream_id=i, record_every=R,
                     max_records=steps // R, init=init, node_weighted=nw)
        made.append((inst, run))
    b = sk.Batch([r for _, r in made])
    assert len(b.classes()) == 2
    b.autotune(trial_steps=20)
    b.advance(steps)
    for i, (inst, run) in enumerate(made):
        E, q, acc = run.observables()
        spins, _ = run.state()
        o = oracle.run(J, K=K, beta=0.9, seed=4, stream=i, chains=chains, init=init, steps=steps,
                       record_every=R)
        assert np.array_equal(E, o["E"]) and np.array_equal(spins, o["spins"]), i
        if i == 1:
            nwE = run.observables_nw()
            assert np.abs(nwE - o["E_nw"]).max() <= 1e-9 * (1 + np.abs(o["E"]).max())
    b.close()
    for inst, run in made:
        run.close()
        inst.close()
