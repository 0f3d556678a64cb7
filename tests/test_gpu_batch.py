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
