"""The team layout (mcmcmc_batch_set_layout with 64 or 128 lanes for star
runs): one chain per team of 2 or 4 warps, one proposal slot per thread.
+-J runs follow the oracle bit for bit (trace, records of E, q and
acceptance, spins, fields) for MCMCMC up to K = 32 x warps and for
Metropolis, with ragged N, odd chain counts (a CTA whose second team has no
chain), a non-uniform root and advances of ragged lengths; Gaussian runs are
decision-replayed against the oracle; the autotuner may pick the layout
without changing any result."""
import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _team_run(J, *, chains, K, rule, beta, lanes, steps, R, init, p_center=0.0, splits=None, trace=True):
    import torch
    st = torch.cuda.Stream()
    inst = sk.Instance(J, stream=st)
    run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=beta, seed=31, record_every=R,
                 max_records=steps // R if R else 0, init=init, p_center=p_center,
                 trace_chains=chains if trace else 0, trace_steps=steps if trace else 0)
    b = sk.Batch([run])
    b.set_layout(lanes, 0)
    cls = b.classes()
    for n in (splits or [steps]):
        b.advance(n)
    out = {"classes": cls, "trace": run.trace() if trace else None}
    if R:
        out["E"], out["q"], out["acc"] = run.observables()
    out["spins"], out["h"], out["step"] = run.state(fields=True)
    b.close(); run.close(); inst.close()
    return out


@pytest.mark.parametrize("N,K,chains,lanes,rule", [
    (64, 8, 1, 64, 0),      # config 1's shape on a 2-warp team
    (100, 1, 3, 64, 0),     # K = 1, ragged N, odd chains (a CTA with an idle team)
    (333, 33, 2, 64, 0),    # K not a multiple of 4, slots in both warps
    (200, 64, 5, 64, 0),    # K = 32 x 2: every thread a slot
    (512, 100, 4, 128, 0),  # 4-warp team, ragged last warp
    (130, 128, 3, 128, 0),  # K = 32 x 4
    (96, 5, 2, 128, 0),     # slots in one warp of four
    (256, 1, 3, 64, 1),     # Metropolis, 2 warps
    (1000, 1, 2, 128, 1),   # Metropolis, 4 warps
])
def test_team_pm1_bit_exact(N, K, chains, lanes, rule):
    need_gpu()
    steps, R = 900, 100
    J = inputs.couplings_pm1(N, 800 + K + N)
    init = inputs.initial_spins(chains, N, 801 + K)
    g = _team_run(J, chains=chains, K=K, rule=rule, beta=0.9, lanes=lanes, steps=steps, R=R, init=init,
                  splits=[1, 299, 600])
    code = 4096 + 2 * sk.SK_J_PM1 + rule
    assert len(g["classes"]) == 1 and g["classes"][0][0] == code and g["classes"][0][1] == lanes, g["classes"]
    o = oracle.run(J, rule=rule, K=K, beta=0.9, seed=31, chains=chains, init=init, steps=steps,
                   record_every=R, trace=True)
    assert g["step"] == steps
    assert np.array_equal(g["trace"], o["trace"])
    assert np.array_equal(g["E"], o["E"]) and np.array_equal(g["acc"], o["acc"])
    if chains > 1:
        assert np.array_equal(g["q"], o["q"])
    assert np.array_equal(g["spins"], o["spins"])
    assert np.array_equal(g["h"], (J.astype(np.int64) @ g["spins"].T.astype(np.int64)).T)


@pytest.mark.parametrize("K,lanes,p_center", [(16, 64, 0.5), (100, 128, 0.05)])
def test_team_pm1_nonuniform_root_bit_exact(K, lanes, p_center):
    need_gpu()
    N, chains, steps, R = 150, 2, 600, 100
    J = inputs.couplings_pm1(N, 850 + K)
    init = inputs.initial_spins(chains, N, 851)
    g = _team_run(J, chains=chains, K=K, rule=0, beta=1.2, lanes=lanes, steps=steps, R=R, init=init,
                  p_center=p_center)
    o = oracle.run(J, K=K, beta=1.2, seed=31, chains=chains, init=init, steps=steps, record_every=R,
                   trace=True, p_center=p_center)
    assert np.array_equal(g["trace"], o["trace"])
    assert np.array_equal(g["E"], o["E"]) and np.array_equal(g["acc"], o["acc"])
    assert np.array_equal(g["spins"], o["spins"])


@pytest.mark.parametrize("N,K,rule,lanes", [(512, 32, 0, 64), (257, 128, 0, 128), (300, 7, 0, 128),
                                            (512, 1, 1, 128)])
def test_team_gauss_decision_replay(N, K, rule, lanes):
    need_gpu()
    chains, steps = 3, 1500
    J = inputs.couplings_gauss(N, 870 + K)
    init = inputs.initial_spins(chains, N, 871)
    g = _team_run(J, chains=chains, K=K, rule=rule, beta=1.0, lanes=lanes, steps=steps, R=0, init=init,
                  splits=[500, 1000])
    for c in range(chains):
        r = oracle.replay(J, g["trace"][c], K=K, rule=rule, beta=1.0, seed=31, chain=c, init=init[c], tol=1e-4)
        assert r["bad"] == 0 and np.array_equal(r["spins"], g["spins"][c]), (c, r)


def test_team_layout_falls_back_where_it_cannot_apply():
    # K > 32 x warps and node-weighted records keep the warp layout
    need_gpu()
    J = inputs.couplings_pm1(128, 5)
    inst = sk.Instance(J)
    big = sk.Run(inst, chains=2, K=200, beta=1.0, seed=1)
    b = sk.Batch([big])
    b.set_layout(128, 0)
    assert b.classes()[0][0] < 1024, b.classes()
    b.close()
    nw = sk.Run(inst, chains=2, K=16, beta=1.0, seed=2, record_every=10, max_records=1, node_weighted=True)
    b = sk.Batch([nw])
    b.set_layout(64, 0)
    assert b.classes()[0][0] < 1024, b.classes()
    b.close(); big.close(); nw.close(); inst.close()


def test_team_in_a_batch_graph_with_recompute_and_autotune():
    # a team class beside a warp-layout class, replayed from a CUDA graph with
    # periodic recomputes (the team kernel keeps the spins' operands), equals
    # plain advances and the oracle; an autotuned batch gives the same results
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, steps = 256, 512
    J = inputs.couplings_pm1(N, 61)
    init = inputs.initial_spins(3, N, 62)
    outs = []
    for mode in ("advance", "graph", "tuned"):
        inst = sk.Instance(J, stream=st)
        a = sk.Run(inst, chains=3, K=24, beta=1.1, seed=5, init=init, recompute_every=128)
        w = sk.Run(inst, chains=2, K=200, beta=1.1, seed=6, stream_id=1, init=init[:2], recompute_every=128)
        b = sk.Batch([a, w])
        if mode == "tuned":
            b.autotune(trial_steps=64)
        else:
            b.set_layout(64, 0)
            codes = sorted(c[0] for c in b.classes())
            assert codes[-1] == 4096 and codes[0] < 1024, codes
        if mode == "graph":
            b.capture(128)
            b.replay(steps // 128)
        else:
            b.advance(steps)
        outs.append([r.state(fields=True) for r in (a, w)])
        for r in (a, w):
            assert r.recompute_stats()["mismatches"] == 0
        b.close(); a.close(); w.close(); inst.close()
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
    oa = oracle.run(J, K=24, beta=1.1, seed=5, chains=3, init=init, steps=steps)
    assert np.array_equal(outs[0][0][0], oa["spins"])
