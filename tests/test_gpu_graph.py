"""MCMCMC on deeper graphs (App. B) through the C ABI: full k-ary trees with a
uniformly drawn root position and the line with the addition process's
binomial root, against the oracle (sko_run_graph): bit-exact trajectories for
+-J couplings, decision replay for Gaussian couplings."""
import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

REPLAY_TOL = 1e-4
GRAPH_CASES = [  # graph, arity, depth, line_nodes, N, chains, beta
    (sk.SK_GRAPH_TREE, 2, 3, 0, 64, 6, 1.0),      # 15 nodes
    (sk.SK_GRAPH_TREE, 3, 2, 0, 100, 5, 0.7),     # 13 nodes, ragged N, odd chains
    (sk.SK_GRAPH_TREE, 2, 7, 0, 100, 4, 1.0),     # 255 nodes: the paper's binary tree
    (sk.SK_GRAPH_TREE, 16, 2, 0, 64, 4, 0.5),     # 273 nodes: several chunks per lane
    (sk.SK_GRAPH_LINE, 0, 0, 8, 64, 4, 1.0),
    (sk.SK_GRAPH_LINE, 0, 0, 37, 100, 5, 0.8),    # ragged line
    (sk.SK_GRAPH_LINE, 0, 0, 128, 64, 4, 1.0),    # the paper's 2^7 line
]


def _ograph(graph):
    return oracle.TREE if graph == sk.SK_GRAPH_TREE else oracle.LINE


def _run(J, graph, arity, depth, L, chains, beta, steps, R, init, seed, stream_id=0, trace=True):
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=chains, K=1, beta=beta, seed=seed, stream_id=stream_id, record_every=R,
                 max_records=steps // R, init=init, trace_chains=chains if trace else 0,
                 trace_steps=steps if trace else 0, graph=graph, arity=arity, depth=depth, line_nodes=L)
    run.advance(steps // 2)
    run.advance(steps - steps // 2)
    E, _, acc = run.observables()
    spins, h, step = run.state(fields=True)
    tr = run.trace() if trace else None
    run.close()
    inst.close()
    return dict(E=E, acc=acc, spins=spins, fields=h, step=step, trace=tr)


@pytest.mark.parametrize("case", range(len(GRAPH_CASES)))
def test_pm1_graph_bit_exact(case):
    need_gpu()
    graph, arity, depth, L, N, chains, beta = GRAPH_CASES[case]
    steps, R = 200, 50
    J = inputs.couplings_pm1(N, 60 + case)
    init = inputs.initial_spins(chains, N, 70 + case)
    g = _run(J, graph, arity, depth, L, chains, beta, steps, R, init, seed=9)
    o = oracle.run_graph(J, graph=_ograph(graph), arity=arity, depth=depth, line_nodes=L, beta=beta, seed=9,
                         chains=chains, init=init, steps=steps, record_every=R, trace=True)
    assert g["step"] == steps
    assert np.array_equal(g["trace"], o["trace"])
    assert np.array_equal(g["E"], o["E"])
    assert np.array_equal(g["acc"], o["acc"])
    assert np.array_equal(g["spins"], o["spins"])
    assert np.array_equal(g["fields"], (J.astype(np.int64) @ g["spins"].T.astype(np.int64)).T)


@pytest.mark.parametrize("graph,arity,depth,L", [(sk.SK_GRAPH_TREE, 3, 3, 0), (sk.SK_GRAPH_LINE, 0, 0, 64)])
def test_gauss_graph_decision_replay(graph, arity, depth, L):
    need_gpu()
    N, chains, steps, R, beta = 96, 4, 400, 100, 1.0
    J = inputs.couplings_gauss(N, 80)
    init = inputs.initial_spins(chains, N, 81)
    g = _run(J, graph, arity, depth, L, chains, beta, steps, R, init, seed=21)
    for c in range(chains):
        r = oracle.replay_graph(J, g["trace"][c], graph=_ograph(graph), arity=arity, depth=depth, line_nodes=L,
                                beta=beta, seed=21, chain=c, init=init[c], tol=REPLAY_TOL)
        assert r["bad"] == 0, (c, r)
        assert r["disagree"] <= 3, (c, r)
        assert np.array_equal(r["spins"], g["spins"][c])
        assert abs(g["E"][-1, c] - oracle.energy(J, g["spins"][c])) / N <= 1e-5


TEAM_CASES = [  # graph, arity, depth, line_nodes, N, chains, lanes per chain (32 x warps per chain)
    (sk.SK_GRAPH_TREE, 2, 7, 0, 100, 5, 64),      # 255 nodes, odd chains: a team without a chain
    (sk.SK_GRAPH_TREE, 16, 2, 0, 64, 4, 256),
    (sk.SK_GRAPH_TREE, 3, 5, 0, 96, 3, 512),      # 364 nodes, 16 warps per chain
    (sk.SK_GRAPH_LINE, 0, 0, 128, 64, 4, 128),
    (sk.SK_GRAPH_LINE, 0, 0, 37, 100, 3, 512),    # ragged line, fewer nodes than threads
]


def _run_layout(J, graph, arity, depth, L, chains, beta, steps, R, init, seed, lanes):
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=chains, K=1, beta=beta, seed=seed, record_every=R, max_records=steps // R,
                 init=init, trace_chains=chains, trace_steps=steps, graph=graph, arity=arity, depth=depth,
                 line_nodes=L)
    b = sk.Batch([run])
    b.set_layout(lanes=lanes)
    cls = b.classes()
    b.advance(steps // 2)
    b.advance(steps - steps // 2)
    E, _, acc = run.observables()
    spins, h, step = run.state(fields=True)
    tr = run.trace()
    b.close()
    run.close()
    inst.close()
    return dict(E=E, acc=acc, spins=spins, fields=h, step=step, trace=tr, classes=cls)


@pytest.mark.parametrize("case", range(len(TEAM_CASES)))
def test_pm1_graph_teams_bit_exact(case):
    """Several warps per chain (named-barrier teams) give the oracle's trajectory."""
    need_gpu()
    graph, arity, depth, L, N, chains, lanes = TEAM_CASES[case]
    steps, R, beta = 120, 40, 0.8
    J = inputs.couplings_pm1(N, 160 + case)
    init = inputs.initial_spins(chains, N, 170 + case)
    g = _run_layout(J, graph, arity, depth, L, chains, beta, steps, R, init, 13, lanes)
    assert g["classes"][0][1] == lanes
    o = oracle.run_graph(J, graph=_ograph(graph), arity=arity, depth=depth, line_nodes=L, beta=beta, seed=13,
                         chains=chains, init=init, steps=steps, record_every=R, trace=True)
    assert g["step"] == steps
    assert np.array_equal(g["trace"], o["trace"])
    assert np.array_equal(g["E"], o["E"])
    assert np.array_equal(g["acc"], o["acc"])
    assert np.array_equal(g["spins"], o["spins"])
    assert np.array_equal(g["fields"], (J.astype(np.int64) @ g["spins"].T.astype(np.int64)).T)


@pytest.mark.parametrize("graph,arity,depth,L,lanes", [(sk.SK_GRAPH_TREE, 2, 5, 0, 256),
                                                       (sk.SK_GRAPH_LINE, 0, 0, 48, 128)])
def test_gauss_graph_teams_decision_replay(graph, arity, depth, L, lanes):
    need_gpu()
    N, chains, steps, R, beta = 96, 4, 300, 100, 1.0
    J = inputs.couplings_gauss(N, 180)
    init = inputs.initial_spins(chains, N, 181)
    g = _run_layout(J, graph, arity, depth, L, chains, beta, steps, R, init, 23, lanes)
    for c in range(chains):
        r = oracle.replay_graph(J, g["trace"][c], graph=_ograph(graph), arity=arity, depth=depth, line_nodes=L,
                                beta=beta, seed=23, chain=c, init=init[c], tol=REPLAY_TOL)
        assert r["bad"] == 0, (c, r)
        assert r["disagree"] <= 3, (c, r)
        assert np.array_equal(r["spins"], g["spins"][c])
        assert abs(g["E"][-1, c] - oracle.energy(J, g["spins"][c])) / N <= 1e-5


def test_star_tree_and_line_share_a_batch():
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, chains, steps, R = 80, 6, 150, 50
    J = inputs.couplings_pm1(N, 90)
    init = inputs.initial_spins(chains, N, 91)
    specs = [dict(graph=0, K=12), dict(graph=sk.SK_GRAPH_TREE, arity=2, depth=4),
             dict(graph=sk.SK_GRAPH_LINE, line_nodes=20)]
    made = []
    for i, sp in enumerate(specs):
        inst = sk.Instance(J, stream=st)
        kw = dict(sp)
        K = kw.pop("K", 1)
        run = sk.Run(inst, chains=chains, K=K, beta=0.9, seed=3, stream_id=i, record_every=R,
                     max_records=steps // R, init=init, **kw)
        made.append((inst, run))
    b = sk.Batch([r for _, r in made])
    assert len(b.classes()) == 3
    b.autotune(trial_steps=20)
    b.advance(steps)
    for i, ((inst, run), sp) in enumerate(zip(made, specs)):
        E, _, acc = run.observables()
        spins, _ = run.state()
        if sp["graph"] == 0:
            o = oracle.run(J, K=12, beta=0.9, seed=3, stream=i, chains=chains, init=init, steps=steps,
                           record_every=R)
        else:
            o = oracle.run_graph(J, graph=_ograph(sp["graph"]), arity=sp.get("arity", 0), depth=sp.get("depth", 0),
                                 line_nodes=sp.get("line_nodes", 0), beta=0.9, seed=3, stream=i, chains=chains,
                                 init=init, steps=steps, record_every=R)
        assert np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"]), i
        assert np.array_equal(spins, o["spins"]), i
    b.close()
    for inst, run in made:
        run.close()
        inst.close()


def test_graph_arguments_checked():
    need_gpu()
    J = inputs.couplings_pm1(32, 1)
    inst = sk.Instance(J)
    for kw in (dict(graph=3), dict(graph=sk.SK_GRAPH_TREE, arity=1, depth=3),
               dict(graph=sk.SK_GRAPH_TREE, arity=2, depth=17), dict(graph=sk.SK_GRAPH_TREE, arity=16, depth=4),
               dict(graph=sk.SK_GRAPH_LINE, line_nodes=1), dict(graph=sk.SK_GRAPH_LINE, line_nodes=8, p_center=0.3),
               dict(graph=sk.SK_GRAPH_LINE, line_nodes=8, rule=sk.SK_RULE_METROPOLIS)):
        with pytest.raises(sk.SKError) as e:
            sk.Run(inst, chains=2, K=4, **kw)
        assert e.value.status == sk.SK_ERR_INVALID_ARG, kw
    inst.close()
