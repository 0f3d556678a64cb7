"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

+-J couplings: bit-exact trajectories (integer energies, same Philox
stream): records of E, acceptance and q, final spins, maintained fields and
the per-step slot log.  Gaussian couplings: every GPU decision is either the
oracle's or a near-tie within the fp32 tolerance (decision replay), and the
GPU's recorded energy per spin equals the oracle's FP64 energy of the same
state within 1e-5.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

# decision replay tolerance on u / P_K: fp32 fields drift by ~sqrt(f T) 2^-24 |h|
# after T steps of f flips (~1e-5 at T = 3000), which moves dE by ~4x that and a
# weight by beta x that (<= 1e-4 at beta = 2); the fp32 prefix sum adds (K+1) 2^-24
REPLAY_TOL = 1e-4
E_PER_SPIN_TOL = 1e-5


def _run_gpu(J, *, chains, K, beta, rule, steps, seed, R=0, init=None, trace=0, scale=1.0,
             stream_id=0, splits=None, p_center=0.0, node_weighted=False):
    inst = sk.Instance(J, scale=scale)
    nrec = steps // R if R else 0
    run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=beta, seed=seed, stream_id=stream_id,
                 record_every=R, max_records=nrec, init=init, trace_chains=trace,
                 trace_steps=steps if trace else 0, p_center=p_center,
                 node_weighted=node_weighted and R > 0)
    for s in (splits or [steps]):
        run.advance(s)
    run.wait()
    out = {}
    if nrec:
        out["E"], out["q"], out["acc"] = run.observables()
        if node_weighted:
            out["E_nw"] = run.observables_nw()
    out["spins"], out["fields"], out["step"] = run.state(fields=True)
    if trace:
        out["trace"] = run.trace()
    run.close()
    inst.close()
    return out


def _nw_close(g, o, tol=1e-9):
    """Node-weighted record energies: the same double-precision sums taken in
    another order (+-J weights are the same integers on both sides)."""
    assert np.abs(g["E_nw"] - o["E_nw"]).max() <= tol * (1.0 + np.abs(o["E"]).max())


def _fields_exact(J, spins):
    return (J.astype(np.int64) @ spins.T.astype(np.int64)).T


@pytest.mark.parametrize("rule,K", [(sk.SK_RULE_MCMCMC, 8)])
def test_pm1_config1_bit_exact(rule, K):
    """+-J N=64, J seed 0, beta=1, one chain from a random start, K=8, 1e5
    steps, Philox seed 1: identical trajectory step by step."""
    need_gpu()
    N, steps, R = 64, 100_000, 1000
    J = inputs.couplings_pm1(N, 0)
    init = inputs.initial_spins(1, N, 1234)
    g = _run_gpu(J, chains=1, K=K, beta=1.0, rule=rule, steps=steps, seed=1, R=R, init=init,
                 trace=1)
    o = oracle.run(J, rule=rule, K=K, beta=1.0, seed=1, chains=1, init=init, steps=steps,
                   record_every=R, trace=True, want_q=False)
    assert np.array_equal(g["trace"][0], o["trace"][0])
    assert np.array_equal(g["E"], o["E"])
    assert np.array_equal(g["acc"], o["acc"])
    assert np.array_equal(g["spins"], o["spins"])
    assert np.array_equal(g["fields"], _fields_exact(J, g["spins"]))
    assert g["step"] == steps


@pytest.mark.parametrize("N,K,chains,beta", [
    (100, 1, 7, 0.5),      # ragged N (padding), odd chains (ragged CTA), K = 1
    (100, 5, 6, 0.3),
    (130, 33, 5, 1.0),     # K not a multiple of 4
    (96, 128, 4, 2.0),     # 32 Philox blocks: every lane busy
    (70, 200, 4, 0.7),     # two blocks per lane (K > 128)
    (64, 256, 2, 1.5),     # maximum K
    (2, 3, 2, 1.0),        # smallest N
])
def test_pm1_bit_exact_shapes(N, K, chains, beta):
    need_gpu()
    steps, R = 1500, 100
    J = inputs.couplings_pm1(N, N + K)
    init = inputs.initial_spins(chains, N, 7)
    nw = K % 2 == 0  # runs with node-weighted records use their own kernels
    g = _run_gpu(J, chains=chains, K=K, beta=beta, rule=sk.SK_RULE_MCMCMC, steps=steps, seed=99,
                 R=R, init=init, trace=min(chains, 3), node_weighted=nw)
    o = oracle.run(J, K=K, beta=beta, seed=99, chains=chains, init=init, steps=steps,
                   record_every=R, trace=True)
    assert np.array_equal(g["trace"], o["trace"][: min(chains, 3)])
    assert np.array_equal(g["E"], o["E"])
    assert np.array_equal(g["acc"], o["acc"])
    if nw:
        _nw_close(g, o)
    if chains >= 2:
        assert np.array_equal(g["q"], o["q"])
    assert np.array_equal(g["spins"], o["spins"])
    assert np.array_equal(g["fields"], _fields_exact(J, g["spins"]))


@pytest.mark.parametrize("N,beta,scale", [(64, 1.0, 1.0), (150, 0.4, 1.0), (256, 1.0, 1 / 16)])
def test_pm1_metropolis_bit_exact(N, beta, scale):
    need_gpu()
    steps, R, chains = 4000, 200, 4
    J = inputs.couplings_pm1(N, 5)
    init = inputs.initial_spins(chains, N, 8)
    g = _run_gpu(J, chains=chains, K=1, beta=beta, rule=sk.SK_RULE_METROPOLIS, steps=steps,
                 seed=3, R=R, init=init, trace=2, scale=scale, node_weighted=True)
    o = oracle.run(J, rule=oracle.METROPOLIS, beta=beta, scale=scale, seed=3, chains=chains,
                   init=init, steps=steps, record_every=R, trace=True)
    assert np.array_equal(g["trace"], o["trace"][:2])
    assert np.array_equal(g["E"], o["E"])
    assert np.array_equal(g["acc"], o["acc"])
    assert np.array_equal(g["q"], o["q"])
    _nw_close(g, o)
    assert np.array_equal(g["spins"], o["spins"])


def test_pm1_scaled_energy_and_random_start():
    need_gpu()
    N, K, chains = 77, 16, 4
    J = inputs.couplings_pm1(N, 3)
    scale = 1.0 / math.sqrt(N)
    g = _run_gpu(J, chains=chains, K=K, beta=1.0, rule=sk.SK_RULE_MCMCMC, steps=0, seed=5,
                 stream_id=9, scale=scale)
    for c in range(chains):
        assert np.array_equal(g["spins"][c], oracle.init_spins(5, 9, c, N))
    g = _run_gpu(J, chains=chains, K=K, beta=1.0, rule=sk.SK_RULE_MCMCMC, steps=800, seed=5,
                 stream_id=9, scale=scale, R=100)
    o = oracle.run(J, K=K, beta=1.0, scale=scale, seed=5, stream=9, chains=chains, steps=800,
                   record_every=100)
    assert np.array_equal(g["E"], o["E"])
    assert np.array_equal(g["spins"], o["spins"])


def test_advance_in_pieces_equals_one_advance():
    # counter-based draws: stopping and resuming is bit-exact (checkpoint/resume)
    need_gpu()
    N, K, chains = 90, 24, 6
    J = inputs.couplings_pm1(N, 4)
    a = _run_gpu(J, chains=chains, K=K, beta=0.8, rule=sk.SK_RULE_MCMCMC, steps=1000, seed=2, R=50)
    b = _run_gpu(J, chains=chains, K=K, beta=0.8, rule=sk.SK_RULE_MCMCMC, steps=1000, seed=2, R=50,
                 splits=[1, 37, 462, 500])
    for k in ("E", "q", "acc", "spins", "fields"):
        assert np.array_equal(a[k], b[k]), k
    # restart from the saved spins: fields are recomputed, trajectory continues
    J2 = J
    c = _run_gpu(J2, chains=chains, K=K, beta=0.8, rule=sk.SK_RULE_MCMCMC, steps=400, seed=2, R=50)
    o = oracle.run(J2, K=K, beta=0.8, seed=2, chains=chains, steps=400, record_every=50)
    assert np.array_equal(c["spins"], o["spins"])


@pytest.mark.parametrize("rule,K,N,beta", [
    (sk.SK_RULE_MCMCMC, 32, 96, 1.0),
    (sk.SK_RULE_MCMCMC, 128, 160, 2.0),
    (sk.SK_RULE_MCMCMC, 200, 64, 0.5),
    (sk.SK_RULE_METROPOLIS, 1, 128, 1.0),
])
def test_gauss_decision_replay(rule, K, N, beta):
    need_gpu()
    steps, chains, R = 3000, 4, 300
    J = inputs.couplings_gauss(N, 17)
    init = inputs.initial_spins(chains, N, 18)
    g = _run_gpu(J, chains=chains, K=K, beta=beta, rule=rule, steps=steps, seed=21, R=R,
                 init=init, trace=chains)
    orule = oracle.MCMCMC if rule == sk.SK_RULE_MCMCMC else oracle.METROPOLIS
    for c in range(chains):
        r = oracle.replay(J, g["trace"][c], rule=orule, K=K, beta=beta, seed=21, chain=c,
                          init=init[c], tol=REPLAY_TOL)
        assert r["bad"] == 0, (c, r)
        assert r["disagree"] <= 3, (c, r)
        assert np.array_equal(r["spins"], g["spins"][c])
        # the GPU's recorded energy of its final state vs the FP64 energy
        assert abs(g["E"][-1, c] - oracle.energy(J, g["spins"][c])) / N <= E_PER_SPIN_TOL
        h = J.astype(np.float64) @ g["spins"][c].astype(np.float64)
        assert np.abs(g["fields"][c] - h).max() < 1e-4


@pytest.mark.parametrize("rule,K", [(sk.SK_RULE_MCMCMC, 32), (sk.SK_RULE_MCMCMC, 128), (sk.SK_RULE_METROPOLIS, 1)])
def test_gauss_node_weighted_records(rule, K):
    """Gaussian couplings: where the GPU and the oracle take the same path (the
    traces agree), the node-weighted record energies agree within the energy
    tolerance (fp32 weights and fields against fp64)."""
    need_gpu()
    N, chains, steps, R = 96, 4, 600, 100
    J = inputs.couplings_gauss(N, 41)
    init = inputs.initial_spins(chains, N, 42)
    g = _run_gpu(J, chains=chains, K=K, beta=1.0, rule=rule, steps=steps, seed=7, R=R, init=init,
                 trace=chains, node_weighted=True)
    orule = oracle.MCMCMC if rule == sk.SK_RULE_MCMCMC else oracle.METROPOLIS
    o = oracle.run(J, rule=orule, K=K, beta=1.0, seed=7, chains=chains, init=init, steps=steps,
                   record_every=R, trace=True)
    same = [c for c in range(chains) if np.array_equal(g["trace"][c], o["trace"][c])]
    assert len(same) >= 2, same
    for c in same:
        assert np.abs(g["E_nw"][:, c] - o["E_nw"][:, c]).max() / N <= E_PER_SPIN_TOL
        assert np.abs(g["E"][:, c] - o["E"][:, c]).max() / N <= E_PER_SPIN_TOL


def test_gauss_statistics_within_3_sigma():
    # independent GPU and oracle ensembles: E/N, q and acceptance per record
    need_gpu()
    N, K, beta, chains, steps, R = 48, 16, 1.0, 512, 1000, 100
    J = inputs.couplings_gauss(N, 31)
    g = _run_gpu(J, chains=chains, K=K, beta=beta, rule=sk.SK_RULE_MCMCMC, steps=steps,
                 seed=100, R=R)
    o = oracle.run(J, K=K, beta=beta, seed=200, chains=chains, steps=steps, record_every=R)
    zs = []
    for key in ("E", "q", "acc"):
        a = np.asarray(g[key], dtype=float)
        b = np.asarray(o[key], dtype=float)
        if key == "q":
            a, b = np.abs(a), np.abs(b)
        se = np.sqrt(a.var(axis=1, ddof=1) / a.shape[1] + b.var(axis=1, ddof=1) / b.shape[1])
        z = (a.mean(axis=1) - b.mean(axis=1)) / np.maximum(se, 1e-12)
        zs.append(z)
    zs = np.concatenate(zs)
    assert np.mean(np.abs(zs) > 3) <= 0.1 and np.abs(zs).max() < 4.5, zs


@pytest.mark.parametrize("N,K,chains,beta,p_center", [
    (64, 8, 4, 1.0, 0.3),      # centre favoured over each leaf
    (100, 33, 5, 0.5, 0.01),   # leaves favoured, ragged N and K
    (96, 128, 2, 2.0, 0.5),    # every lane busy
    (70, 200, 2, 0.7, 0.2),    # two Philox blocks per lane
])
def test_pm1_nonuniform_root_bit_exact(N, K, chains, beta, p_center):
    """Non-uniform root of the star (App. B.2): root threshold and integer
    slot factors give the oracle's trajectory exactly."""
    need_gpu()
    steps, R = 1500, 100
    J = inputs.couplings_pm1(N, 3 * N + K)
    init = inputs.initial_spins(chains, N, 9)
    g = _run_gpu(J, chains=chains, K=K, beta=beta, rule=sk.SK_RULE_MCMCMC, steps=steps, seed=41,
                 R=R, init=init, trace=chains, p_center=p_center)
    o = oracle.run(J, K=K, beta=beta, seed=41, chains=chains, init=init, steps=steps,
                   record_every=R, trace=True, p_center=p_center)
    assert np.array_equal(g["trace"], o["trace"])
    assert np.array_equal(g["E"], o["E"])
    assert np.array_equal(g["acc"], o["acc"])
    assert np.array_equal(g["spins"], o["spins"])
    assert np.array_equal(g["fields"], _fields_exact(J, g["spins"]))


@pytest.mark.parametrize("K,N,beta,p_center", [(16, 96, 1.0, 0.7), (128, 128, 1.5, 0.05)])
def test_gauss_nonuniform_root_decision_replay(K, N, beta, p_center):
    need_gpu()
    steps, chains, R = 3000, 4, 300
    J = inputs.couplings_gauss(N, 19)
    init = inputs.initial_spins(chains, N, 20)
    g = _run_gpu(J, chains=chains, K=K, beta=beta, rule=sk.SK_RULE_MCMCMC, steps=steps, seed=23,
                 R=R, init=init, trace=chains, p_center=p_center)
    for c in range(chains):
        r = oracle.replay(J, g["trace"][c], K=K, beta=beta, seed=23, chain=c, init=init[c],
                          tol=REPLAY_TOL, p_center=p_center)
        assert r["bad"] == 0, (c, r)
        assert r["disagree"] <= 3, (c, r)
        assert np.array_equal(r["spins"], g["spins"][c])


def test_uniform_p_center_equals_uniform_root_and_limits():
    need_gpu()
    N, K, chains, steps = 80, 12, 4, 2000
    J = inputs.couplings_pm1(N, 4)
    init = inputs.initial_spins(chains, N, 5)
    a = _run_gpu(J, chains=chains, K=K, beta=0.6, rule=sk.SK_RULE_MCMCMC, steps=steps, seed=6,
                 init=init, trace=chains)
    b = _run_gpu(J, chains=chains, K=K, beta=0.6, rule=sk.SK_RULE_MCMCMC, steps=steps, seed=6,
                 init=init, trace=chains, p_center=1.0 / (K + 1))
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["spins"], b["spins"])
    inst = sk.Instance(J)
    for bad in (1.0, -0.2, 1e-9, float("nan")):
        with pytest.raises(sk.SKError) as e:
            sk.Run(inst, chains=2, K=K, p_center=bad)
        assert e.value.status == sk.SK_ERR_INVALID_ARG
    inst.close()


@pytest.mark.parametrize("N,count", [(200, 9), (1000, 20), (1500, 3)])
def test_energy_entry_point(N, count):
    # one CTA per block of 8 configurations (ragged last block); above 256
    # spins the columns of J are split over several CTAs and summed after
    need_gpu()
    for J in (inputs.couplings_pm1(N, 1), inputs.couplings_gauss(N, 2)):
        S = inputs.initial_spins(count, N, 3)
        inst = sk.Instance(J, scale=0.5)
        E = inst.energy(S)
        inst.close()
        for c in range(count):
            want = oracle.energy(J, S[c], scale=0.5)
            if J.dtype == np.int8:
                assert E[c] == want
            else:
                assert abs(E[c] - want) <= 1e-9 * N


def test_batch_equals_runs_alone():
    # uneven N, K, beta, couplings and rules in one launch; each run identical alone
    need_gpu()
    specs = [(64, sk.SK_J_PM1, 8, 1.0, sk.SK_RULE_MCMCMC, 6),
             (200, sk.SK_J_GAUSS, 40, 0.7, sk.SK_RULE_MCMCMC, 10),
             (333, sk.SK_J_PM1, 150, 2.0, sk.SK_RULE_MCMCMC, 5),
             (128, sk.SK_J_GAUSS, 1, 1.0, sk.SK_RULE_METROPOLIS, 4),
             (96, sk.SK_J_PM1, 1, 0.5, sk.SK_RULE_METROPOLIS, 3)]
    steps, R = 600, 100

    def make(i, spec):
        N, kind, K, beta, rule, chains = spec
        J = inputs.couplings(N, kind, 50 + i)
        inst = sk.Instance(J)
        run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=beta, seed=7, stream_id=i,
                     record_every=R, max_records=steps // R)
        return inst, run

    alone = []
    for i, spec in enumerate(specs):
        inst, run = make(i, spec)
        run.advance(steps)
        alone.append((run.observables(), run.state(fields=True)))
        run.close(); inst.close()
    made = [make(i, spec) for i, spec in enumerate(specs)]
    b = sk.Batch([r for _, r in made])
    b.advance(250)
    b.advance(steps - 250)
    for (inst, run), (obs, st) in zip(made, alone):
        o2 = run.observables()
        s2 = run.state(fields=True)
        for x, y in zip(obs, o2):
            assert np.array_equal(x, y)
        assert np.array_equal(st[0], s2[0]) and np.array_equal(st[1], s2[1]) and st[2] == s2[2]
    b.close()
    for inst, run in made:
        run.close(); inst.close()


def test_invalid_arguments_fail_loudly():
    need_gpu()
    J = inputs.couplings_pm1(16, 1)
    with pytest.raises(sk.SKError) as e:
        bad = J.copy(); bad[0, 1] = 2; bad[1, 0] = 2
        sk.Instance(bad)
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    with pytest.raises(sk.SKError):
        bad = J.copy(); bad[0, 1] = -bad[0, 1]
        sk.Instance(bad)
    inst = sk.Instance(J)
    with pytest.raises(sk.SKError):
        sk.Run(inst, chains=2, K=0)
    with pytest.raises(sk.SKError):
        sk.Run(inst, chains=2, K=257)
    with pytest.raises(sk.SKError):
        sk.Run(inst, chains=0, K=4)
    with pytest.raises(sk.SKError):
        sk.Run(inst, chains=2, K=4, beta=-1.0)
    with pytest.raises(sk.SKError):
        sk.Run(inst, chains=2, K=4, init=np.zeros((2, 16), dtype=np.int8))
    plain = sk.Run(inst, chains=2, K=4, record_every=10, max_records=2)
    with pytest.raises(sk.SKError):
        plain.observables_nw()  # created without node-weighted records
    plain.close()
    inst.close()
    with pytest.raises(sk.SKError):
        sk.Instance(np.zeros((8193, 8193), dtype=np.int8))


@pytest.mark.parametrize("N,chains", [(700, 100), (64, 65), (2048, 130)])
def test_start_fields(N, chains):
    """Fields of the start state (register-tiled h = J s over ragged site and
    chain tiles): +-J exact, Gaussian within the blocked-summation bound of
    fp32, (32 + N/32) 2^-24 sum_j |J_ij|."""
    need_gpu()
    init = inputs.initial_spins(chains, N, 3)
    for J in (inputs.couplings_pm1(N, 5), inputs.couplings_gauss(N, 6)):
        inst = sk.Instance(J)
        for start in (init, None):
            run = sk.Run(inst, chains=chains, K=8, init=start, seed=12)
            spins, h, _ = run.state(fields=True)
            if start is not None:
                assert np.array_equal(spins, init)
            else:
                for c in (0, chains - 1):
                    assert np.array_equal(spins[c], oracle.init_spins(12, 0, c, N))
            exact = J.astype(np.float64) @ spins.T.astype(np.float64)
            if J.dtype == np.int8:
                assert np.array_equal(h, exact.T.astype(np.int64))
            else:
                bound = (32 + N / 32) * 2.0 ** -24 * np.abs(J).astype(np.float64).sum(axis=1)
                assert (np.abs(h - exact.T) <= bound[None, :]).all()
            run.close()
        inst.close()


def test_rejected_inputs_change_nothing():
    """Couplings or start spins that fail the device checks leave the instance
    and the run as they were: the chain continues bit-exactly."""
    need_gpu()
    N, K, chains = 48, 8, 4
    J = inputs.couplings_pm1(N, 31)
    init = inputs.initial_spins(chains, N, 32)
    inst = sk.Instance(J)
    run = sk.Run(inst, chains=chains, K=K, beta=0.7, seed=3, init=init, trace_chains=chains,
                 trace_steps=400)
    run.advance(200)
    cases = []
    b = J.copy(); b[3, 3] = 1; cases.append((b, "diagonal"))
    b = J.copy(); b[5, 9] = 2; b[9, 5] = 2; cases.append((b, "not in"))
    b = J.copy(); b[7, 2] = -b[7, 2]; cases.append((b, "symmetric at (2,7)"))
    for bad, what in cases:
        with pytest.raises(sk.SKError) as e:
            inst.set_couplings(bad)
        assert e.value.status == sk.SK_ERR_INVALID_ARG and what in str(e.value), (what, str(e.value))
    badS = init.copy(); badS[2, 17] = 0
    with pytest.raises(sk.SKError) as e:
        run.reset(badS)
    assert e.value.status == sk.SK_ERR_INVALID_ARG and str(2 * N + 17) in str(e.value)
    # device spins at an address 3 bytes past a 16-byte boundary: the bytes
    # before the first boundary, the 16-byte words and the ragged end are
    # checked, and the first bad spin is the one reported
    import torch
    buf = torch.empty(chains * N + 8, dtype=torch.int8, device="cuda")
    dev = buf[3:3 + chains * N]
    for bad_at in ((190,), (5, 100), (100, 150), (12, 13), (176, 189)):
        flat = init.reshape(-1).copy()
        for x in bad_at:
            flat[x] = 3
        dev.copy_(torch.from_numpy(flat))
        with pytest.raises(sk.SKError) as e:
            run.reset(dev.view(chains, N))
        assert e.value.status == sk.SK_ERR_INVALID_ARG and f"spin {min(bad_at)} " in str(e.value), str(e.value)
        with pytest.raises(sk.SKError) as e:
            sk.reset_many([run], [dev.view(chains, N)])
        assert e.value.status == sk.SK_ERR_INVALID_ARG and f"spin {min(bad_at)} " in str(e.value), str(e.value)
    torch.cuda.synchronize()
    run.advance(200)
    tr = run.trace()
    spins, h, step = run.state(fields=True)
    o = oracle.run(J, K=K, beta=0.7, seed=3, chains=chains, init=init, steps=400, trace=True)
    assert step == 400
    assert np.array_equal(tr, o["trace"]) and np.array_equal(spins, o["spins"])
    assert np.array_equal(h, (J.astype(np.int64) @ spins.T.astype(np.int64)).T)
    Jg = inputs.couplings_gauss(N, 33)
    ig = sk.Instance(Jg)
    b = Jg.copy(); b[4, 6] = np.nan; b[6, 4] = np.nan
    with pytest.raises(sk.SKError) as e:
        ig.set_couplings(b)
    assert "not finite" in str(e.value)
    ig.set_couplings(Jg * 0.5)  # a valid replacement is taken
    run.close(); inst.close(); ig.close()


def test_inputs_while_compute_is_queued():
    """New couplings and start spins given twice in a row while a long advance
    is still queued: the second copy of each must wait until the first has
    been consumed (its staging buffer is still to be read), and the run then
    follows the last couplings and spins bit-exactly."""
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, K, chains, steps = 192, 32, 8, 300
    J0, J1, J2 = (inputs.couplings_pm1(N, 400 + i) for i in range(3))
    init1, init2 = inputs.initial_spins(chains, N, 410), inputs.initial_spins(chains, N, 411)
    inst = sk.Instance(J0, stream=st)
    big = sk.Run(inst, chains=4096, K=128, beta=1.0, seed=2)  # keeps the stream busy
    run = sk.Run(inst, chains=chains, K=K, beta=0.9, seed=6, trace_chains=chains, trace_steps=steps)
    big.advance(400)
    inst.set_couplings(J1)
    inst.set_couplings(J2)
    run.reset(init1)
    run.reset(init2)
    run.advance(steps)
    tr = run.trace()
    spins, h, step = run.state(fields=True)
    o = oracle.run(J2, K=K, beta=0.9, seed=6, chains=chains, init=init2, steps=steps, trace=True)
    assert step == steps
    assert np.array_equal(tr, o["trace"]) and np.array_equal(spins, o["spins"])
    assert np.array_equal(h, (J2.astype(np.int64) @ spins.T.astype(np.int64)).T)
    big.close(); run.close(); inst.close()


@pytest.mark.parametrize("rule,K,lanes,warps", [(sk.SK_RULE_MCMCMC, 8, 32, 8), (sk.SK_RULE_MCMCMC, 128, 32, 8),
                                                 (sk.SK_RULE_MCMCMC, 128, 16, 8), (sk.SK_RULE_MCMCMC, 200, 16, 8),
                                                 (sk.SK_RULE_MCMCMC, 40, 8, 8), (sk.SK_RULE_METROPOLIS, 1, 32, 8),
                                                 (sk.SK_RULE_MCMCMC, 8, 32, 32), (sk.SK_RULE_MCMCMC, 30, 16, 24)])
def test_few_warps_variant_bit_exact(rule, K, lanes, warps):
    """The 128-register step kernel (at most 16 warps per CTA: the update's
    row loads eight iterations deep, and for MCMCMC with rows through L1 the
    next step's draws and J_ab gathered during the update) follows the
    oracle bit-exactly, ragged N and chain counts included."""
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, chains, steps, R = 333, 7, 300, 100
    J = inputs.couplings_pm1(N, 500 + K)
    init = inputs.initial_spins(chains, N, 501 + K)
    inst = sk.Instance(J, stream=st)
    run = sk.Run(inst, chains=chains, K=K, rule=rule, beta=0.8, seed=17, record_every=R,
                 max_records=steps // R, init=init, trace_chains=chains, trace_steps=steps)
    b = sk.Batch([run], warps_per_cta=warps)
    b.set_layout(lanes, 2)
    assert b.info()["warps_per_cta"] <= max(16, warps)
    b.advance(steps // 3)
    b.advance(steps - steps // 3)
    tr = run.trace()
    E, _, acc = run.observables()
    spins, h, step = run.state(fields=True)
    o = oracle.run(J, K=K, rule=rule, beta=0.8, seed=17, chains=chains, init=init, steps=steps,
                   record_every=R, trace=True)
    assert step == steps
    assert np.array_equal(tr, o["trace"]) and np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"])
    assert np.array_equal(spins, o["spins"])
    assert np.array_equal(h, (J.astype(np.int64) @ spins.T.astype(np.int64)).T)
    b.close(); run.close(); inst.close()


@pytest.mark.parametrize("K,lanes,chains,warps", [
    (8, 32, 1, 8), (8, 32, 7, 8), (5, 16, 5, 8), (4, 8, 6, 8), (1, 4, 9, 8), (3, 32, 2, 8), (9, 32, 3, 8),
    (32, 16, 4, 8), (17, 16, 2, 8), (24, 32, 3, 8), (33, 32, 3, 8), (40, 8, 5, 8),
    # the throughput variants (20, 24, 32 warps: 96, 80, 64 registers) with 16-lane and whole-warp chains
    (8, 32, 40, 32), (32, 32, 21, 24), (5, 16, 50, 20), (32, 16, 33, 32), (2, 16, 19, 24)])
def test_untraced_uniform_root_loop_bit_exact(K, lanes, chains, warps):
    """+-J items whose chains have the uniform root, no traced steps and a
    weight table short enough for shared memory run the step loop compiled
    for that case; for K <= 8 (K <= 32) in the 128-register variant it scans
    the slot weights of 2 (8) lanes only and draws the sites of lanes/2
    (lanes/8) steps at once.
    Energies, acceptances, overlaps, spins and fields follow the oracle bit
    for bit over advances of ragged lengths (site batches cut at any step)."""
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, steps, R = 200, 333, 111
    J = inputs.couplings_pm1(N, 700 + K)
    init = inputs.initial_spins(chains, N, 701 + K)
    inst = sk.Instance(J, stream=st)
    run = sk.Run(inst, chains=chains, K=K, beta=0.9, seed=23, record_every=R, max_records=steps // R, init=init)
    b = sk.Batch([run], warps_per_cta=warps)
    b.set_layout(lanes, 2)
    for n in (37, 100, steps - 137):
        b.advance(n)
    E, q, acc = run.observables()
    spins, h, step = run.state(fields=True)
    o = oracle.run(J, K=K, beta=0.9, seed=23, chains=chains, init=init, steps=steps, record_every=R)
    assert step == steps
    assert np.array_equal(E, o["E"]) and np.array_equal(acc, o["acc"])
    if chains > 1:
        assert np.array_equal(q, o["q"])
    assert np.array_equal(spins, o["spins"])
    assert np.array_equal(h, (J.astype(np.int64) @ spins.T.astype(np.int64)).T)
    b.close(); run.close(); inst.close()


@pytest.mark.parametrize("K,lanes,warps", [(96, 32, 16), (8, 32, 16), (32, 32, 16), (20, 16, 16), (5, 4, 16),
                                          (8, 32, 32), (32, 32, 24), (20, 16, 32), (32, 16, 20)])
def test_few_warps_variant_gaussian_replay(K, lanes, warps):
    # the same variant on Gaussian couplings (K <= 32: sites drawn in
    # batches of steps): every chain's recorded trajectory is one the
    # oracle's node rule takes from the same draws
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, chains, steps = 257, 5, 400
    J = inputs.couplings_gauss(N, 610)
    init = inputs.initial_spins(chains, N, 611)
    inst = sk.Instance(J, stream=st)
    run = sk.Run(inst, chains=chains, K=K, beta=1.0, seed=23, init=init, trace_chains=chains,
                 trace_steps=steps)
    b = sk.Batch([run], warps_per_cta=warps)
    b.set_layout(lanes, 2)
    b.advance(150)
    b.advance(steps - 150)
    tr = run.trace()
    spins, _ = run.state()
    for c in range(chains):
        r = oracle.replay(J, tr[c], K=K, beta=1.0, seed=23, chain=c, init=init[c], tol=1e-4)
        assert r["bad"] == 0 and np.array_equal(r["spins"], spins[c]), (c, r)
    b.close(); run.close(); inst.close()


def test_large_n_many_chains_small_k_gets_a_layout():
    # a large-N run forced to 4 lanes per chain with TMA-staged rows: 8
    # chains per warp do not fit in one CTA's shared memory, so the plan
    # gives each chain more lanes; +-J bit-exact against the oracle, and a
    # Gaussian run's fields equal to J s of its final spins
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, chains, K, steps = 4500, 600, 8, 20
    J = inputs.couplings_pm1(N, 620)
    init = inputs.initial_spins(chains, N, 621)
    inst = sk.Instance(J, stream=st)
    run = sk.Run(inst, chains=chains, K=K, beta=1.0, seed=3, init=init)
    b = sk.Batch([run])
    b.set_layout(4, 1)
    assert b.classes()[0][1] > 4
    b.advance(steps)
    b.close()
    spins, h, step = run.state(fields=True)
    assert step == steps
    for c0 in (0, chains - 3):  # chains are independent: the oracle runs a few of them
        o = oracle.run(J, K=K, beta=1.0, seed=3, chain0=c0, chains=3, init=init[c0:c0 + 3], steps=steps,
                       want_q=False)
        assert np.array_equal(spins[c0:c0 + 3], o["spins"]), c0
    sub = np.r_[0:8, chains - 8:chains]
    exact = (J.astype(np.float64) @ spins[sub].T.astype(np.float64)).T  # integers: exact in fp64
    assert np.array_equal(h[sub], exact.astype(np.int32))
    run.close(); inst.close()
    Jg = inputs.couplings_gauss(3000, 622)
    inst = sk.Instance(Jg, stream=st)
    run = sk.Run(inst, chains=chains, rule=sk.SK_RULE_METROPOLIS, beta=1.0, seed=4)
    b = sk.Batch([run])
    b.set_layout(4, 1)
    assert b.classes()[0][1] > 4
    b.advance(steps)
    b.close()
    spins, h, _ = run.state(fields=True)
    exact = (Jg.astype(np.float64) @ spins[sub].T.astype(np.float64)).T
    assert np.abs(h[sub] - exact).max() < 1e-4
    run.close(); inst.close()


def test_largest_n():
    need_gpu()
    N, K, chains, steps = 8192, 64, 2, 60
    J = inputs.couplings_pm1(N, 9)
    init = inputs.initial_spins(chains, N, 9)
    g = _run_gpu(J, chains=chains, K=K, beta=0.05, rule=sk.SK_RULE_MCMCMC, steps=steps, seed=4,
                 R=20, init=init, trace=2)
    o = oracle.run(J, K=K, beta=0.05, seed=4, chains=chains, init=init, steps=steps,
                   record_every=20, trace=True)
    assert np.array_equal(g["trace"], o["trace"])
    assert np.array_equal(g["E"], o["E"])
    assert np.array_equal(g["spins"], o["spins"])


@pytest.mark.parametrize("method", [sk.SK_SETGEN_DIRECT, sk.SK_SETGEN_CUMULATIVE])
@pytest.mark.parametrize("n", [1, 2, 5, 12, 20])
def test_set_generation_against_oracle(n, method):
    """sk_set_generation (App. D.2 recursion over subset masks, one launch per
    cardinality), direct and cumulative forms, against the oracle's forms:
    double precision, the same order of terms per mask (differences only from
    fused multiply-adds)."""
    torch = need_gpu()
    rng = np.random.default_rng(n)
    P = rng.random((n, n))
    np.fill_diagonal(P, 0.0)
    col = P.sum(axis=0, keepdims=True)
    P = P / (1.5 * np.where(col > 0, col, 1.0))
    got = sk.set_generation(P, method=method)
    want = oracle.setgen_dp(P) if method == sk.SK_SETGEN_DIRECT else oracle.setgen_cumulative(P)
    assert got[0] == 1.0 and got[-1] == 0.0
    assert np.all(np.abs(got - want) <= 1e-13 * np.abs(want) + 1e-300)
    assert np.all(np.abs(got - oracle.setgen_dp(P)) <= 1e-12 * np.abs(want) + 1e-300)
    dev = torch.zeros(1 << n, dtype=torch.float64, device="cuda")
    sk.set_generation(P, out=dev, method=method)
    assert np.array_equal(dev.cpu().numpy(), got)


def test_set_generation_arguments():
    need_gpu()
    with pytest.raises(sk.SKError):
        sk.set_generation(np.zeros((29, 29)))
    with pytest.raises(sk.SKError):
        sk.set_generation(-np.ones((3, 3)))
    with pytest.raises(sk.SKError) as e:
        sk.set_generation(np.zeros((3, 3)), method=3)
    assert e.value.status == sk.SK_ERR_INVALID_ARG


def test_batched_inputs_and_records_equal_single_calls():
    """sk_set_couplings_many / mcmcmc_reset_many / mcmcmc_observables_many give
    the same state and records as the per-instance calls; a bad input in any
    of them leaves every instance and run unchanged (all or nothing)."""
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, K, chains, R, steps = 72, 16, 6, 50, 200
    Js = [inputs.couplings_pm1(N, 100 + i) for i in range(3)]
    Js2 = [inputs.couplings_pm1(N, 200 + i) for i in range(3)]
    inits = [inputs.initial_spins(chains, N, 300 + i) for i in range(3)]
    insts = [sk.Instance(J, stream=st) for J in Js]
    runs = [sk.Run(x, chains=chains, K=K, beta=0.8, seed=5, stream_id=i, record_every=R,
                   max_records=steps // R) for i, x in enumerate(insts)]
    b = sk.Batch(runs)
    sk.set_couplings_many(insts, Js2)
    sk.reset_many(runs, inits)
    b.advance(steps)
    outs = [(np.zeros((steps // R, chains)), np.zeros((steps // R, chains // 2)),
             np.zeros((steps // R, chains), dtype=np.uint32)) for _ in runs]
    sk.observables_many(runs, 0, steps // R, outs)
    for i, r in enumerate(runs):
        o = oracle.run(Js2[i], K=K, beta=0.8, seed=5, stream=i, chains=chains, init=inits[i], steps=steps,
                       record_every=R)
        assert np.array_equal(outs[i][0], o["E"]) and np.array_equal(outs[i][2], o["acc"]), i
        assert np.array_equal(outs[i][1], o["q"]), i
        E, q, acc = r.observables()
        assert np.array_equal(E, outs[i][0])
    # all or nothing
    spins_before = [r.state()[0] for r in runs]
    bad = [J.copy() for J in Js]
    bad[2][1, 2] = -bad[2][1, 2]
    with pytest.raises(sk.SKError) as e:
        sk.set_couplings_many(insts, bad)
    assert "instance 2" in str(e.value)
    bs = [x.copy() for x in inits]
    bs[1][0, 0] = 3
    with pytest.raises(sk.SKError) as e:
        sk.reset_many(runs, bs)
    assert "run 1" in str(e.value)
    for i, r in enumerate(runs):
        spins, h, step = r.state(fields=True)
        assert step == steps and np.array_equal(spins, spins_before[i])
        assert np.array_equal(h, (Js2[i].astype(np.int64) @ spins.T.astype(np.int64)).T)  # old couplings kept
    b.close()
    for r in runs:
        r.close()
    for x in insts:
        x.close()


def test_batched_start_equals_single_starts_gaussian():
    """The batched start (one start launch and one tensor-core launch for all
    runs) writes the same spins and fields as mcmcmc_reset run by run."""
    torch = need_gpu()
    st = torch.cuda.Stream()
    N, chains = 200, 130   # ragged tiles
    Js = [inputs.couplings_gauss(N, 400 + i) for i in range(3)]
    inits = [inputs.initial_spins(chains, N, 500 + i) for i in range(3)]
    insts = [sk.Instance(J, stream=st) for J in Js]
    runs = [sk.Run(x, chains=chains, K=8, seed=2, stream_id=i, record_every=10, max_records=3)
            for i, x in enumerate(insts)]
    sk.reset_many(runs, [inits[0], None, inits[2]])
    got = [r.state(fields=True) for r in runs]
    for i, r in enumerate(runs):
        r.reset(inits[i] if i != 1 else None)
        s1, h1, step = r.state(fields=True)
        assert step == 0
        assert np.array_equal(got[i][0], s1) and np.array_equal(got[i][1], h1), i
        E, q, acc = r.observables()
        assert not E.any() and not acc.any()
    for r in runs:
        r.close()
    for x in insts:
        x.close()
