"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here calls the CUDA path.  Each test states what would break it:
 - Philox: published known-answer vectors and cuRAND's host Philox generator;
 - the node rule: exact detailed balance and stationarity of enumerated
   one-step transition matrices w.r.t. the brute-force Boltzmann weights
   (Sec. A.2, Eq. eq_det_balance_graph_solution), which fails for a dropped
   J_ab term, a wrong sign, a wrong root probability or a wrong slot weight;
 - K = 1 reduces to the two-node heat-bath chain (Sec. III.A, Eq. eq_node_two_conf);
 - beta = 0 has closed-form slot probabilities of the uniform-root star
   (App. B.2);
 - a star always rooted at the current state is NOT reversible (negative
   control: the detailed-balance test has teeth);
 - long runs reproduce the exact Boltzmann histogram and energy.
"""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    rows = _read_kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(oracle.philox(ctr, key)) == want


def test_philox_matches_curand_host_generator():
    path = "/usr/local/cuda/lib64/libcurand.so"
    if not os.path.exists(path):
        pytest.skip("libcurand not present")
    cr = ctypes.CDLL(path)
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    seed = 0x0123456789ABCDEF
    assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    n = 4 * 64
    out = np.zeros(n, dtype=np.uint32)
    assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    cr.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    # cuRAND's host Philox emits block i from counter (0, 0, i, 0)
    for i in range(n // 4):
        assert list(oracle.philox([0, 0, i, 0], key)) == list(out[4 * i:4 * i + 4])


def _pm1(N, seed):
    return inputs.couplings_pm1(N, seed)


def _gauss(N, seed):
    return inputs.couplings_gauss(N, seed)


def test_energy_definition_and_fields():
    # E = -sum_{i<j} J s s; E = -1/2 sum s h; single and double flip differences
    rng = np.random.default_rng(3)
    for J in (_pm1(9, 1), _gauss(9, 2)):
        s = inputs.initial_spins(1, 9, 5)[0]
        E = oracle.energy(J, s)
        Jd = J.astype(np.float64)
        want = -sum(Jd[i, j] * s[i] * s[j] for i in range(9) for j in range(i + 1, 9))
        assert abs(E - want) < 1e-12
        h = oracle.fields(J, s)
        assert np.allclose(h, Jd @ s.astype(np.float64), atol=1e-12)
        assert abs(E - (-0.5 * float(s @ h))) < 1e-12
        for _ in range(20):
            a, b = rng.choice(9, 2, replace=False)
            t = s.copy(); t[a] = -t[a]
            assert abs(oracle.energy(J, t) - E - 2 * s[a] * h[a]) < 1e-12
            t[b] = -t[b]
            d2 = 2 * s[a] * h[a] + 2 * s[b] * h[b] - 4 * Jd[a, b] * s[a] * s[b]
            assert abs(oracle.energy(J, t) - E - d2) < 1e-12
        assert abs(oracle.energy(J, s, scale=0.25) - 0.25 * E) < 1e-12


def _check_balance(P, pi, tol):
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-12)
    assert (P >= -1e-15).all()
    stat = np.abs(pi @ P - pi).max()
    flow = pi[:, None] * P
    db = np.abs(flow - flow.T).max()
    return stat, db


@pytest.mark.parametrize("kind", ["pm1", "gauss"])
@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_star_detailed_balance(kind, K):
    N = 6 if K <= 3 else 5
    J = _pm1(N, 11) if kind == "pm1" else _gauss(N, 12)
    beta = 0.7 if kind == "gauss" else 0.3
    pi = oracle.boltzmann(J, beta)
    P = oracle.transition_matrix(J, K=K, beta=beta)
    stat, db = _check_balance(P, pi, 1e-12)
    assert stat < 1e-13 and db < 1e-14, (stat, db)


def test_star_detailed_balance_integer_tables():
    # the +-J trajectories use integer weights: reversible to within table rounding
    J = _pm1(6, 21)
    for beta in (0.2, 1.0, 3.0):
        pi = oracle.boltzmann(J, beta)
        P = oracle.transition_matrix(J, K=3, beta=beta, weight_mode=1)
        stat, db = _check_balance(P, pi, 1e-12)
        assert stat < 1e-12 and db < 1e-12, (beta, stat, db)


def test_metropolis_detailed_balance_and_closed_form():
    J = _gauss(6, 31)
    beta = 1.3
    pi = oracle.boltzmann(J, beta)
    P = oracle.transition_matrix(J, rule=oracle.METROPOLIS, beta=beta)
    stat, db = _check_balance(P, pi, 1e-12)
    assert stat < 1e-13 and db < 1e-14
    # min(1, P_eq(c1)/P_eq(c0)) / N for each single flip (Sec. II)
    s = np.ones(6, dtype=np.int8)
    E0 = oracle.energy(J, s)
    for i in range(6):
        t = s.copy(); t[i] = -1
        want = min(1.0, math.exp(-beta * (oracle.energy(J, t) - E0))) / 6
        assert abs(P[0, 1 << i] - want) < 1e-14
    Jp = _pm1(6, 32)
    pi = oracle.boltzmann(Jp, 0.8)
    P = oracle.transition_matrix(Jp, rule=oracle.METROPOLIS, beta=0.8, weight_mode=1)
    stat, db = _check_balance(P, pi, 1e-12)
    assert stat < 1e-12 and db < 1e-12


def test_k1_is_two_node_heat_bath():
    # Sec. III.A: the two-node graph with P_node ~ P_eq is heat-bath:
    # P(c -> c^(i)) = (1/N) / (1 + exp(beta dE_i)) for every state and site.
    N, beta = 6, 0.9
    for J in (_gauss(N, 41), _pm1(N, 42)):
        P = oracle.transition_matrix(J, K=1, beta=beta)
        for x in range(1 << N):
            s = np.array([(-1 if (x >> i) & 1 else 1) for i in range(N)], dtype=np.int8)
            E0 = oracle.energy(J, s)
            for i in range(N):
                t = s.copy(); t[i] = -t[i]
                dE = oracle.energy(J, t) - E0
                assert abs(P[x, x ^ (1 << i)] - (1.0 / N) / (1.0 + math.exp(beta * dE))) < 1e-14


@pytest.mark.parametrize("K", [1, 2, 4])
def test_beta_zero_closed_form(K):
    # beta = 0: every slot equally likely.  Root = centre w.p. 1/(K+1), else a leaf.
    N = 5
    P = oracle.transition_matrix(_gauss(N, 51), K=K, beta=0.0)
    pc, pl = 1.0 / (K + 1), K / (K + 1)
    single = pc * (K / (K + 1)) / N + pl * (1.0 / (K + 1)) / N
    double = pl * ((K - 1) / (K + 1)) * 2.0 / N**2
    stay = pc / (K + 1) + pl * (1.0 / (K + 1) + ((K - 1) / (K + 1)) / N)
    for x in range(1 << N):
        assert abs(P[x, x] - stay) < 1e-14
        for i in range(N):
            assert abs(P[x, x ^ (1 << i)] - single) < 1e-14
            for j in range(i + 1, N):
                assert abs(P[x, x ^ (1 << i) ^ (1 << j)] - double) < 1e-14


def test_centre_rooted_star_is_not_reversible():
    # negative control: heat-bath over the K+1 nodes of a star always rooted at
    # the current state violates detailed balance for K >= 2 (App. B.2 needs p_r)
    J = _gauss(5, 61)
    beta = 0.7
    pi = oracle.boltzmann(J, beta)
    P = oracle.transition_matrix(J, K=3, beta=beta, root_mode=1)
    stat, db = _check_balance(P, pi, 1e-12)
    assert stat > 1e-4 and db > 1e-4
    # ... while K = 1 is the heat-bath chain either way
    P1 = oracle.transition_matrix(J, K=1, beta=beta, root_mode=1)
    stat, db = _check_balance(P1, pi, 1e-12)
    assert stat < 1e-13 and db < 1e-14


@pytest.mark.parametrize("kind", ["pm1", "gauss"])
@pytest.mark.parametrize("K,p_center", [(2, 0.05), (2, 0.9), (3, 0.3), (4, 0.5)])
def test_nonuniform_root_detailed_balance(kind, K, p_center):
    # App. B.2: any root distribution p_r with the node weights P_eq p_r(node)
    # leaves P_eq invariant and the chain reversible
    N = 5
    J = _pm1(N, 13) if kind == "pm1" else _gauss(N, 14)
    beta = 0.4 if kind == "pm1" else 0.8
    pi = oracle.boltzmann(J, beta)
    P = oracle.transition_matrix(J, K=K, beta=beta, p_center=p_center)
    stat, db = _check_balance(P, pi, 1e-12)
    assert stat < 1e-13 and db < 1e-14, (stat, db)
    if kind == "pm1":  # the integer tables with the integer root factors
        P = oracle.transition_matrix(J, K=K, beta=beta, weight_mode=1, p_center=p_center)
        stat, db = _check_balance(P, pi, 1e-12)
        assert stat < 1e-12 and db < 1e-12, (stat, db)
    # negative control: the same root probabilities without the p_r factor
    P = oracle.transition_matrix(J, K=K, beta=beta, root_mode=2, p_center=p_center)
    stat, db = _check_balance(P, pi, 1e-12)
    assert db > 1e-5, db


@pytest.mark.parametrize("K,p_center", [(2, 0.2), (4, 0.5), (3, 0.25)])
def test_nonuniform_root_beta_zero_closed_form(K, p_center):
    # beta = 0: slot j is chosen with probability p_r(j) / sum_slots p_r.  With
    # the centre as root (probability p_c): stay w.p. p_c, flip one of the K
    # leaves' sites otherwise.  With a leaf as root (1 - p_c): stay at the root
    # (p_l) or at a leaf whose site repeats a = site_1, flip a (the centre,
    # p_c), or flip a and b != a (a leaf).  (These p_center are exact: the
    # factor ratio p_c / p_l is a power of two.)
    N = 5
    P = oracle.transition_matrix(_gauss(N, 52), K=K, beta=0.0, p_center=p_center)
    pc = p_center
    pl = (1.0 - pc) / K
    single = pc * (K * pl) / N + (1 - pc) * pc / N
    double = (1 - pc) * ((K - 1) * pl) * 2.0 / N**2
    stay = pc * pc + (1 - pc) * (pl + (K - 1) * pl / N)
    for x in range(1 << N):
        assert abs(P[x, x] - stay) < 1e-14
        for i in range(N):
            assert abs(P[x, x ^ (1 << i)] - single) < 1e-14
            for j in range(i + 1, N):
                assert abs(P[x, x ^ (1 << i) ^ (1 << j)] - double) < 1e-14


def test_uniform_p_center_is_the_uniform_root():
    # p_center = 1/(K+1) is the uniform root: same transition matrix, and the
    # same trajectories (the root thresholds differ on ~2^-53 of the draws)
    N, K = 6, 3
    J = _pm1(N, 15)
    P0 = oracle.transition_matrix(J, K=K, beta=0.5, weight_mode=1)
    P1 = oracle.transition_matrix(J, K=K, beta=0.5, weight_mode=1, p_center=1.0 / (K + 1))
    assert np.abs(P0 - P1).max() < 1e-15
    Jb = _pm1(48, 16)
    a = oracle.run(Jb, K=8, beta=0.7, seed=3, chains=4, steps=2000, trace=True)
    b = oracle.run(Jb, K=8, beta=0.7, seed=3, chains=4, steps=2000, trace=True, p_center=1.0 / 9)
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["spins"], b["spins"])
    with pytest.raises(RuntimeError):
        oracle.run(Jb, K=8, beta=0.7, p_center=1.0)
    with pytest.raises(RuntimeError):
        oracle.run(Jb, K=8, beta=0.7, p_center=1e-9)  # leaf factor below 2^-20


def test_nonuniform_root_one_step_sampler_matches_exact_row():
    # the trajectory code's root threshold and factors sample the enumerated row
    N, K, beta = 5, 3, 0.6
    for kind, J in (("pm1", _pm1(N, 72)), ("gauss", _gauss(N, 73))):
        wm = 1 if kind == "pm1" else 0
        for p_center in (0.1, 0.7):
            P = oracle.transition_matrix(J, K=K, beta=beta, weight_mode=wm, p_center=p_center)
            x0 = 0b10110
            s0 = np.array([(-1 if (x0 >> i) & 1 else 1) for i in range(N)], dtype=np.int8)
            C = 30000
            r = oracle.run(J, K=K, beta=beta, seed=11, chains=C, init=np.tile(s0, (C, 1)), steps=1,
                           p_center=p_center)
            ys = ((r["spins"] < 0).astype(np.int64) << np.arange(N)).sum(axis=1)
            counts = np.bincount(ys, minlength=1 << N).astype(float)
            assert _chi2_pvalue(counts, P[x0] * C) > 1e-3, (kind, p_center)


def _state(x, N):
    return np.array([(-1 if (x >> i) & 1 else 1) for i in range(N)], dtype=np.int8)


@pytest.mark.parametrize("kind,rule,p_center", [("pm1", oracle.MCMCMC, 0.0), ("gauss", oracle.MCMCMC, 0.0),
                                                ("gauss", oracle.MCMCMC, 0.6), ("gauss", oracle.METROPOLIS, 0.0),
                                                ("pm1", oracle.METROPOLIS, 0.0)])
def test_node_weighted_energy_is_the_conditional_expectation(kind, rule, p_center):
    # Eq. eq_monte_carlo_graph: for the recorded state x and the graph T of the
    # next step, sum_j P_node(j) E(c_j) = E[E(next state) | x, T]; averaged over
    # T it is sum_y P(x, y) E(y), and it has less variance than E(next state)
    N, K, beta = 5, 3, 0.6
    J = _pm1(N, 74) if kind == "pm1" else _gauss(N, 75)
    wm = 1 if kind == "pm1" else 0
    P = oracle.transition_matrix(J, rule=rule, K=K, beta=beta, weight_mode=wm, p_center=p_center)
    Es = np.array([oracle.energy(J, _state(x, N)) for x in range(1 << N)])
    PE = P @ Es
    x0 = 0b00110
    C = 20000
    # record after step 0 (state x1, graph of step 1) and after step 1 (state x2)
    r = oracle.run(J, rule=rule, K=K, beta=beta, seed=13, chains=C, init=np.tile(_state(x0, N), (C, 1)),
                   steps=2, record_every=1, p_center=p_center)
    init = np.tile(_state(x0, N), (C, 1))
    r1 = oracle.run(J, rule=rule, K=K, beta=beta, seed=13, chains=C, init=init, steps=1, p_center=p_center)
    x1 = ((r1["spins"] < 0).astype(np.int64) << np.arange(N)).sum(axis=1)
    nw, e2 = r["E_nw"][0], r["E"][1]
    d = nw - PE[x1]
    assert abs(d.mean()) < 4 * d.std() / math.sqrt(C) + 1e-12, (d.mean(), d.std())
    assert abs(nw.mean() - e2.mean()) < 4 * e2.std() / math.sqrt(C)
    assert nw.var() < e2.var()


def test_node_weighted_energy_by_explicit_star():
    # after one step, build the K+1 configurations of the next step's star
    # from its draws, weight their full energies exp(-beta E), compare
    N, K, beta, seed = 9, 6, 0.8, 5
    J = _gauss(N, 76)
    rng = np.random.default_rng(3)
    C = 6
    init = rng.choice(np.array([-1, 1], dtype=np.int8), size=(C, N))
    r = oracle.run(J, K=K, beta=beta, seed=seed, chains=C, init=init, steps=1, record_every=1)
    for chain in range(C):
        s1 = r["spins"][chain]
        w = oracle.philox([0, 1, chain, 0], [seed, 0])
        U0 = (int(w[1]) << 32) | int(w[0])
        leaf = (U0 * (K + 1)) >> 64 != 0
        sites = []
        for d in range(1, K + 1):
            b = oracle.philox([1 + (d - 1) // 4, 1, chain, 0], [seed, 0])
            sites.append((int(b[(d - 1) % 4]) * N) >> 32)
        confs = [s1.copy()]
        for d in range(1, K + 1):
            c = s1.copy()
            if not leaf:
                c[sites[d - 1]] *= -1
            else:
                c[sites[0]] *= -1
                if d >= 2:
                    c[sites[d - 1]] *= -1
            confs.append(c)
        E = np.array([oracle.energy(J, c) for c in confs])
        wts = np.exp(-beta * (E - E.min()))
        want = float((wts * E).sum() / wts.sum())
        assert abs(r["E_nw"][0, chain] - want) < 1e-12, (chain, r["E_nw"][0, chain], want)


def test_node_weighted_long_run_matches_exact_mean():
    N, K, beta = 12, 8, 1.0
    J = _pm1(N, 0)
    pi = oracle.boltzmann(J, beta)
    Es = np.array([oracle.energy(J, _state(x, N)) for x in range(1 << N)])
    exact = float((pi * Es).sum())
    C = 4000
    r = oracle.run(J, K=K, beta=beta, seed=21, chains=C, steps=400, record_every=100)
    nw = r["E_nw"][1:].ravel()
    e = r["E"][1:].ravel()
    assert abs(nw.mean() - exact) < 5 * e.std() / math.sqrt(C)
    assert nw.var() < e.var()


GRAPHS = [dict(graph=oracle.TREE, arity=2, depth=1), dict(graph=oracle.TREE, arity=3, depth=1),
          dict(graph=oracle.TREE, arity=2, depth=2), dict(graph=oracle.LINE, line_nodes=3),
          dict(graph=oracle.LINE, line_nodes=4), dict(graph=oracle.LINE, line_nodes=6)]


@pytest.mark.parametrize("kind", ["pm1", "gauss"])
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_graph_detailed_balance(kind, gi):
    # App. B: a tree populated from a uniformly placed root is self-thermalising;
    # the line's binomial root position with node weights ~ P_eq binom(L-1, v)
    # (Eq. eq_create_line_graph) is reversible too
    N = 4
    J = _pm1(N, 17) if kind == "pm1" else _gauss(N, 18)
    beta = 0.5 if kind == "pm1" else 0.9
    pi = oracle.boltzmann(J, beta)
    P = oracle.transition_matrix_graph(J, beta=beta, **GRAPHS[gi])
    stat, db = _check_balance(P, pi, 1e-12)
    assert stat < 1e-12 and db < 1e-13, (stat, db)
    if kind == "pm1":
        P = oracle.transition_matrix_graph(J, beta=beta, weight_mode=1, **GRAPHS[gi])
        stat, db = _check_balance(P, pi, 1e-12)
        assert stat < 1e-12 and db < 1e-12, (stat, db)


def test_tree_of_depth_one_is_the_star():
    J = _gauss(5, 19)
    for K in (1, 2, 3):
        if K == 1:
            Pt = oracle.transition_matrix_graph(J, beta=0.8, graph=oracle.LINE, line_nodes=2)
        else:
            Pt = oracle.transition_matrix_graph(J, beta=0.8, graph=oracle.TREE, arity=K, depth=1)
        Ps = oracle.transition_matrix(J, K=K, beta=0.8)
        assert np.abs(Pt - Ps).max() < 1e-15, K


def test_line_beta_zero_closed_form():
    # L = 3, beta = 0: root at node 0, 1, 2 w.p. 1/4, 1/2, 1/4 and node v chosen
    # w.p. binom(2, v)/4; worked out by hand over the two edge sites
    N = 5
    P = oracle.transition_matrix_graph(_gauss(N, 53), beta=0.0, graph=oracle.LINE, line_nodes=3)
    stay = 3 / 8 + 1 / (8 * N)
    single = 1 / (2 * N)
    double = 1 / (4 * N * N)
    for x in range(1 << N):
        assert abs(P[x, x] - stay) < 1e-14
        for i in range(N):
            assert abs(P[x, x ^ (1 << i)] - single) < 1e-14
            for j in range(i + 1, N):
                assert abs(P[x, x ^ (1 << i) ^ (1 << j)] - double) < 1e-14


@pytest.mark.parametrize("gi", [2, 4])
def test_graph_one_step_sampler_matches_exact_row(gi):
    N, beta = 4, 0.6
    J = _pm1(N, 77)
    P = oracle.transition_matrix_graph(J, beta=beta, weight_mode=1, **GRAPHS[gi])
    x0 = 0b0110
    C = 30000
    r = oracle.run_graph(J, beta=beta, seed=17, chains=C, init=np.tile(_state(x0, N), (C, 1)), steps=1,
                         **GRAPHS[gi])
    ys = ((r["spins"] < 0).astype(np.int64) << np.arange(N)).sum(axis=1)
    counts = np.bincount(ys, minlength=1 << N).astype(float)
    assert _chi2_pvalue(counts, P[x0] * C) > 1e-3


@pytest.mark.parametrize("g", [dict(graph=oracle.TREE, arity=2, depth=3), dict(graph=oracle.LINE, line_nodes=8)])
def test_graph_long_run_matches_boltzmann_n12(g):
    N, beta = 12, 1.0
    J = _pm1(N, 0)
    pi = oracle.boltzmann(J, beta)
    Es = np.array([oracle.energy(J, _state(x, N)) for x in range(1 << N)])
    C = 6000
    r = oracle.run_graph(J, beta=beta, seed=5, chains=C, steps=150, **g)
    ys = ((r["spins"] < 0).astype(np.int64) << np.arange(N)).sum(axis=1)
    counts = np.bincount(ys, minlength=1 << N).astype(float)
    levels = np.unique(Es)
    obs = np.array([counts[Es == e].sum() for e in levels])
    exp_ = np.array([pi[Es == e].sum() for e in levels]) * C
    assert _chi2_pvalue(obs, exp_) > 1e-3


def _setgen_P(n, seed):
    rng = np.random.default_rng(seed)
    P = rng.random((n, n))
    np.fill_diagonal(P, 0.0)
    col = P.sum(axis=0, keepdims=True)
    return P / (1.5 * np.where(col > 0, col, 1.0))  # P[e, p] = P_gen(e | p), leaves mass outside S


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_setgen_recursion_equals_the_process(n):
    # App. D.2's recursion on the first addition against the definition of
    # App. D.1: every order of the missing elements, each addition from a
    # uniformly chosen parent of the current set
    P = _setgen_P(n, 10 + n)
    dp = oracle.setgen_dp(P)
    for M in range(1 << n):
        bf = oracle.setgen_bruteforce(P, M)
        assert abs(dp[M] - bf) <= 1e-15 * max(1.0, abs(bf)), (M, dp[M], bf)


@pytest.mark.parametrize("n", [1, 2, 4, 7, 12])
def test_setgen_cumulative_form_equals_the_recursion(n):
    # App. D.2's O(n 2^n) form: the cumulative table c(M, e) built by removing
    # one term per added element, then Eq. eq_rec_set_short; against the
    # definition (n <= 7) and the first-addition recursion
    P = _setgen_P(n, 40 + n)
    cu = oracle.setgen_cumulative(P)
    dp = oracle.setgen_dp(P)
    assert np.all(np.abs(cu - dp) <= 1e-14 * np.maximum(1.0, np.abs(dp)))
    if n <= 7:
        for M in range(1 << n):
            bf = oracle.setgen_bruteforce(P, M)
            assert abs(cu[M] - bf) <= 1e-15 * max(1.0, abs(bf)), (M, cu[M], bf)


def test_setgen_cumulative_orientation_matters():
    # a pin on the reading of the garbled cumulative definition: with P_gen
    # transposed (generated element and parent swapped) the table gives a
    # different answer for asymmetric P -- the test above would catch that
    # mistake
    n = 5
    P = _setgen_P(n, 77)
    assert not np.allclose(oracle.setgen_cumulative(P.T.copy()), oracle.setgen_dp(P))


def test_setgen_closed_forms():
    # n = 2: the missing element a comes from the only other element b
    P = _setgen_P(2, 3)
    dp = oracle.setgen_dp(P)
    assert dp[0] == 1.0 and abs(dp[1] - P[0, 1]) < 1e-16 and abs(dp[2] - P[1, 0]) < 1e-16 and dp[3] == 0.0
    # parent-independent proposals q: any order, any parent: |M|! q^|M|
    n, q = 8, 0.013
    Pu = np.full((n, n), q)
    np.fill_diagonal(Pu, 0.0)
    dp = oracle.setgen_dp(Pu)
    for M in range((1 << n) - 1):
        k = bin(M).count("1")
        assert abs(dp[M] - math.factorial(k) * q ** k) <= 1e-14 * math.factorial(k) * q ** k


def test_setgen_printed_normalisation_differs_by_a_cardinality_factor():
    # reading of App. D.2: the printed recursion carries 1/(|S'| |S minus S'|) and a
    # 1/|S| base case; against the process it differs by a factor that depends
    # only on |S'| (it cancels between sets of one cardinality)
    n = 6
    P = _setgen_P(n, 99)
    dp = oracle.setgen_dp(P)
    printed = np.zeros(1 << n)
    full = (1 << n) - 1
    for M in range(1, full):
        cur = [p for p in range(n) if not (M >> p) & 1]
        mem = [e for e in range(n) if (M >> e) & 1]
        if len(mem) == 1:
            e = mem[0]
            printed[M] = sum(P[e, p] for p in range(n) if p != e) / n
        else:
            printed[M] = sum(P[e, p] * printed[M & ~(1 << e)] for e in mem for p in cur) / (len(mem) * len(cur))
    for k in range(1, n):
        ratios = [printed[M] / dp[M] for M in range(1, full) if bin(M).count("1") == k]
        assert max(ratios) - min(ratios) <= 1e-12 * max(ratios), k


def test_weight_table_shape():
    W = oracle.weight_table(1.0, 400)
    assert int(W[0]) == 1 << 52
    assert all(int(W[d]) >= int(W[d + 1]) for d in range(len(W) - 1))
    # the first dropped entry is the first that rounds to zero
    assert 2.0 ** 52 * math.exp(-2.0 * len(W)) < 0.5
    W0 = oracle.weight_table(0.0, 40)
    assert len(W0) == 41 and all(int(w) == 1 << 52 for w in W0)


def _chi2_pvalue(obs, exp_counts):
    from scipy.stats import chi2
    m = exp_counts > 5
    x = ((obs[m] - exp_counts[m]) ** 2 / exp_counts[m]).sum()
    rest_o, rest_e = obs[~m].sum(), exp_counts[~m].sum()
    dof = int(m.sum()) - 1
    if rest_e > 0:
        x += (rest_o - rest_e) ** 2 / max(rest_e, 1e-9)
        dof += 1
    return chi2.sf(x, dof)


def test_one_step_sampler_matches_exact_row():
    # the Philox-driven step (draws, root, sites, integer selection) samples the
    # enumerated transition row: many chains, one step each, from a fixed state
    N, K, beta = 5, 3, 0.6
    J = _pm1(N, 71)
    P = oracle.transition_matrix(J, K=K, beta=beta, weight_mode=1)
    x0 = 0b01101
    s0 = np.array([(-1 if (x0 >> i) & 1 else 1) for i in range(N)], dtype=np.int8)
    C = 40000
    r = oracle.run(J, K=K, beta=beta, seed=7, chains=C, init=np.tile(s0, (C, 1)), steps=1)
    ys = ((r["spins"] < 0).astype(np.int64) << np.arange(N)).sum(axis=1)
    counts = np.bincount(ys, minlength=1 << N).astype(float)
    assert _chi2_pvalue(counts, P[x0] * C) > 1e-3


def test_long_run_histogram_matches_boltzmann_n12():
    # config-1 companion: +-J N = 12, beta = 1, K = 8, histogram over states
    N, K, beta = 12, 8, 1.0
    J = _pm1(N, 0)
    pi = oracle.boltzmann(J, beta)
    # many independent chains, the final state of each after 300 steps
    C = 20000
    r = oracle.run(J, K=K, beta=beta, seed=2, chains=C, steps=300)
    ys = ((r["spins"] < 0).astype(np.int64) << np.arange(N)).sum(axis=1)
    counts = np.bincount(ys, minlength=1 << N).astype(float)
    # compare the energy-level histogram (coarse-grained by exact energy)
    Es = np.array([oracle.energy(J, np.array([(-1 if (x >> i) & 1 else 1) for i in range(N)],
                                                dtype=np.int8)) for x in range(1 << N)])
    levels = np.unique(Es)
    obs = np.array([counts[Es == e].sum() for e in levels])
    exp_ = np.array([pi[Es == e].sum() for e in levels]) * C
    assert _chi2_pvalue(obs, exp_) > 1e-3
    mean_E = float((counts * Es).sum() / C)
    exact = float((pi * Es).sum())
    sd = math.sqrt(float((pi * (Es - exact) ** 2).sum()) / C)
    assert abs(mean_E - exact) < 4 * sd


def test_metropolis_long_run_energy_matches_exact():
    N, beta = 10, 0.8
    J = _gauss(N, 81)
    pi = oracle.boltzmann(J, beta)
    Es = np.array([oracle.energy(J, np.array([(-1 if (x >> i) & 1 else 1) for i in range(N)],
                                                dtype=np.int8)) for x in range(1 << N)])
    C = 8000
    r = oracle.run(J, rule=oracle.METROPOLIS, beta=beta, seed=3, chains=C, steps=600)
    exact = float((pi * Es).sum())
    sd = math.sqrt(float((pi * (Es - exact) ** 2).sum()) / C)
    assert abs(r["final_E"].mean() - exact) < 4 * sd


def test_fields_stay_consistent_over_a_run():
    # maintained fields == recomputed fields: exact for +-J, 1e-9 for Gaussian
    for J in (_pm1(40, 91), _gauss(40, 92)):
        oracle.run(J, K=16, beta=1.0, seed=5, chains=2, steps=3000, resync_every=7)
        oracle.run(J, rule=oracle.METROPOLIS, beta=1.0, seed=5, chains=2, steps=3000,
                   resync_every=7)


def test_records_consistent_with_final_state():
    J = _pm1(32, 101)
    r = oracle.run(J, K=8, beta=0.5, seed=9, chains=4, steps=500, record_every=100)
    assert r["E"].shape == (5, 4)
    assert np.array_equal(r["E"][-1], r["final_E"])
    for c in range(4):
        assert r["E"][-1, c] == oracle.energy(J, r["spins"][c])
    q = (r["spins"][0].astype(float) @ r["spins"][1]) / 32
    assert r["q"][-1, 0] == q
    assert (r["acc"] <= 100).all()


def test_random_start_is_philox_domain_one():
    s = oracle.init_spins(seed=77, stream=3, chain=5, N=300)
    key = [77, 0]
    bits = []
    for b in range(3):
        w = oracle.philox([b, 0, 5, (1 << 24) | 3], key)
        for k in range(128):
            bits.append((int(w[k // 32]) >> (k % 32)) & 1)
    want = np.array([-1 if x else 1 for x in bits[:300]], dtype=np.int8)
    assert np.array_equal(s, want)
    # balanced start
    s = oracle.init_spins(seed=1, stream=0, chain=0, N=100000)
    assert abs(int(s.astype(np.int64).sum())) < 5 * math.sqrt(100000)


def test_high_temperature_energy_gaussian():
    # textbook high-temperature (annealed) SK result, leading order in beta:
    # <E> ~ -beta sum_{i<j} J_ij^2 (Sherrington & Kirkpatrick 1975); loose check
    N, beta = 128, 0.3
    J = _gauss(N, 111)
    want = -beta * float(np.triu(J.astype(np.float64) ** 2, 1).sum())
    r = oracle.run(J, rule=oracle.METROPOLIS, beta=beta, seed=4, chains=32, steps=40000,
                   record_every=1000)
    got = r["E"][10:].mean()
    assert abs(got - want) < 0.08 * abs(want), (got, want)


# ---------------------------------------------------------------------------
# couplings drawn from a seed (Philox domain 2): the generator behind
# sk_create_instance with NULL couplings, pinned by the properties its
# definition fixes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [oracle.PM1, oracle.GAUSS])
def test_generated_couplings_are_a_valid_instance(kind):
    N = 200
    J = oracle.gen_couplings(N, kind, 12345)
    assert np.array_equal(J, J.T)
    assert np.all(np.diag(J) == 0)
    if kind == oracle.PM1:
        assert set(np.unique(J[~np.eye(N, dtype=bool)])) == {-1, 1}
    else:
        assert np.all(np.isfinite(J))
    assert not np.array_equal(J, oracle.gen_couplings(N, kind, 12346))   # another seed, another draw
    assert np.array_equal(J, oracle.gen_couplings(N, kind, 12345))       # deterministic


def test_generated_pm1_couplings_are_equiprobable_bits():
    # the +-J signs are the block's bits: fair coin flips, independent of position
    N = 700
    J = oracle.gen_couplings(N, oracle.PM1, 7)
    up = J[np.triu_indices(N, 1)]
    n = up.size
    z = (np.sum(up == 1) - n / 2) / math.sqrt(n / 4)
    assert abs(z) < 4.5, z
    # neighbouring columns (bits of one word) and rows are uncorrelated
    a = J[np.triu_indices(N, 2)].astype(float)
    b = np.roll(J, -1, axis=1)[np.triu_indices(N, 2)].astype(float)
    assert abs(np.mean(a * b)) < 4.5 / math.sqrt(a.size)
    # the mapping as defined: J_01 = -1 iff bit 1 of word 0 of block (0, 0, 0, 2 << 24)
    w = oracle.philox([0, 0, 0, 2 << 24], [7, 0])
    assert J[0, 1] == (-1 if (int(w[0]) >> 1) & 1 else 1)
    w = oracle.philox([600 >> 7, 3, 0, 2 << 24], [7, 0])
    b = 600 % 128
    assert J[3, 600] == (-1 if (int(w[b // 32]) >> (b % 32)) & 1 else 1)


def test_generated_gaussian_couplings_are_n01_over_n():
    scipy_stats = pytest.importorskip("scipy.stats")
    N = 600
    J = oracle.gen_couplings(N, oracle.GAUSS, 99).astype(np.float64)
    x = J[np.triu_indices(N, 1)] * math.sqrt(N)   # should be N(0, 1)
    n = x.size
    assert abs(x.mean()) < 4.5 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 4.5 * math.sqrt(2.0 / n)
    assert scipy_stats.kstest(x, "norm").pvalue > 1e-3
    # fourth moment of a normal: 3
    assert abs(np.mean(x ** 4) - 3.0) < 4.5 * math.sqrt(96.0 / n)
    # the Box-Muller recipe as defined, for one pair
    w = [int(v) for v in oracle.philox([5, 2, 1, 2 << 24], [99, 0])]
    u1 = ((w[0] >> 5) * 67108864.0 + (w[1] >> 6)) * 2.0 ** -53
    u2 = ((w[2] >> 5) * 67108864.0 + (w[3] >> 6)) * 2.0 ** -53
    z = math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)
    assert abs(J[2, 5] - np.float32(z / math.sqrt(N))) <= np.spacing(np.float32(abs(J[2, 5])))
