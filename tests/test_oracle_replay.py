"""Pins of the oracle's decision-replay checker (oracle.replay / replay_graph).

Every Gaussian parity test of the CUDA path rests on this checker: the oracle
walks the chain with its own random numbers but follows the slot log taken on
the GPU, and a step whose slot differs from the oracle's own choice is
admissible only when the oracle's draw u lies within tol * P_K of that slot's
interval [P_{j-1}, P_j) -- a near-tie that fp32 rounding may decide either way
(the node choice of Sec. A.2, Eq. eq_det_balance_graph_solution, taken as the
first slot whose inclusive weight prefix exceeds u).  Metropolis (Sec. II): a
flipped decision is admissible when |u - p_acc| <= tol.

What fixes the checker here, independently of its own code:
  - the per-step draws and prefix sums (run_detail) are the ones the chain's
    choices are taken with: the chosen slot is the first j with P_j > u, and the
    detail trajectory equals the trace of oracle.run;
  - replaying the oracle's own trace disagrees nowhere;
  - a slot whose interval lies far from u is flagged at exactly that step
    (a checker that took its own choice after applying the forced slot, or
    compared nothing, passes it);
  - at a near-tie with distance d of u to the boundary shared by two slots, the
    neighbour across the boundary is admitted for tol * P_K above d and flagged
    below it, with u above the boundary (the neighbour's upper end) and below it
    (its lower end), u < P_K / 2 and P_K > 2 (so that a window of tol * u or of
    tol alone, or an off-by-one in the interval ends, fails one of the cases).
"""
import numpy as np
import pytest

import oracle
from paper_2102_05613_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


def _first_above(P, u):
    """The definition of the node choice: the first slot whose inclusive prefix exceeds u."""
    return int(np.argmax(P > u))


STAR_CASES = [  # kind, rule, K, p_center
    (oracle.GAUSS, oracle.MCMCMC, 8, 0.0),
    (oracle.GAUSS, oracle.MCMCMC, 33, 0.3),
    (oracle.PM1, oracle.MCMCMC, 16, 0.0),
    (oracle.GAUSS, oracle.METROPOLIS, 1, 0.0),
    (oracle.PM1, oracle.METROPOLIS, 1, 0.0),
]


def _J(kind, N, seed):
    return inputs.couplings(N, kind, seed)


@pytest.mark.parametrize("kind,rule,K,p_center", STAR_CASES)
def test_detail_is_the_trajectory_and_the_choice(kind, rule, K, p_center):
    J = _J(kind, 20, 3)
    steps = 600
    d = oracle.run_detail(J, rule=rule, K=K, beta=1.0, seed=9, stream=2, chain=5, steps=steps,
                          p_center=p_center)
    r = oracle.run(J, rule=rule, K=K, beta=1.0, seed=9, stream=2, chain0=5, chains=1, steps=steps,
                   trace=True, p_center=p_center)
    assert np.array_equal(d["own"], r["trace"][0])
    if rule == oracle.METROPOLIS:
        # accepted iff u < p_acc (p_acc = 1 for a move downhill)
        acc = d["u"] < d["P"][:, 0]
        assert np.array_equal(acc.astype(np.int32), d["own"])
        assert np.all((d["P"] > 0) & (d["P"] <= 1.0))
    else:
        P = d["P"]
        assert np.all(np.diff(P, axis=1) >= 0)
        assert np.all((d["u"] >= 0) & (d["u"] < P[:, -1]))
        if kind == oracle.GAUSS:  # the +-J prefix sums exceed 2^53 and are rounded as doubles here
            own = np.array([_first_above(P[t], d["u"][t]) for t in range(steps)])
            assert np.array_equal(own, d["own"])


@pytest.mark.parametrize("kind,rule,K,p_center", STAR_CASES)
def test_replay_of_own_trace_is_clean(kind, rule, K, p_center):
    J = _J(kind, 24, 4)
    r = oracle.run(J, rule=rule, K=K, beta=1.5, seed=11, stream=1, chain0=3, chains=1, steps=2000,
                   trace=True, p_center=p_center)
    rp = oracle.replay(J, r["trace"][0], rule=rule, K=K, beta=1.5, seed=11, stream=1, chain=3,
                       tol=1e-4, p_center=p_center)
    assert (rp["bad"], rp["disagree"], rp["first_bad"]) == (0, 0, -1)
    assert np.array_equal(rp["spins"], r["spins"][0])
    assert rp["final_E"] == pytest.approx(r["final_E"][0], abs=1e-12)


def _far_slot(P, u, min_gap):
    """A slot of positive width whose interval [P_{j-1}, P_j) is at least
    min_gap away from u, or None."""
    lo = np.concatenate(([0.0], P[:-1]))
    for j in np.argsort(-np.abs(0.5 * (lo + P) - u)):
        if P[j] > lo[j] and (u < lo[j] - min_gap or u >= P[j] + min_gap):
            return int(j)
    return None


def test_replay_flags_a_far_slot_at_its_step():
    J = _J(oracle.GAUSS, 24, 5)
    K, steps = 8, 400
    d = oracle.run_detail(J, K=K, beta=1.0, seed=13, chain=0, steps=steps)
    flagged = 0
    for t_bad in (7, 150, 333):
        P, u = d["P"][t_bad], d["u"][t_bad]
        g = _far_slot(P, u, 0.05 * P[-1])
        assert g is not None and g != d["own"][t_bad]
        tr = d["own"].copy()
        tr[t_bad] = g
        rp = oracle.replay(J, tr, K=K, beta=1.0, seed=13, chain=0, tol=1e-4)
        assert rp["first_bad"] == t_bad and rp["bad"] >= 1 and rp["disagree"] >= 1
        flagged += 1
    assert flagged == 3


def test_replay_flags_a_flipped_metropolis_decision():
    J = _J(oracle.GAUSS, 24, 6)
    d = oracle.run_detail(J, rule=oracle.METROPOLIS, beta=1.0, seed=17, chain=1, steps=500)
    gap = np.abs(d["u"] - d["P"][:, 0])
    t_bad = int(np.nonzero(gap > 0.1)[0][20])
    tr = d["own"].copy()
    tr[t_bad] ^= 1
    rp = oracle.replay(J, tr, rule=oracle.METROPOLIS, beta=1.0, seed=17, chain=1, tol=1e-4)
    assert rp["first_bad"] == t_bad and rp["bad"] >= 1


def _near_ties(P, u, own):
    """Steps with u < P_K/2 and P_K > 2 next to a boundary b = P_j between two
    slots of positive width: (t, neighbour slot, distance, side) for the
    closest such step with u above its boundary (the neighbour below, whose
    upper end is b) and the closest with u below it (the neighbour above)."""
    best = {}
    for t in range(len(u)):
        PK = P[t, -1]
        if not (u[t] < 0.5 * PK and PK > 2.0):
            continue
        lo = np.concatenate(([0.0], P[t, :-1]))
        w = P[t] - lo
        j = own[t]
        # u in [lo_j, P_j): the boundaries of the chosen slot are lo_j (side
        # "above": the neighbour is the slot below) and P_j ("below")
        if j > 0:
            k = j - 1
            while k >= 0 and w[k] <= 0:
                k -= 1
            if k >= 0:
                dist = u[t] - lo[j]
                if "above" not in best or dist / PK < best["above"][2] / P[best["above"][0], -1]:
                    best["above"] = (t, k, dist)
        if j + 1 < P.shape[1]:
            k = j + 1
            while k < P.shape[1] and w[k] <= 0:
                k += 1
            if k < P.shape[1]:
                dist = P[t, j] - u[t]
                if "below" not in best or dist / PK < best["below"][2] / P[best["below"][0], -1]:
                    best["below"] = (t, k, dist)
    return best


def _check_near_tie(replay_fn, own, t, g, dist, PK, u):
    tr = own[: t + 1].copy()
    tr[t] = g
    assert dist > 0 and u < 0.5 * PK and PK > 2.0
    ok = replay_fn(tr, 1.5 * dist / PK)
    assert (ok["bad"], ok["disagree"], ok["first_bad"]) == (0, 1, -1)
    no = replay_fn(tr, 0.75 * dist / PK)
    assert (no["bad"], no["disagree"], no["first_bad"]) == (1, 1, t)


def test_replay_near_tie_window_is_tol_times_total():
    J = _J(oracle.GAUSS, 24, 7)
    K, steps = 16, 3000
    d = oracle.run_detail(J, K=K, beta=0.7, seed=19, chain=2, steps=steps)
    ties = _near_ties(d["P"], d["u"], d["own"])
    assert set(ties) == {"above", "below"}
    for side, (t, g, dist) in ties.items():
        _check_near_tie(lambda tr, tol: oracle.replay(J, tr, K=K, beta=0.7, seed=19, chain=2, tol=tol),
                        d["own"], t, g, dist, d["P"][t, -1], d["u"][t])


def test_replay_metropolis_near_tie_window_is_tol():
    J = _J(oracle.GAUSS, 24, 8)
    d = oracle.run_detail(J, rule=oracle.METROPOLIS, beta=1.0, seed=23, chain=0, steps=4000)
    pacc = d["P"][:, 0]
    gap = np.where(pacc < 1.0, np.abs(d["u"] - pacc), np.inf)
    t = int(np.argmin(gap))
    dist = float(gap[t])
    tr = d["own"][: t + 1].copy()
    tr[t] ^= 1
    ok = oracle.replay(J, tr, rule=oracle.METROPOLIS, beta=1.0, seed=23, chain=0, tol=1.5 * dist)
    assert (ok["bad"], ok["disagree"]) == (0, 1)
    no = oracle.replay(J, tr, rule=oracle.METROPOLIS, beta=1.0, seed=23, chain=0, tol=0.75 * dist)
    assert (no["bad"], no["first_bad"]) == (1, t)


GRAPHS = [dict(graph=oracle.TREE, arity=2, depth=3), dict(graph=oracle.LINE, line_nodes=8),
          dict(graph=oracle.TREE, arity=3, depth=2)]


@pytest.mark.parametrize("kind", [oracle.GAUSS, oracle.PM1])
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_graph_replay_of_own_trace_is_clean(kind, gi):
    gk = GRAPHS[gi]
    J = _J(kind, 20, 9)
    r = oracle.run_graph(J, beta=1.0, seed=29, chain0=1, chains=1, steps=800, trace=True, **gk)
    d = oracle.run_graph_detail(J, beta=1.0, seed=29, chain=1, steps=800, **gk)
    assert np.array_equal(d["own"], r["trace"][0])
    if kind == oracle.GAUSS:
        own = np.array([_first_above(d["P"][t], d["u"][t]) for t in range(800)])
        assert np.array_equal(own, d["own"])
    rp = oracle.replay_graph(J, r["trace"][0], beta=1.0, seed=29, chain=1, tol=1e-4, **gk)
    assert (rp["bad"], rp["disagree"], rp["first_bad"]) == (0, 0, -1)
    assert np.array_equal(rp["spins"], r["spins"][0])


def test_graph_replay_flags_a_far_node_at_its_step():
    gk = GRAPHS[0]
    J = _J(oracle.GAUSS, 24, 10)
    d = oracle.run_graph_detail(J, beta=1.0, seed=31, chain=0, steps=300, **gk)
    for t_bad in (5, 200):
        P, u = d["P"][t_bad], d["u"][t_bad]
        g = _far_slot(P, u, 0.05 * P[-1])
        assert g is not None and g != d["own"][t_bad]
        tr = d["own"].copy()
        tr[t_bad] = g
        rp = oracle.replay_graph(J, tr, beta=1.0, seed=31, chain=0, tol=1e-4, **gk)
        assert rp["first_bad"] == t_bad and rp["bad"] >= 1


def test_graph_replay_near_tie_window_is_tol_times_total():
    gk = GRAPHS[0]
    J = _J(oracle.GAUSS, 24, 11)
    d = oracle.run_graph_detail(J, beta=0.5, seed=37, chain=3, steps=3000, **gk)
    ties = _near_ties(d["P"], d["u"], d["own"])
    assert set(ties) == {"above", "below"}
    for side, (t, g, dist) in ties.items():
        _check_near_tie(lambda tr, tol: oracle.replay_graph(J, tr, beta=0.5, seed=37, chain=3, tol=tol, **gk),
                        d["own"], t, g, dist, d["P"][t, -1], d["u"][t])
