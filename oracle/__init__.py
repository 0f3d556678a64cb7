"""FP64 CPU oracle for MCMCMC on the SK spin glass (test infrastructure).

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py use
this package.  It wraps sk_oracle.c (plain C, double precision), which shares
no code with the CUDA path.  Every function cites the part of the paper it
restates; see sk_oracle.c for the algorithm.

Pinned by tests/test_oracle.py against: Philox known-answer vectors, the
closed-form two-node heat-bath rule (Sec. III.A, Eq. eq_node_two_conf), exact
detailed balance and stationarity of enumerated transition matrices
(Sec. A.2, Eq. eq_det_balance_graph_solution), closed forms at beta = 0,
brute-force Boltzmann distributions, and the high-temperature SK energy.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

PM1, GAUSS = 0, 1
MCMCMC, METROPOLIS = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i, d, u32, u64 = C.c_void_p, C.c_int, C.c_double, C.c_uint32, C.c_uint64
        L.sko_philox.argtypes = [vp, vp, vp]
        L.sko_philox.restype = None
        L.sko_energy.argtypes = [i, i, vp, d, vp]
        L.sko_energy.restype = d
        L.sko_fields.argtypes = [i, i, vp, vp, vp]
        L.sko_fields.restype = None
        L.sko_gen_couplings.argtypes = [i, i, u64, vp]
        L.sko_gen_couplings.restype = None
        L.sko_init_spins.argtypes = [u64, u32, u32, i, vp]
        L.sko_init_spins.restype = None
        L.sko_weight_table.argtypes = [d, i, vp]
        L.sko_weight_table.restype = i
        L.sko_run.argtypes = [i, i, vp, d, i, i, d, u64, u32, u32, u32, vp, u64, u32,
                              vp, vp, vp, vp, vp, vp, u32]
        L.sko_run.restype = i
        L.sko_run_p.argtypes = L.sko_run.argtypes + [d, vp]
        L.sko_run_p.restype = i
        L.sko_replay.argtypes = [i, i, vp, d, i, i, d, u64, u32, u32, vp, u64, vp, d,
                                 vp, vp, vp, vp]
        L.sko_replay.restype = C.c_longlong
        L.sko_replay_p.argtypes = L.sko_replay.argtypes + [d]
        L.sko_replay_p.restype = C.c_longlong
        L.sko_boltzmann.argtypes = [i, i, vp, d, d, vp]
        L.sko_boltzmann.restype = i
        L.sko_transition_matrix.argtypes = [i, i, vp, d, i, i, d, i, i, vp]
        L.sko_transition_matrix.restype = i
        L.sko_transition_matrix_p.argtypes = [i, i, vp, d, i, i, d, i, i, d, vp]
        L.sko_transition_matrix_p.restype = i
        L.sko_run_graph.argtypes = [i, i, vp, d, i, i, i, i, d, u64, u32, u32, u32, vp, u64, u32,
                                    vp, vp, vp, vp, vp]
        L.sko_run_graph.restype = i
        L.sko_replay_graph.argtypes = [i, i, vp, d, i, i, i, i, d, u64, u32, u32, vp, u64, vp, d,
                                       vp, vp, vp, vp]
        L.sko_replay_graph.restype = C.c_longlong
        L.sko_run_detail.argtypes = [i, i, vp, d, i, i, d, u64, u32, u32, vp, u64, d, vp, vp, vp]
        L.sko_run_detail.restype = i
        L.sko_run_graph_detail.argtypes = [i, i, vp, d, i, i, i, i, d, u64, u32, u32, vp, u64, vp, vp, vp]
        L.sko_run_graph_detail.restype = i
        L.sko_transition_matrix_graph.argtypes = [i, i, vp, d, i, i, i, i, d, i, i, vp]
        L.sko_transition_matrix_graph.restype = i
        L.sko_setgen_bruteforce.argtypes = [i, vp, u32]
        L.sko_setgen_bruteforce.restype = d
        L.sko_setgen_dp.argtypes = [i, vp, vp]
        L.sko_setgen_dp.restype = i
        L.sko_setgen_cumulative.argtypes = [i, vp, vp]
        L.sko_setgen_cumulative.restype = i
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _kind_of(J: np.ndarray) -> int:
    if J.dtype == np.int8:
        return PM1
    if J.dtype == np.float32:
        return GAUSS
    raise TypeError("couplings must be int8 (+-J) or float32 (Gaussian)")


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().sko_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def energy(J: np.ndarray, s: np.ndarray, scale: float = 1.0) -> float:
    """E = -scale sum_{i<j} J_ij s_i s_j (Sec. IV.A, sign convention J -> -J)."""
    J = np.ascontiguousarray(J)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return lib().sko_energy(J.shape[0], _kind_of(J), _ptr(J), scale, _ptr(s))


def fields(J: np.ndarray, s: np.ndarray) -> np.ndarray:
    J = np.ascontiguousarray(J)
    s = np.ascontiguousarray(s, dtype=np.int8)
    h = np.zeros(J.shape[0])
    lib().sko_fields(J.shape[0], _kind_of(J), _ptr(J), _ptr(s), _ptr(h))
    return h


def gen_couplings(N: int, kind: int, seed: int) -> np.ndarray:
    """Couplings drawn from a seed by Philox domain 2 (+-1 bits, or the
    Box-Muller N(0, 1/N) normal rounded to float32); see sko_gen_couplings."""
    out = np.zeros((N, N), dtype=np.int8 if kind == PM1 else np.float32)
    lib().sko_gen_couplings(N, kind, seed, _ptr(out))
    return out


def init_spins(seed: int, stream: int, chain: int, N: int) -> np.ndarray:
    s = np.zeros(N, dtype=np.int8)
    lib().sko_init_spins(seed, stream, chain, N, _ptr(s))
    return s


def weight_table(beta_eff: float, dmax: int) -> np.ndarray:
    W = np.zeros(dmax + 1, dtype=np.uint64)
    n = lib().sko_weight_table(beta_eff, dmax, _ptr(W))
    return W[:n]


def run(J, *, rule=MCMCMC, K=8, beta=1.0, scale=1.0, seed=1, stream=0, chain0=0,
        chains=1, init=None, steps=100, record_every=0, trace=False, resync_every=0,
        want_q=True, p_center=0.0):
    """Runs chains chain0..chain0+chains-1 for `steps` steps (see sko_run_p;
    p_center = 0 is the uniform root)."""
    J = np.ascontiguousarray(J)
    N = J.shape[0]
    nrec = steps // record_every if record_every else 0
    E = np.zeros((nrec, chains))
    Enw = np.zeros((nrec, chains))
    acc = np.zeros((nrec, chains), dtype=np.uint32)
    q = np.zeros((nrec, chains // 2)) if (want_q and chains >= 2) else None
    fin = np.zeros((chains, N), dtype=np.int8)
    finE = np.zeros(chains)
    tr = np.zeros((chains, steps), dtype=np.int32) if trace else None
    init_a = None if init is None else np.ascontiguousarray(init, dtype=np.int8).reshape(chains, N)
    rc = lib().sko_run_p(N, _kind_of(J), _ptr(J), scale, rule, K, beta, seed, stream, chain0,
                         chains, _ptr(init_a), steps, record_every, _ptr(E), _ptr(acc), _ptr(q),
                         _ptr(fin), _ptr(finE), _ptr(tr), resync_every, float(p_center), _ptr(Enw))
    if rc != 0:
        raise RuntimeError(f"sko_run failed with {rc}")
    return dict(E=E, acc=acc, q=q, spins=fin, final_E=finE, trace=tr, E_nw=Enw)


def replay(J, slots, *, rule=MCMCMC, K=8, beta=1.0, scale=1.0, seed=1, stream=0, chain=0,
           init=None, tol=1e-4, p_center=0.0):
    """Follows a slot sequence chosen elsewhere and counts inadmissible steps
    (see sko_replay)."""
    J = np.ascontiguousarray(J)
    N = J.shape[0]
    sl = np.ascontiguousarray(slots, dtype=np.int32)
    dis = C.c_longlong(0)
    first = C.c_longlong(-1)
    fin = np.zeros(N, dtype=np.int8)
    finE = C.c_double(0.0)
    init_a = None if init is None else np.ascontiguousarray(init, dtype=np.int8)
    bad = lib().sko_replay_p(N, _kind_of(J), _ptr(J), scale, rule, K, beta, seed, stream, chain,
                             _ptr(init_a), len(sl), _ptr(sl), tol, C.byref(dis), C.byref(first),
                             _ptr(fin), C.byref(finE), float(p_center))
    if bad < 0:
        raise RuntimeError(f"sko_replay failed with {bad}")
    return dict(bad=int(bad), disagree=int(dis.value), first_bad=int(first.value),
                spins=fin, final_E=finE.value)


def run_detail(J, *, rule=MCMCMC, K=8, beta=1.0, scale=1.0, seed=1, stream=0, chain=0, init=None,
               steps=100, p_center=0.0):
    """One chain's own trajectory with each step's choice, draw u and
    inclusive prefix sums P of the slot weights (Metropolis: P = the
    acceptance probability), see sko_run_detail."""
    J = np.ascontiguousarray(J)
    N = J.shape[0]
    stride = 1 if rule == METROPOLIS else K + 1
    own = np.zeros(steps, dtype=np.int32)
    u = np.zeros(steps)
    P = np.zeros((steps, stride))
    init_a = None if init is None else np.ascontiguousarray(init, dtype=np.int8)
    rc = lib().sko_run_detail(N, _kind_of(J), _ptr(J), scale, rule, K, beta, seed, stream, chain,
                              _ptr(init_a), steps, float(p_center), _ptr(own), _ptr(u), _ptr(P))
    if rc != 0:
        raise RuntimeError(f"sko_run_detail failed with {rc}")
    return dict(own=own, u=u, P=P)


def boltzmann(J, beta, scale=1.0) -> np.ndarray:
    """Exact P_eq over all 2^N states (state bit i set <=> s_i = -1)."""
    J = np.ascontiguousarray(J)
    N = J.shape[0]
    pi = np.zeros(1 << N)
    if lib().sko_boltzmann(N, _kind_of(J), _ptr(J), scale, beta, _ptr(pi)) != 0:
        raise ValueError("N too large for enumeration")
    return pi


def transition_matrix(J, *, rule=MCMCMC, K=2, beta=1.0, scale=1.0, root_mode=0,
                      weight_mode=0, p_center=0.0) -> np.ndarray:
    """Exact one-step transition matrix by enumeration (small N, K <= 8);
    root_mode 0 the method (uniform root, or the centre with probability
    p_center and root-weighted slots), 1 always the centre, 2 the centre with
    probability p_center but no root weights (see sko_transition_matrix_p)."""
    J = np.ascontiguousarray(J)
    N = J.shape[0]
    P = np.zeros((1 << N, 1 << N))
    rc = lib().sko_transition_matrix_p(N, _kind_of(J), _ptr(J), scale, rule, K, beta, root_mode,
                                       weight_mode, float(p_center), _ptr(P))
    if rc != 0:
        raise ValueError(f"transition_matrix failed with {rc}")
    return P


TREE, LINE = 1, 2


def graph_nodes(graph, arity=2, depth=1, line_nodes=2):
    """Nodes of a template: (k^(D+1)-1)/(k-1) for the k-ary tree, L for the line."""
    if graph == TREE:
        return (arity ** (depth + 1) - 1) // (arity - 1)
    return line_nodes


def run_graph(J, *, graph=TREE, arity=2, depth=1, line_nodes=2, beta=1.0, scale=1.0, seed=1, stream=0,
              chain0=0, chains=1, init=None, steps=100, record_every=0, trace=False):
    """MCMCMC on a k-ary tree (uniform root) or a line (binomial root); see sko_run_graph."""
    J = np.ascontiguousarray(J)
    N = J.shape[0]
    nrec = steps // record_every if record_every else 0
    E = np.zeros((nrec, chains))
    acc = np.zeros((nrec, chains), dtype=np.uint32)
    fin = np.zeros((chains, N), dtype=np.int8)
    finE = np.zeros(chains)
    tr = np.zeros((chains, steps), dtype=np.int32) if trace else None
    init_a = None if init is None else np.ascontiguousarray(init, dtype=np.int8).reshape(chains, N)
    rc = lib().sko_run_graph(N, _kind_of(J), _ptr(J), scale, graph, arity, depth, line_nodes, beta, seed,
                             stream, chain0, chains, _ptr(init_a), steps, record_every, _ptr(E), _ptr(acc),
                             _ptr(fin), _ptr(finE), _ptr(tr))
    if rc != 0:
        raise RuntimeError(f"sko_run_graph failed with {rc}")
    return dict(E=E, acc=acc, spins=fin, final_E=finE, trace=tr)


def replay_graph(J, slots, *, graph=TREE, arity=2, depth=1, line_nodes=2, beta=1.0, scale=1.0, seed=1,
                 stream=0, chain=0, init=None, tol=1e-4):
    J = np.ascontiguousarray(J)
    N = J.shape[0]
    sl = np.ascontiguousarray(slots, dtype=np.int32)
    dis = C.c_longlong(0)
    first = C.c_longlong(-1)
    fin = np.zeros(N, dtype=np.int8)
    finE = C.c_double(0.0)
    init_a = None if init is None else np.ascontiguousarray(init, dtype=np.int8)
    bad = lib().sko_replay_graph(N, _kind_of(J), _ptr(J), scale, graph, arity, depth, line_nodes, beta, seed,
                                 stream, chain, _ptr(init_a), len(sl), _ptr(sl), tol, C.byref(dis),
                                 C.byref(first), _ptr(fin), C.byref(finE))
    if bad < 0:
        raise RuntimeError(f"sko_replay_graph failed with {bad}")
    return dict(bad=int(bad), disagree=int(dis.value), first_bad=int(first.value), spins=fin,
                final_E=finE.value)


def run_graph_detail(J, *, graph=TREE, arity=2, depth=1, line_nodes=2, beta=1.0, scale=1.0, seed=1,
                     stream=0, chain=0, init=None, steps=100):
    """run_detail on a graph: P has one column per node."""
    J = np.ascontiguousarray(J)
    N = J.shape[0]
    V = graph_nodes(graph, arity, depth, line_nodes)
    own = np.zeros(steps, dtype=np.int32)
    u = np.zeros(steps)
    P = np.zeros((steps, V))
    init_a = None if init is None else np.ascontiguousarray(init, dtype=np.int8)
    rc = lib().sko_run_graph_detail(N, _kind_of(J), _ptr(J), scale, graph, arity, depth, line_nodes, beta,
                                    seed, stream, chain, _ptr(init_a), steps, _ptr(own), _ptr(u), _ptr(P))
    if rc != 0:
        raise RuntimeError(f"sko_run_graph_detail failed with {rc}")
    return dict(own=own, u=u, P=P)


def transition_matrix_graph(J, *, graph=TREE, arity=2, depth=1, line_nodes=2, beta=1.0, scale=1.0,
                            weight_mode=0, root_weights=1) -> np.ndarray:
    """Exact one-step transition matrix on a graph by enumeration (N <= 10, <= 8 nodes)."""
    J = np.ascontiguousarray(J)
    N = J.shape[0]
    P = np.zeros((1 << N, 1 << N))
    rc = lib().sko_transition_matrix_graph(N, _kind_of(J), _ptr(J), scale, graph, arity, depth, line_nodes,
                                           beta, weight_mode, root_weights, _ptr(P))
    if rc != 0:
        raise ValueError(f"transition_matrix_graph failed with {rc}")
    return P


def setgen_bruteforce(P, M: int) -> float:
    """P_gen(S | S minus M) by enumerating the orders of M's elements (n <= 12)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    return lib().sko_setgen_bruteforce(P.shape[0], _ptr(P), int(M))


def setgen_cumulative(P) -> np.ndarray:
    """The same probabilities by the paper's cumulative form (O(n 2^n), n <= 20)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    n = P.shape[0]
    out = np.zeros(1 << n)
    if lib().sko_setgen_cumulative(n, _ptr(P), _ptr(out)) != 0:
        raise ValueError("n outside 1..20")
    return out


def setgen_dp(P) -> np.ndarray:
    """P_gen(S | S minus M) for every mask M by the first-addition recursion (n <= 26)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    n = P.shape[0]
    out = np.zeros(1 << n)
    if lib().sko_setgen_dp(n, _ptr(P), _ptr(out)) != 0:
        raise ValueError("n outside 1..26")
    return out
