"""Thin ctypes binding of the sampler's C ABI (include/sk_mcmcmc.h).

Argument marshalling only: every step of the sampler runs in the CUDA
library.  The functions keep the C names; small classes wrap the opaque
handles.  Inputs may be numpy arrays (host) or torch CUDA tensors (device,
passed by pointer); outputs come back as numpy arrays unless a device
tensor is supplied.  Loading fails loudly when the library has not been
built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

from . import build as _build

(SK_OK, SK_ERR_INVALID_ARG, SK_ERR_OOM, SK_ERR_CUDA, SK_ERR_TIMEOUT, SK_ERR_NOT_READY, SK_ERR_DEVICE,
 SK_ERR_BUSY, SK_ERR_CANCELLED) = range(9)
SK_J_PM1, SK_J_GAUSS = 0, 1
SK_RULE_MCMCMC, SK_RULE_METROPOLIS = 0, 1
SK_MEM_HOST, SK_MEM_DEVICE = 0, 1
SK_MAX_K, SK_MAX_N = 256, 8192

_STATUS = {0: "SK_OK", 1: "SK_ERR_INVALID_ARG", 2: "SK_ERR_OOM", 3: "SK_ERR_CUDA",
           4: "SK_ERR_TIMEOUT", 5: "SK_ERR_NOT_READY", 6: "SK_ERR_DEVICE", 7: "SK_ERR_BUSY",
           8: "SK_ERR_CANCELLED"}

# every symbol declared in include/sk_mcmcmc.h
EXPORTS = ["sk_create_instance", "sk_get_couplings", "sk_set_couplings", "sk_destroy_instance", "sk_energy",
           "mcmcmc_create", "mcmcmc_advance", "mcmcmc_run", "mcmcmc_reset", "mcmcmc_wait",
           "mcmcmc_observables", "mcmcmc_observables_nw", "mcmcmc_state", "mcmcmc_recompute", "mcmcmc_recompute_stats",
           "mcmcmc_trace", "mcmcmc_counters", "mcmcmc_free",
           "mcmcmc_batch_create", "mcmcmc_batch_advance", "mcmcmc_batch_capture",
           "mcmcmc_batch_replay", "mcmcmc_batch_autotune", "mcmcmc_batch_info",
           "mcmcmc_batch_classes", "mcmcmc_batch_set_layout", "mcmcmc_batch_set_cluster",
           "mcmcmc_batch_set_fused",
           "mcmcmc_batch_free", "mcmcmc_run_noalloc", "sk_last_error",
           "sk_peak_l2_read", "sk_peak_smem", "sk_peak_tensor"]


class SKError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class RunParams(C.Structure):
    _fields_ = [("chains", C.c_uint32), ("K", C.c_uint32), ("rule", C.c_uint32),
                ("record_every", C.c_uint32), ("max_records", C.c_uint64),
                ("beta", C.c_double), ("seed", C.c_uint64), ("stream_id", C.c_uint32),
                ("trace_chains", C.c_uint32), ("trace_steps", C.c_uint64),
                ("init_spins", C.c_void_p), ("init_mem", C.c_uint32),
                ("recompute_every", C.c_uint32), ("recompute_terms", C.c_uint32),
                ("p_center", C.c_double), ("node_weighted", C.c_uint32), ("graph", C.c_uint32),
                ("arity", C.c_uint32), ("depth", C.c_uint32), ("line_nodes", C.c_uint32),
                ("fault_inject", C.c_uint32)]


class RecomputeStats(C.Structure):
    _fields_ = [("max_field_drift", C.c_double), ("max_energy_drift", C.c_double),
                ("mismatches", C.c_uint64), ("recomputes", C.c_uint64)]


SK_RECOMPUTE_CHECK, SK_RECOMPUTE_RESYNC, SK_RECOMPUTE_OUTPUT = 0, 1, 2
SK_FAULT_WITHHOLD_ROW, SK_FAULT_WITHHOLD_TILE = 1, 2
SK_GRAPH_STAR, SK_GRAPH_TREE, SK_GRAPH_LINE = 0, 1, 2


_lib = None


def lib(build_if_missing: bool = True):
    """The loaded CUDA library; builds it in-tree if it is missing."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA sampler library not built ({path}); run build() first")
        L = C.CDLL(path)
        vp, u32, u64, d = C.c_void_p, C.c_uint32, C.c_uint64, C.c_double
        P = C.POINTER(C.c_void_p)
        sig = {
            "sk_create_instance": [u32, u32, vp, u32, u64, d, vp, P],
            "sk_get_couplings": [vp, vp, u32],
            "sk_set_couplings": [vp, vp, u32],
            "sk_destroy_instance": [vp],
            "sk_energy": [vp, vp, u32, u32, vp],
            "mcmcmc_create": [vp, C.POINTER(RunParams), P],
            "mcmcmc_advance": [vp, u64],
            "mcmcmc_run": [vp, C.POINTER(RunParams), u64, P],
            "mcmcmc_reset": [vp, vp, u32],
            "mcmcmc_wait": [vp, u64],
            "mcmcmc_observables": [vp, u64, u64, vp, vp, vp, u32],
            "mcmcmc_observables_nw": [vp, u64, u64, vp, u32],
            "sk_set_generation": [u32, vp, vp, u32, u32, vp],
            "sk_set_couplings_many": [vp, u32, vp, u32],
            "mcmcmc_reset_many": [vp, u32, vp, u32],
            "mcmcmc_observables_many": [vp, u32, u64, u64, vp, vp, vp, u32],
            "mcmcmc_state": [vp, vp, vp, vp, u32],
            "mcmcmc_trace": [vp, vp, u32],
            "mcmcmc_counters": [vp, vp, vp],
            "mcmcmc_recompute": [vp, u32, u32, C.POINTER(RecomputeStats), vp, u32],
            "mcmcmc_recompute_stats": [vp, C.POINTER(RecomputeStats)],
            "mcmcmc_free": [vp],
            "mcmcmc_batch_create": [P, u32, u32, P],
            "mcmcmc_batch_advance": [vp, u64],
            "mcmcmc_batch_capture": [vp, u64],
            "mcmcmc_batch_replay": [vp, u32],
            "mcmcmc_batch_autotune": [vp, u32, vp],
            "mcmcmc_batch_classes": [vp, u32, vp, vp],
            "mcmcmc_batch_set_layout": [vp, u32, u32],
            "mcmcmc_batch_set_cluster": [vp, u32, u32],
            "mcmcmc_batch_set_fused": [vp, u32],
            "mcmcmc_batch_info": [vp, vp, vp, vp, vp],
            "mcmcmc_batch_free": [vp],
            "mcmcmc_run_noalloc": [u32, u32, vp, d, u32, u32, u32, d, u64, u32, u64, vp, vp, vp],
            "sk_peak_l2_read": [u64, u32, u32, vp, C.POINTER(d)],
            "sk_peak_smem": [u32, u32, u32, vp, C.POINTER(d)],
            "sk_peak_tensor": [u32, u32, u32, vp, C.POINTER(d)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.sk_last_error.argtypes = []
        L.sk_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(status):
    if status != SK_OK:
        raise SKError(status, lib().sk_last_error().decode())


def _ptr_mem(a):
    """(pointer, mem) of a numpy array or a torch tensor."""
    if a is None:
        return None, SK_MEM_HOST
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p), SK_MEM_HOST
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr()), (SK_MEM_DEVICE if a.is_cuda else SK_MEM_HOST)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


class Instance:
    """sk_create_instance / sk_destroy_instance (couplings resident on the GPU)."""

    def __init__(self, J, scale: float = 1.0, stream=None, *, N: int = 0, kind: int = SK_J_GAUSS, seed: int = 0):
        """J: the couplings (numpy host array or torch CUDA tensor, int8 for
        +-J, float32 for Gaussian), or None to draw N spins' couplings of
        `kind` on the device from `seed` (see sk_create_instance)."""
        if J is None:
            if not 2 <= int(N) <= SK_MAX_N or kind not in (SK_J_PM1, SK_J_GAUSS):
                raise ValueError("drawn couplings need 2 <= N <= SK_MAX_N and a coupling kind")
            self.kind, self.N = int(kind), int(N)
            p, mem = None, SK_MEM_HOST
        else:
            if isinstance(J, np.ndarray):
                J = np.ascontiguousarray(J)
                dt = J.dtype
            else:
                dt = {"torch.int8": np.int8, "torch.float32": np.float32}[str(J.dtype)]
            if dt == np.int8:
                self.kind = SK_J_PM1
            elif dt == np.float32:
                self.kind = SK_J_GAUSS
            else:
                raise TypeError("couplings must be int8 (+-J) or float32 (Gaussian)")
            self.N = int(J.shape[0])
            p, mem = _ptr_mem(J)
        self.scale = float(scale)
        self._stream = stream
        h = C.c_void_p()
        _check(lib().sk_create_instance(self.N, self.kind, p, mem, int(seed), self.scale,
                                        _stream_handle(stream), C.byref(h)))
        self.handle = h

    def couplings(self) -> np.ndarray:
        """sk_get_couplings: the N x N couplings as a host array."""
        out = np.zeros((self.N, self.N), dtype=np.int8 if self.kind == SK_J_PM1 else np.float32)
        _check(lib().sk_get_couplings(self.handle, out.ctypes.data_as(C.c_void_p), SK_MEM_HOST))
        return out

    def set_couplings(self, J):
        p, mem = _ptr_mem(J if not isinstance(J, np.ndarray) else np.ascontiguousarray(J))
        _check(lib().sk_set_couplings(self.handle, p, mem))

    def energy(self, spins) -> np.ndarray:
        if isinstance(spins, np.ndarray):
            spins = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1, self.N)
            count = spins.shape[0]
        else:
            count = spins.numel() // self.N
        out = np.zeros(count)
        p, mem = _ptr_mem(spins)
        _check(lib().sk_energy(self.handle, p, count, mem, out.ctypes.data_as(C.c_void_p)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().sk_destroy_instance(self.handle))
            self.handle = None

    def __del__(self):
        # at interpreter exit the order in which objects (and the CUDA
        # runtime) are torn down is not defined: leave the memory to the
        # process exit rather than call into the library then
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Run:
    """mcmcmc_create / advance / observables / state / free."""

    def __init__(self, inst: Instance, *, chains: int, K: int = 8, rule: int = SK_RULE_MCMCMC,
                 beta: float = 1.0, seed: int = 1, stream_id: int = 0, record_every: int = 0,
                 max_records: int = 0, init=None, trace_chains: int = 0, trace_steps: int = 0,
                 recompute_every: int = 0, recompute_terms: int = 0, p_center: float = 0.0,
                 node_weighted: bool = False, graph: int = 0, arity: int = 0, depth: int = 0,
                 line_nodes: int = 0, fault_inject: int = 0):
        self.inst = inst
        self.chains, self.K, self.rule = int(chains), int(K), int(rule)
        self.record_every, self.max_records = int(record_every), int(max_records)
        self.trace_chains, self.trace_steps = int(trace_chains), int(trace_steps)
        self._init = None
        pr = RunParams()
        pr.chains, pr.K, pr.rule = self.chains, self.K, self.rule
        pr.record_every, pr.max_records = self.record_every, self.max_records
        pr.beta, pr.seed, pr.stream_id = float(beta), int(seed), int(stream_id)
        pr.trace_chains, pr.trace_steps = self.trace_chains, self.trace_steps
        pr.recompute_every, pr.recompute_terms = int(recompute_every), int(recompute_terms)
        pr.p_center = float(p_center)
        pr.node_weighted = 1 if node_weighted else 0
        pr.graph, pr.arity, pr.depth, pr.line_nodes = int(graph), int(arity), int(depth), int(line_nodes)
        pr.fault_inject = int(fault_inject)
        if init is not None:
            if isinstance(init, np.ndarray):
                init = np.ascontiguousarray(init, dtype=np.int8)
            self._init = init
            p, mem = _ptr_mem(init)
            pr.init_spins, pr.init_mem = p, mem
        h = C.c_void_p()
        _check(lib().mcmcmc_create(inst.handle, C.byref(pr), C.byref(h)))
        self.handle = h

    def advance(self, steps: int):
        _check(lib().mcmcmc_advance(self.handle, int(steps)))

    def reset(self, spins=None):
        if isinstance(spins, np.ndarray):
            spins = np.ascontiguousarray(spins, dtype=np.int8)
        p, mem = _ptr_mem(spins)
        _check(lib().mcmcmc_reset(self.handle, p, mem))

    def wait(self, timeout_ns: int = 0):
        _check(lib().mcmcmc_wait(self.handle, int(timeout_ns)))

    def observables(self, first: int = 0, count=None, out=None):
        if count is None:
            count = self.max_records - first
        C_ = self.chains
        if out is None:
            E = np.zeros((count, C_))
            q = np.zeros((count, C_ // 2))
            acc = np.zeros((count, C_), dtype=np.uint32)
            mem = SK_MEM_HOST
            ptrs = [x.ctypes.data_as(C.c_void_p) for x in (E, q, acc)]
        else:
            E, q, acc = out
            mem = SK_MEM_DEVICE if getattr(E, "is_cuda", False) else SK_MEM_HOST
            ptrs = [_ptr_mem(x)[0] for x in (E, q, acc)]
        _check(lib().mcmcmc_observables(self.handle, first, count, ptrs[0], ptrs[1], ptrs[2], mem))
        return E, q, acc

    def observables_nw(self, first: int = 0, count=None):
        """Node-weighted energies of records [first, first+count) (mcmcmc_observables_nw)."""
        if count is None:
            count = self.max_records - first
        E = np.zeros((count, self.chains))
        _check(lib().mcmcmc_observables_nw(self.handle, first, count, E.ctypes.data_as(C.c_void_p), SK_MEM_HOST))
        return E

    def state(self, fields: bool = False):
        N = self.inst.N
        s = np.zeros((self.chains, N), dtype=np.int8)
        h = None
        if fields:
            h = np.zeros((self.chains, N), dtype=np.int32 if self.inst.kind == SK_J_PM1 else np.float32)
        step = C.c_uint64(0)
        _check(lib().mcmcmc_state(self.handle, s.ctypes.data_as(C.c_void_p),
                                  None if h is None else h.ctypes.data_as(C.c_void_p),
                                  C.byref(step), SK_MEM_HOST))
        return (s, h, step.value) if fields else (s, step.value)

    def trace(self) -> np.ndarray:
        t = np.zeros((self.trace_chains, self.trace_steps), dtype=np.int32)
        _check(lib().mcmcmc_trace(self.handle, t.ctypes.data_as(C.c_void_p), SK_MEM_HOST))
        return t

    def recompute(self, mode: int = SK_RECOMPUTE_CHECK, terms: int = 3, out: bool = False,
                  sync: bool = True):
        """mcmcmc_recompute; returns (stats dict, H or None).  sync=False only
        enqueues (no stats)."""
        if not sync and not out:
            _check(lib().mcmcmc_recompute(self.handle, int(mode), int(terms), None, None,
                                          SK_MEM_HOST))
            return None, None
        st = RecomputeStats()
        H = None
        ptr = None
        if out:
            mode = SK_RECOMPUTE_OUTPUT
            H = np.zeros((self.chains, self.inst.N), dtype=np.float32)
            ptr = H.ctypes.data_as(C.c_void_p)
        _check(lib().mcmcmc_recompute(self.handle, int(mode), int(terms), C.byref(st), ptr, SK_MEM_HOST))
        return ({k: getattr(st, k) for k, _ in RecomputeStats._fields_}, H)

    def recompute_stats(self):
        st = RecomputeStats()
        _check(lib().mcmcmc_recompute_stats(self.handle, C.byref(st)))
        return {k: getattr(st, k) for k, _ in RecomputeStats._fields_}

    def counters(self):
        """(spins flipped, J rows needed) since the last reset."""
        f, r = C.c_uint64(0), C.c_uint64(0)
        _check(lib().mcmcmc_counters(self.handle, C.byref(f), C.byref(r)))
        return f.value, r.value

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().mcmcmc_free(self.handle))
            self.handle = None

    def __del__(self):
        # at interpreter exit the order in which objects (and the CUDA
        # runtime) are torn down is not defined: leave the memory to the
        # process exit rather than call into the library then
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """mcmcmc_batch_create / advance / free: many runs, one persistent launch."""

    def __init__(self, runs, warps_per_cta: int = 0):
        self.runs = list(runs)
        arr = (C.c_void_p * len(self.runs))(*[r.handle.value for r in self.runs])
        h = C.c_void_p()
        _check(lib().mcmcmc_batch_create(C.cast(arr, C.POINTER(C.c_void_p)), len(self.runs),
                                         int(warps_per_cta), C.byref(h)))
        self.handle = h

    def advance(self, steps: int):
        _check(lib().mcmcmc_batch_advance(self.handle, int(steps)))

    def capture(self, steps: int):
        _check(lib().mcmcmc_batch_capture(self.handle, int(steps)))

    def replay(self, times: int = 1):
        _check(lib().mcmcmc_batch_replay(self.handle, int(times)))

    def autotune(self, trial_steps: int = 20) -> int:
        w = C.c_uint32(0)
        _check(lib().mcmcmc_batch_autotune(self.handle, int(trial_steps), C.byref(w)))
        return w.value

    def classes(self):
        """[(kernel class, lanes per chain, shared bytes per chain, warps per CTA, items, CTAs)]"""
        n = C.c_uint32(0)
        _check(lib().mcmcmc_batch_classes(self.handle, 0, C.byref(n), None))
        d = np.zeros(6 * max(n.value, 1), dtype=np.uint32)
        _check(lib().mcmcmc_batch_classes(self.handle, n.value, C.byref(n),
                                          d.ctypes.data_as(C.c_void_p)))
        return [tuple(int(x) for x in d[6 * k:6 * k + 6]) for k in range(n.value)]

    def set_layout(self, lanes: int = 0, staging: int = 0):
        """mcmcmc_batch_set_layout: lanes per chain (0, 4, 8, 16, 32; graph
        runs also 64, 128, 256, 512 = 2..16 warps per chain; star runs 64 or
        128 = the team layout of 2 or 4 warps per chain, one slot per
        thread); staging 0 default, 1 TMA-staged rows, 2 rows read through
        L1."""
        _check(lib().mcmcmc_batch_set_layout(self.handle, int(lanes), int(staging)))

    def set_cluster(self, ctas: int, chains: int = 0):
        """mcmcmc_batch_set_cluster: the cluster-per-chain layout with `ctas`
        CTAs per cluster (1, 2, 4, 8, 16; 0 = back to the warp layouts) and
        `chains` chains per cluster (0 default, 1, 2, 4, 8), for every star
        class that can take it."""
        _check(lib().mcmcmc_batch_set_cluster(self.handle, int(ctas), int(chains)))

    def set_fused(self, warps_per_cta: int):
        """mcmcmc_batch_set_fused: every star run in one persistent launch of
        warps_per_cta (2, 4, 8, 16) warps per CTA; 0 = one launch per class."""
        _check(lib().mcmcmc_batch_set_fused(self.handle, int(warps_per_cta)))

    def info(self):
        v = [C.c_uint32(0) for _ in range(4)]
        _check(lib().mcmcmc_batch_info(self.handle, *[C.byref(x) for x in v]))
        return dict(grid=v[0].value, warps_per_cta=v[1].value, smem_bytes=v[2].value,
                    items=v[3].value)

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().mcmcmc_batch_free(self.handle))
            self.handle = None

    def __del__(self):
        # at interpreter exit the order in which objects (and the CUDA
        # runtime) are torn down is not defined: leave the memory to the
        # process exit rather than call into the library then
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def run_noalloc(couplings, spins, energy, *, scale=1.0, K=8, rule=SK_RULE_MCMCMC, beta=1.0,
                seed=1, stream_id=0, steps=0, stream=None):
    """mcmcmc_run_noalloc: device couplings (N x N torch tensor, int8 or
    float32), device spins (chains x N int8, updated in place) and a device
    float64 energy vector (chains), all owned by the caller.  The buffers are
    checked here (type, shape, contiguity, one CUDA device) before the C call,
    which trusts the pointers it is given: TypeError or ValueError otherwise."""
    for name, t in (("couplings", couplings), ("spins", spins), ("energy", energy)):
        if not all(hasattr(t, a) for a in ("data_ptr", "dtype", "shape", "is_contiguous", "device")):
            raise TypeError(f"{name} must be a torch tensor")
    kinds = {"torch.int8": SK_J_PM1, "torch.float32": SK_J_GAUSS}
    if str(couplings.dtype) not in kinds:
        raise TypeError("couplings must be int8 (+-J) or float32 (Gaussian)")
    if str(spins.dtype) != "torch.int8":
        raise TypeError("spins must be int8")
    if str(energy.dtype) != "torch.float64":
        raise TypeError("energy must be float64")
    if couplings.dim() != 2 or couplings.shape[0] != couplings.shape[1]:
        raise ValueError(f"couplings must be a square matrix, got shape {tuple(couplings.shape)}")
    N = int(couplings.shape[0])
    if spins.dim() != 2 or spins.shape[1] != N or spins.shape[0] < 1:
        raise ValueError(f"spins must have shape (chains, {N}), got {tuple(spins.shape)}")
    chains = int(spins.shape[0])
    if energy.numel() != chains:
        raise ValueError(f"energy must hold {chains} values, got {energy.numel()}")
    for name, t in (("couplings", couplings), ("spins", spins), ("energy", energy)):
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    devs = {str(t.device) for t in (couplings, spins, energy)}
    if any(not t.is_cuda for t in (couplings, spins, energy)) or len(devs) != 1:
        raise ValueError(f"couplings, spins and energy must be on one CUDA device, got {sorted(devs)}")
    import torch
    if couplings.device.index != torch.cuda.current_device():
        raise ValueError(f"the buffers are on {couplings.device}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    kind = kinds[str(couplings.dtype)]
    _check(lib().mcmcmc_run_noalloc(N, kind, C.c_void_p(couplings.data_ptr()), float(scale), chains,
                                    int(K), int(rule), float(beta), int(seed), int(stream_id),
                                    int(steps), C.c_void_p(spins.data_ptr()),
                                    C.c_void_p(energy.data_ptr()), _stream_handle(stream)))


# ---------------------------------------------------------------------------
# measured memory ceilings (sk_peaks.h)
# ---------------------------------------------------------------------------
SK_PEAK_SMEM_VEC16, SK_PEAK_SMEM_GATHER4 = 0, 1


def peak_l2_read(working_set_bytes: int = 48 << 20, passes: int = 8, reps: int = 5, stream=None) -> float:
    """sk_peak_l2_read: L2 read bandwidth (GB/s) on a resident working set."""
    out = C.c_double(0.0)
    _check(lib().sk_peak_l2_read(int(working_set_bytes), int(passes), int(reps), _stream_handle(stream),
                                 C.byref(out)))
    return out.value


def peak_smem(mode: int = SK_PEAK_SMEM_VEC16, iters: int = 4096, reps: int = 5, stream=None) -> float:
    """sk_peak_smem: shared-memory load bandwidth (GB/s), conflict-free 16-byte
    loads or random 4-byte gathers (useful bytes)."""
    out = C.c_double(0.0)
    _check(lib().sk_peak_smem(int(mode), int(iters), int(reps), _stream_handle(stream), C.byref(out)))
    return out.value


def peak_tensor(kind: int = SK_J_PM1, tiles: int = 64, reps: int = 5, stream=None) -> float:
    """sk_peak_tensor: TFLOP/s of the recompute kernel's own tcgen05 MMA loop
    with its operand ring filled once (kind 0: FP8 e4m3, 1: bf16)."""
    out = C.c_double(0.0)
    _check(lib().sk_peak_tensor(int(kind), int(tiles), int(reps), _stream_handle(stream), C.byref(out)))
    return out.value


# ---------------------------------------------------------------------------
# request server
# ---------------------------------------------------------------------------
class Job(C.Structure):
    _fields_ = [("N", C.c_uint32), ("kind", C.c_uint32), ("couplings", C.c_void_p),
                ("couplings_id", C.c_uint64), ("scale", C.c_double), ("chains", C.c_uint32),
                ("K", C.c_uint32), ("rule", C.c_uint32), ("beta", C.c_double), ("seed", C.c_uint64),
                ("stream_id", C.c_uint32), ("steps", C.c_uint64), ("init_spins", C.c_void_p),
                ("p_center", C.c_double)]


class JobStatus(C.Structure):
    _fields_ = [("state", C.c_uint32), ("error", C.c_int), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("footprint_bytes", C.c_uint64)]


class ServerStats(C.Structure):
    _fields_ = [("chain_steps", C.c_uint64), ("candidates", C.c_uint64), ("quanta", C.c_uint64),
                ("completed", C.c_uint64), ("busy_seconds", C.c_double),
                ("elapsed_seconds", C.c_double), ("device_bytes_in_use", C.c_uint64),
                ("queued", C.c_uint64), ("running", C.c_uint64), ("admit_seconds", C.c_double),
                ("retire_seconds", C.c_double), ("plan_seconds", C.c_double)]


SK_JOB_QUEUED, SK_JOB_RUNNING, SK_JOB_DONE, SK_JOB_FAILED, SK_JOB_CANCELLED = range(5)
EXPORTS += ["sk_set_generation", "sk_set_couplings_many", "mcmcmc_reset_many", "mcmcmc_observables_many"]
EXPORTS += ["sk_server_create", "sk_server_add_couplings", "sk_server_submit", "sk_server_poll",
            "sk_server_result", "sk_server_wait_all", "sk_server_stats", "sk_server_destroy",
            "sk_server_cancel"]


def _server_sigs(L):
    vp, u32, u64, d = C.c_void_p, C.c_uint32, C.c_uint64, C.c_double
    sig = {"sk_server_create": [u64, u32, C.POINTER(C.c_void_p)],
           "sk_server_add_couplings": [vp, u64, u32, u32, vp, d],
           "sk_server_submit": [vp, C.POINTER(Job), C.POINTER(C.c_uint64)],
           "sk_server_poll": [vp, u64, C.POINTER(JobStatus)],
           "sk_server_result": [vp, u64, vp, vp, C.POINTER(C.c_uint64)],
           "sk_server_wait_all": [vp, u64],
           "sk_server_cancel": [vp, u64],
           "sk_server_stats": [vp, C.POINTER(ServerStats)],
           "sk_server_destroy": [vp]}
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int


def _check_server(status, what):
    if status != SK_OK:
        raise SKError(status, what)


class Server:
    """sk_server_*: continuous batching of sampling jobs on one GPU."""

    def __init__(self, budget_bytes: int, quantum_steps: int = 256):
        _server_sigs(lib())
        h = C.c_void_p()
        _check_server(lib().sk_server_create(int(budget_bytes), int(quantum_steps), C.byref(h)),
                      "sk_server_create")
        self.handle = h
        self._keep = {}

    def add_couplings(self, couplings_id: int, J, scale: float = 1.0):
        J = np.ascontiguousarray(J)
        kind = SK_J_PM1 if J.dtype == np.int8 else SK_J_GAUSS
        _check_server(lib().sk_server_add_couplings(self.handle, int(couplings_id), J.shape[0], kind,
                                                    J.ctypes.data_as(C.c_void_p), float(scale)),
                      "sk_server_add_couplings")

    def submit(self, *, N, kind, chains, steps, K=8, rule=SK_RULE_MCMCMC, beta=1.0, seed=1,
               stream_id=0, J=None, couplings_id=0, scale=1.0, init=None, p_center=0.0) -> int:
        j = Job()
        j.N, j.kind, j.chains, j.steps = int(N), int(kind), int(chains), int(steps)
        j.K, j.rule, j.beta, j.seed, j.stream_id = int(K), int(rule), float(beta), int(seed), int(stream_id)
        j.couplings_id, j.scale, j.p_center = int(couplings_id), float(scale), float(p_center)
        if J is not None:
            J = np.ascontiguousarray(J)
            j.couplings = J.ctypes.data_as(C.c_void_p).value
        if init is not None:
            init = np.ascontiguousarray(init, dtype=np.int8)
            j.init_spins = init.ctypes.data_as(C.c_void_p).value
        t = C.c_uint64(0)
        _check_server(lib().sk_server_submit(self.handle, C.byref(j), C.byref(t)), "sk_server_submit")
        return t.value

    def poll(self, ticket: int) -> dict:
        st = JobStatus()
        _check_server(lib().sk_server_poll(self.handle, int(ticket), C.byref(st)), "sk_server_poll")
        return {k: getattr(st, k) for k, _ in JobStatus._fields_}

    def result(self, ticket: int, chains: int, N: int):
        E = np.zeros(chains)
        S = np.zeros((chains, N), dtype=np.int8)
        f = C.c_uint64(0)
        _check_server(lib().sk_server_result(self.handle, int(ticket), E.ctypes.data_as(C.c_void_p),
                                             S.ctypes.data_as(C.c_void_p), C.byref(f)),
                      "sk_server_result")
        return E, S, f.value

    def cancel(self, ticket: int):
        """sk_server_cancel: withdraw a queued or running job."""
        _check_server(lib().sk_server_cancel(self.handle, int(ticket)), "sk_server_cancel")

    def wait_all(self, timeout_ns: int = 0):
        _check_server(lib().sk_server_wait_all(self.handle, int(timeout_ns)), "sk_server_wait_all")

    def stats(self) -> dict:
        st = ServerStats()
        _check_server(lib().sk_server_stats(self.handle, C.byref(st)), "sk_server_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().sk_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        # at interpreter exit the order in which objects (and the CUDA
        # runtime) are torn down is not defined: leave the memory to the
        # process exit rather than call into the library then
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


SK_SETGEN_AUTO, SK_SETGEN_DIRECT, SK_SETGEN_CUMULATIVE = 0, 1, 2


def set_generation(P, out=None, stream=None, method: int = SK_SETGEN_AUTO):
    """sk_set_generation: P_gen(S | S minus M) for every bit mask M of an
    n-element set, P[e, p] = P_gen(e | p), by the direct recursion or the
    cumulative form (method).  Returns a numpy array unless a device tensor
    `out` of 2^n doubles is given."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    n = P.shape[0]
    if out is None:
        res = np.zeros(1 << n)
        _check(lib().sk_set_generation(n, P.ctypes.data_as(C.c_void_p), res.ctypes.data_as(C.c_void_p),
                                       SK_MEM_HOST, int(method), _stream_handle(stream)))
        return res
    p, mem = _ptr_mem(out)
    _check(lib().sk_set_generation(n, P.ctypes.data_as(C.c_void_p), p, mem, int(method), _stream_handle(stream)))
    return out


def _ptr_array(items):
    """(ctypes array of pointers, mem) of numpy arrays / torch tensors (None -> NULL)."""
    arr = (C.c_void_p * len(items))()
    mem = SK_MEM_HOST
    for i, x in enumerate(items):
        p, m = _ptr_mem(x)
        arr[i] = p.value if isinstance(p, C.c_void_p) else p
        if x is not None:
            mem = m
    return arr, mem


def set_couplings_many(insts, couplings):
    """sk_set_couplings_many: new couplings for many instances, all or nothing."""
    cs = [np.ascontiguousarray(J) if isinstance(J, np.ndarray) else J for J in couplings]
    hs = (C.c_void_p * len(insts))(*[x.handle.value for x in insts])
    arr, mem = _ptr_array(cs)
    _check(lib().sk_set_couplings_many(hs, len(insts), arr, mem))


def reset_many(runs, spins=None):
    """mcmcmc_reset_many: restart many runs from given spins (or the Philox start), all or nothing."""
    hs = (C.c_void_p * len(runs))(*[r.handle.value for r in runs])
    if spins is None:
        _check(lib().mcmcmc_reset_many(hs, len(runs), None, SK_MEM_HOST))
        return
    ss = [np.ascontiguousarray(x, dtype=np.int8) if isinstance(x, np.ndarray) else x for x in spins]
    arr, mem = _ptr_array(ss)
    _check(lib().mcmcmc_reset_many(hs, len(runs), arr, mem))


def observables_many(runs, first, count, outs):
    """mcmcmc_observables_many: records [first, first+count) of many runs into
    outs[i] = (energy, overlap, accepted) buffers (numpy or pinned/device torch)."""
    hs = (C.c_void_p * len(runs))(*[r.handle.value for r in runs])
    E, m1 = _ptr_array([o[0] for o in outs])
    Q, _ = _ptr_array([o[1] for o in outs])
    A, _ = _ptr_array([o[2] for o in outs])
    _check(lib().mcmcmc_observables_many(hs, len(runs), first, count, E, Q, A, m1))
