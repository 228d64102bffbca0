"""ctypes binding of libdeco.so (include/deco.h).

Argument marshalling only: every computation of the hot path runs in the CUDA
kernels behind the C ABI.  Device buffers are passed as torch CUDA tensors
(their data pointers), host buffers as NumPy arrays, streams as
torch.cuda.Stream objects or raw cudaStream_t integers.  There is no CPU
fallback: if libdeco.so cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdeco.so")

DECO_OK = 0
DECO_ERR_ARG = -1
DECO_ERR_GRAPH = -2
DECO_ERR_OOM = -3
DECO_ERR_CUDA = -4
DECO_ERR_NONFINITE = -5
DECO_ERR_TIMEOUT = -6
DECO_ERR_UNSUPPORTED = -7
STATUS_NAMES = {0: "DECO_OK", -1: "DECO_ERR_ARG", -2: "DECO_ERR_GRAPH", -3: "DECO_ERR_OOM",
                -4: "DECO_ERR_CUDA", -5: "DECO_ERR_NONFINITE", -6: "DECO_ERR_TIMEOUT",
                -7: "DECO_ERR_UNSUPPORTED"}

DECO_OBJ_MULTILINEAR01 = 0
DECO_OBJ_LAPLACIAN = 1
DECO_PREC_FP32 = 0
DECO_PREC_BF16 = 1
DECO_INIT_UNIFORM = 0
DECO_INIT_IDI = 1
DECO_INIT_DUI = 2
DECO_INIT_IDI_HALF_UNIFORM = 3
DECO_INIT_EXPLICIT = 4
DECO_INIT_MEAN = 5
DECO_PHASE_INIT_BEST = 0
DECO_PHASE_INIT_FRESH = 1
DECO_GRAPH_SKIP_SYMMETRY_CHECK = 0x1
DECO_KERNEL_AUTO = 0
DECO_KERNEL_GLOBAL = 1
DECO_KERNEL_ONCHIP = 2
DECO_KERNEL_DENSE = 3
DECO_KERNEL_DENSE_PER_STEP = 1 << 12
DECO_KERNEL_LEAN = 1 << 20
DECO_KERNEL_ROW_PAIRS = 1 << 21
DECO_KERNEL_PIPELINED = 1 << 22
DECO_KERNEL_PIPE_MIXED_ADD = 1 << 30
DECO_KERNEL_PIPE_L2_HINTS = 1 << 19
DECO_KERNEL_PIPE_WIDE = 1 << 2


def DECO_KERNEL_PIPE_ENTRIES(e: int) -> int:
    """Entries of a row per stage of the pipelined form: e = 0: 16, 1: 8, 2: 24, 3: 32."""
    return e << 23


def DECO_KERNEL_PIPE_STAGES(s: int) -> int:
    """Shared-memory stages per warp of the pipelined form: s = 0: 3, 1: 2, 2: 4."""
    return s << 25


def DECO_KERNEL_PIPE_WARPS(w: int) -> int:
    """Warps per block of the pipelined form: 0 = as many as fit (at most 8), 1..7."""
    return w << 27


def DECO_KERNEL_COLUMN_SLABS(s: int) -> int:
    """2^s column slabs run one after another (with DECO_KERNEL_GLOBAL)."""
    return s << 16

# every function include/deco.h declares (checked by the CPU test-suite)
EXPORTED = [
    "deco_create_graph", "deco_destroy_graph", "deco_graph_info", "deco_eval_cut",
    "deco_eval_cuts", "deco_step", "deco_run_phase", "deco_run_phase_noalloc", "deco_round_cut",
    "deco_init_block", "deco_autotune", "deco_set_tuning", "deco_create_batch", "deco_destroy_batch",
    "deco_batch_graph", "deco_solve_batch", "deco_mpnn_create", "deco_mpnn_destroy", "deco_mpnn_num_params",
    "deco_mpnn_get_params", "deco_mpnn_set_params", "deco_mpnn_infer", "deco_mpnn_loss_grad",
    "deco_mpnn_train_step", "deco_mpnn_train",
    "deco_idi_mean", "deco_dui_mean", "deco_solve", "deco_solve_budget", "deco_greedy", "deco_local_search",
    "deco_probe_mma_rate", "deco_probe_smem_rate", "deco_probe_wait_timeout", "deco_debug_fail_scratch_alloc", "deco_debug_pool_usage",
    "deco_last_error", "deco_abi_version",
]


class DecoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class deco_step_args(ctypes.Structure):
    _fields_ = [("objective", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("momentum", ctypes.c_float),
                ("alpha_cols", ctypes.c_void_p), ("steps_cols", ctypes.c_void_p),
                ("t", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class deco_params(ctypes.Structure):
    _fields_ = [("objective", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("init", ctypes.c_int32), ("polish_steps", ctypes.c_int32),
                ("eta", ctypes.c_float), ("scale", ctypes.c_float), ("beta", ctypes.c_float),
                ("uniform_half_width", ctypes.c_float), ("kernel", ctypes.c_int32),
                ("local_search", ctypes.c_int32), ("phase_init", ctypes.c_int32), ("eval_every", ctypes.c_int32)]


class deco_phase(ctypes.Structure):
    _fields_ = [("lift", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("momentum", ctypes.c_float)]


class deco_population(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int32), ("rounds", ctypes.c_int32), ("t_lo", ctypes.c_int32),
                ("t_hi", ctypes.c_int32), ("e_lo", ctypes.c_float), ("e_hi", ctypes.c_float),
                ("momentum", ctypes.c_float), ("n_lifts", ctypes.c_int32), ("lifts", ctypes.c_int32 * 8)]


class deco_result(ctypes.Structure):
    _fields_ = [("best_cut", ctypes.c_int64), ("best_init", ctypes.c_int32),
                ("best_phase", ctypes.c_int32), ("edge_updates", ctypes.c_int64),
                ("device_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdeco.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I32, I64, U32, U64, F32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float
    sig = {
        "deco_create_graph": (ctypes.c_int, [I32, I64, P, P, P, U32, ctypes.POINTER(P)]),
        "deco_destroy_graph": (None, [P]),
        "deco_graph_info": (ctypes.c_int, [P, P, P, P]),
        "deco_eval_cut": (ctypes.c_int, [P, P, P]),
        "deco_eval_cuts": (ctypes.c_int, [P, I32, P, P, P]),
        "deco_step": (ctypes.c_int, [P, I32, I32, P, P, P, ctypes.POINTER(deco_step_args), P, P]),
        "deco_run_phase": (ctypes.c_int, [P, I32, I32, P, P, I32, ctypes.POINTER(deco_step_args), I32, P, P]),
        "deco_run_phase_noalloc": (ctypes.c_int, [P, I32, I32, P, P, I32, ctypes.POINTER(deco_step_args), P, P]),
        "deco_autotune": (ctypes.c_int, [P, I32, I32, I32, F32, I32, P, P, P]),
        "deco_set_tuning": (ctypes.c_int, [P, I32, I32, I32]),
        "deco_create_batch": (ctypes.c_int, [P, I32, ctypes.POINTER(P)]),
        "deco_destroy_batch": (None, [P]),
        "deco_batch_graph": (ctypes.c_int, [P, ctypes.POINTER(P)]),
        "deco_solve_batch": (ctypes.c_int, [P, I32, ctypes.POINTER(deco_params), ctypes.POINTER(deco_population),
                                            U64, P, P, P, P, P, P, P, ctypes.POINTER(deco_result)]),
        "deco_mpnn_create": (ctypes.c_int, [I32, I32, U64, ctypes.POINTER(P)]),
        "deco_mpnn_destroy": (None, [P]),
        "deco_mpnn_num_params": (ctypes.c_int, [P, P]),
        "deco_mpnn_get_params": (ctypes.c_int, [P, P, I64]),
        "deco_mpnn_set_params": (ctypes.c_int, [P, P, I64]),
        "deco_mpnn_infer": (ctypes.c_int, [P, P, P, U64, I32, P, P]),
        "deco_mpnn_loss_grad": (ctypes.c_int, [P, P, P, P, U64, P, P, P]),
        "deco_mpnn_train_step": (ctypes.c_int, [P, P, P, P, U64, F32, P, P]),
        "deco_mpnn_train": (ctypes.c_int, [P, P, P, P, U64, F32, I32, P, P]),
        "deco_round_cut": (ctypes.c_int, [P, I32, I32, I32, I32, P, P, P, P, P]),
        "deco_init_block": (ctypes.c_int, [P, I32, I32, I32, ctypes.POINTER(deco_params), U64, I32, P, P, P, P]),
        "deco_idi_mean": (ctypes.c_int, [P, F32, U64, I32, P, P]),
        "deco_dui_mean": (ctypes.c_int, [P, U64, I32, P, P]),
        "deco_solve": (ctypes.c_int, [P, I32, ctypes.POINTER(deco_phase), I32, ctypes.POINTER(deco_params),
                                      U64, P, P, P, P, P, ctypes.POINTER(deco_result)]),
        "deco_solve_budget": (ctypes.c_int, [P, I32, ctypes.POINTER(deco_phase), I32, ctypes.POINTER(deco_params),
                                             U64, ctypes.c_double, I32, P, P, P, P, ctypes.POINTER(deco_result)]),
        "deco_greedy": (ctypes.c_int, [P, I32, U64, P, P, P]),
        "deco_local_search": (ctypes.c_int, [P, I32, P, I32, P, P, P]),
        "deco_probe_mma_rate": (ctypes.c_int, [I32, I32, I32, P, P]),
        "deco_probe_smem_rate": (ctypes.c_int, [I32, I32, P, P]),
        "deco_probe_wait_timeout": (ctypes.c_int, [I32, P, P]),
        "deco_debug_fail_scratch_alloc": (ctypes.c_int, [I32]),
        "deco_debug_pool_usage": (ctypes.c_int, [P, P, I32]),
        "deco_last_error": (ctypes.c_char_p, []),
        "deco_abi_version": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def last_error() -> str:
    return lib.deco_last_error().decode()


def _check(rc: int):
    if rc != DECO_OK:
        raise DecoError(rc, last_error())


def _ptr(x) -> Optional[int]:
    """Raw address of a torch tensor / NumPy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s) -> Optional[int]:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


class Graph:
    """Owning handle of a deco_graph (destroyed with the object)."""

    def __init__(self, handle: int, n: int, nnz: int):
        self.handle = handle
        self.n = n
        self.nnz = nnz

    def close(self):
        if self.handle:
            lib.deco_destroy_graph(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)


def deco_create_graph(n: int, row_ptr, col_idx, weights=None, flags: int = 0) -> Graph:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    h = ctypes.c_void_p()
    nnz = ci.size
    _check(lib.deco_create_graph(int(n), int(nnz), _ptr(rp), _ptr(ci) if ci.size else None,
                                 _ptr(w), int(flags), ctypes.byref(h)))
    return Graph(h.value, int(n), int(nnz))


def graph_from(g, flags: int = 0) -> Graph:
    """deco_create_graph from a graphgen.Graph-like object (n, row_ptr, col_idx, weights)."""
    return deco_create_graph(g.n, g.row_ptr, g.col_idx, g.weights, flags)


def deco_destroy_graph(g: Graph):
    g.close()


def deco_graph_info(g: Graph):
    n, nnz, wt = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib.deco_graph_info(g, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(wt)))
    return n.value, nnz.value, wt.value


def deco_eval_cut(g: Graph, z) -> int:
    zz = np.ascontiguousarray(z, dtype=np.uint8)
    if zz.size != g.n:
        raise ValueError("z must have n entries")
    out = ctypes.c_int64()
    _check(lib.deco_eval_cut(g, _ptr(zz), ctypes.byref(out)))
    return out.value


def deco_eval_cuts(g: Graph, B: int, z_dev, cuts_dev, stream=None):
    _check(lib.deco_eval_cuts(g, int(B), _ptr(z_dev), _ptr(cuts_dev), _stream(stream)))


def deco_solve_budget(g: Graph, B: int, phases: Sequence, p: deco_params, seed: int, budget_ms: float,
                      max_repeats: int = 1 << 30, warm=None, stream=None):
    """pDECO repeated until budget_ms of device time (or max_repeats); returns
    (deco_result, best assignment uint8[n], repetitions run)."""
    arr = (deco_phase * len(phases))(*[deco_phase(int(l), int(s), float(a), float(m)) for l, s, a, m in phases])
    assignment = np.zeros(g.n, dtype=np.uint8)
    warm_p = None if warm is None else np.ascontiguousarray(warm, dtype=np.uint8)
    out = deco_result()
    reps = ctypes.c_int32(0)
    _check(lib.deco_solve_budget(g, int(B), arr, len(phases), ctypes.byref(p), int(seed), float(budget_ms),
                                 int(max_repeats), _ptr(warm_p), _ptr(assignment), ctypes.byref(reps),
                                 _stream(stream), ctypes.byref(out)))
    return out, assignment, int(reps.value)


def deco_greedy(g: Graph, B: int, seed: int, z_dev, cuts_dev, stream=None):
    """Greedy comparator (App. C.1): B runs on Feistel orderings; z_dev n x B uint8, cuts_dev B int64."""
    _check(lib.deco_greedy(g, int(B), int(seed), _ptr(z_dev), _ptr(cuts_dev), _stream(stream)))


def deco_local_search(g: Graph, B: int, z_dev, max_rounds: int, cuts_dev=None, stream=None) -> int:
    """1-flip local search in place on z_dev (n x B uint8); returns the rounds that flipped a node."""
    r = ctypes.c_int32(0)
    _check(lib.deco_local_search(g, int(B), _ptr(z_dev), int(max_rounds), _ptr(cuts_dev), ctypes.byref(r),
                                 _stream(stream)))
    return int(r.value)


def step_args(objective=DECO_OBJ_MULTILINEAR01, precision=DECO_PREC_FP32, alpha=0.01, momentum=0.0,
              alpha_cols=None, steps_cols=None, t=0) -> deco_step_args:
    return deco_step_args(objective, precision, alpha, momentum, _ptr(alpha_cols), _ptr(steps_cols), t, 0)


def deco_step(g: Graph, C: int, ld: int, y_in, y_out, v, args: deco_step_args, flag=None, stream=None):
    _check(lib.deco_step(g, int(C), int(ld), _ptr(y_in), _ptr(y_out), _ptr(v), ctypes.byref(args),
                         _ptr(flag), _stream(stream)))


def deco_run_phase(g: Graph, C: int, ld: int, y, v, steps: int, args: deco_step_args,
                   kernel: int = DECO_KERNEL_AUTO, flag=None, stream=None):
    _check(lib.deco_run_phase(g, int(C), int(ld), _ptr(y), _ptr(v), int(steps), ctypes.byref(args),
                              int(kernel), _ptr(flag), _stream(stream)))


def deco_run_phase_noalloc(g: Graph, C: int, ld: int, y, v, steps: int, args: deco_step_args, flag=None,
                           stream=None):
    """deco_run_phase for callers that cannot let the library allocate device
    memory (their own pool holds the device, or allocation latency is not
    acceptable): the step kernel's second block lives in a fixed 16 MiB array
    inside the library.  Blocks larger than that are refused."""
    _check(lib.deco_run_phase_noalloc(g, int(C), int(ld), _ptr(y), _ptr(v), int(steps), ctypes.byref(args),
                                      _ptr(flag), _stream(stream)))


def deco_autotune(g: Graph, C: int, precision: int = DECO_PREC_FP32, objective: int = DECO_OBJ_MULTILINEAR01,
                  momentum: float = 0.9, probe_steps: int = 50, stream=None):
    """Time every launch shape of a C-column phase on g; returns (selector, us_per_step)."""
    sel = ctypes.c_int32()
    us = ctypes.c_float()
    _check(lib.deco_autotune(g, int(C), int(precision), int(objective), float(momentum), int(probe_steps),
                             ctypes.byref(sel), ctypes.byref(us), _stream(stream)))
    return sel.value, us.value


def deco_probe_mma_rate(n: int = 128, issuers: int = 1, count: int = 4096, stream=None) -> float:
    """ns per tcgen05.mma (M = 128, N = n, K = 16) per SM with `issuers` issuing threads."""
    ns = ctypes.c_float()
    _check(lib.deco_probe_mma_rate(int(n), int(issuers), int(count), ctypes.byref(ns), _stream(stream)))
    return ns.value


def deco_probe_smem_rate(width: int = 16, iters: int = 1 << 16, stream=None) -> float:
    """Shared-memory load bandwidth of the GPU in GB/s (all SMs; see include/deco.h)."""
    gbs = ctypes.c_float()
    _check(lib.deco_probe_smem_rate(int(width), int(iters), ctypes.byref(gbs), _stream(stream)))
    return gbs.value


def deco_probe_wait_timeout(which: int, stream=None):
    """Run one of the kernels' bounded waits on something that never completes
    (0 dense mbarrier, 1 dense grid barrier, 2 on-chip exchange mbarrier);
    returns (status, waited ms).  DECO_ERR_TIMEOUT is the expected status."""
    ms = ctypes.c_float()
    st = lib.deco_probe_wait_timeout(int(which), ctypes.byref(ms), _stream(stream))
    if st not in (DECO_OK, DECO_ERR_TIMEOUT):
        _check(st)
    return st, ms.value


def deco_debug_fail_scratch_alloc(k: int):
    """Fail the k-th scratch allocation from now on with DECO_ERR_OOM (0 disarms)."""
    _check(lib.deco_debug_fail_scratch_alloc(int(k)))


def deco_debug_pool_usage(reset: bool = False):
    """(bytes in use, high-water mark) of the current device's stream-ordered
    memory pool, which every scratch buffer of the library comes from; with
    reset the high-water mark then restarts from the current use."""
    now, high = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.deco_debug_pool_usage(ctypes.byref(now), ctypes.byref(high), 1 if reset else 0))
    return int(now.value), int(high.value)


def deco_set_tuning(g: Graph, C: int, precision: int, kernel: int):
    _check(lib.deco_set_tuning(g, int(C), int(precision), int(kernel)))


def deco_round_cut(g: Graph, B: int, lift: int, ld: int, precision: int, y, zbits, cuts, best=None,
                   stream=None):
    _check(lib.deco_round_cut(g, int(B), int(lift), int(ld), int(precision), _ptr(y), _ptr(zbits),
                              _ptr(cuts), _ptr(best), _stream(stream)))


def params(objective=DECO_OBJ_MULTILINEAR01, precision=DECO_PREC_FP32, init=DECO_INIT_UNIFORM,
           polish_steps=0, eta=0.8, scale=1e-4, beta=0.2, uniform_half_width=1.0,
           kernel=DECO_KERNEL_AUTO, local_search=0, phase_init=0, eval_every=0) -> deco_params:
    return deco_params(objective, precision, init, polish_steps, eta, scale, beta, uniform_half_width,
                       kernel, local_search, phase_init, eval_every)


def deco_init_block(g: Graph, B: int, lift: int, ld: int, p: deco_params, seed: int, phase: int, y,
                    mean=None, x0=None, stream=None):
    _check(lib.deco_init_block(g, int(B), int(lift), int(ld), ctypes.byref(p), int(seed), int(phase),
                               _ptr(mean), _ptr(x0), _ptr(y), _stream(stream)))


def deco_idi_mean(g: Graph, beta: float, seed: int, phase: int, h, stream=None):
    _check(lib.deco_idi_mean(g, float(beta), int(seed), int(phase), _ptr(h), _stream(stream)))


def deco_dui_mean(g: Graph, seed: int, phase: int, h, stream=None):
    _check(lib.deco_dui_mean(g, int(seed), int(phase), _ptr(h), _stream(stream)))


def deco_solve(g: Graph, B: int, phases: Sequence, p: deco_params, seed: int, x0=None, mean=None,
               want_assignment: bool = True, want_phase_cuts: bool = True, stream=None):
    """pDECO over `phases` (sequence of (lift, steps, alpha, momentum)).

    Returns (deco_result, assignment uint8[n] or None, phase_cuts int64[n_phases, B] or None).
    """
    arr = (deco_phase * len(phases))(*[deco_phase(int(l), int(s), float(a), float(m)) for l, s, a, m in phases])
    assignment = np.zeros(g.n, dtype=np.uint8) if want_assignment else None
    pc = np.zeros((len(phases), B), dtype=np.int64) if want_phase_cuts else None
    x0p = x0
    if isinstance(x0, np.ndarray):
        x0p = np.ascontiguousarray(x0, dtype=np.float32)
    meanp = mean
    if isinstance(mean, np.ndarray):
        meanp = np.ascontiguousarray(mean, dtype=np.float32)
    res = deco_result()
    _check(lib.deco_solve(g, int(B), arr, len(phases), ctypes.byref(p), int(seed), _ptr(x0p), _ptr(meanp),
                          _ptr(assignment), _ptr(pc), _stream(stream), ctypes.byref(res)))
    return res, assignment, pc


class Batch:
    """Owning handle of a deco_batch (the disjoint union of several graphs)."""

    def __init__(self, handle: int, sizes):
        self.handle = handle
        self.sizes = list(sizes)
        self.n = int(sum(self.sizes))

    def close(self):
        if self.handle:
            lib.deco_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)

    def graph(self) -> Graph:
        """Non-owning view of the union graph (for deco_autotune / deco_set_tuning)."""
        h = ctypes.c_void_p()
        _check(lib.deco_batch_graph(self, ctypes.byref(h)))
        view = Graph(h.value, self.n, 0)
        view.close = lambda: None          # owned by the batch
        return view


def deco_create_batch(graphs: Sequence[Graph]) -> Batch:
    arr = (ctypes.c_void_p * len(graphs))(*[g.handle for g in graphs])
    h = ctypes.c_void_p()
    _check(lib.deco_create_batch(arr, len(graphs), ctypes.byref(h)))
    return Batch(h.value, [g.n for g in graphs])


def deco_destroy_batch(b: Batch):
    b.close()


def population(candidates=32, rounds=5, t_lo=500, t_hi=2000, e_lo=-4.0, e_hi=-1.0, momentum=0.9,
               lifts=(1, 2)) -> deco_population:
    arr = (ctypes.c_int32 * 8)(*(list(lifts) + [0] * (8 - len(lifts))))
    return deco_population(candidates, rounds, t_lo, t_hi, e_lo, e_hi, momentum, len(lifts), arr)


def deco_solve_batch(b: Batch, B: int, p: deco_params, pop: deco_population, seed: int,
                     want_assignment=False, want_round_cuts=False, stream=None):
    """Returns (deco_result, best_cuts[n_graphs], extras dict)."""
    G = len(b.sizes)
    best = np.zeros(G, dtype=np.int64)
    assignment = np.zeros(b.n, dtype=np.uint8) if want_assignment else None
    rc = np.zeros((pop.rounds, G, B), dtype=np.int64) if want_round_cuts else None
    scores = np.zeros((pop.rounds, pop.candidates), dtype=np.int64)
    fe = np.zeros(pop.candidates, dtype=np.float32)
    fT = np.zeros(pop.candidates, dtype=np.int32)
    res = deco_result()
    _check(lib.deco_solve_batch(b, int(B), ctypes.byref(p), ctypes.byref(pop), int(seed), _ptr(best),
                                _ptr(assignment), _ptr(rc), _ptr(scores), _ptr(fe), _ptr(fT), _stream(stream),
                                ctypes.byref(res)))
    return res, best, {"assignment": assignment, "round_cuts": rc, "round_scores": scores,
                       "final_e": fe, "final_T": fT}


class Mpnn:
    """Owning handle of the learned-proposal network (deco_mpnn)."""

    def __init__(self, hidden: int = 64, layers: int = 3, seed: int = 0):
        h = ctypes.c_void_p()
        _check(lib.deco_mpnn_create(int(hidden), int(layers), int(seed), ctypes.byref(h)))
        self.handle = h.value
        self.hidden, self.layers = hidden, layers
        c = ctypes.c_int64()
        _check(lib.deco_mpnn_num_params(self.handle, ctypes.byref(c)))
        self.n_params = c.value

    def close(self):
        if self.handle:
            lib.deco_mpnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(lib.deco_mpnn_get_params(self, _ptr(out), self.n_params))
        return out

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib.deco_mpnn_set_params(self, _ptr(th), th.size))

    def infer(self, target, h_dev, feat_seed: int = 0, precision: int = DECO_PREC_FP32, stream=None):
        g, b = (target, None) if isinstance(target, Graph) else (None, target)
        _check(lib.deco_mpnn_infer(self, g, b, int(feat_seed), int(precision), _ptr(h_dev), _stream(stream)))

    def loss_grad(self, target, z_dev, grad_dev=None, feat_seed: int = 0, stream=None) -> float:
        g, b = (target, None) if isinstance(target, Graph) else (None, target)
        loss = ctypes.c_double()
        _check(lib.deco_mpnn_loss_grad(self, g, b, _ptr(z_dev), int(feat_seed), ctypes.byref(loss),
                                       _ptr(grad_dev), _stream(stream)))
        return loss.value

    def train_step(self, target, z_dev, lr: float = 1e-3, feat_seed: int = 0, stream=None) -> float:
        g, b = (target, None) if isinstance(target, Graph) else (None, target)
        loss = ctypes.c_double()
        _check(lib.deco_mpnn_train_step(self, g, b, _ptr(z_dev), int(feat_seed), float(lr), ctypes.byref(loss),
                                        _stream(stream)))
        return loss.value

    def train(self, target, z_dev, steps: int, lr: float = 1e-3, feat_seed: int = 0, stream=None) -> np.ndarray:
        g, b = (target, None) if isinstance(target, Graph) else (None, target)
        losses = np.zeros(max(int(steps), 1), dtype=np.float64)
        _check(lib.deco_mpnn_train(self, g, b, _ptr(z_dev), int(feat_seed), float(lr), int(steps), _ptr(losses),
                                   _stream(stream)))
        return losses[:steps]


def deco_abi_version() -> int:
    return lib.deco_abi_version()
