"""GB300 (sm_103a) solver of the Picard-iteration / adaptive-control-variate
BSDE method of Labart & Lelong (arXiv:1102.4666): pricing and hedging of
European and American basket options in local-volatility models.

This module is a thin ctypes binding of the C ABI in include/bsde.h: it only
marshals arguments.  Every step of Algorithm 2 runs in the CUDA kernels of
_lib/libbsde_gb300.so; there is no CPU fallback, and importing this package
raises when the library has not been built (``python -c "import
__graft_entry__ as g; g.build()"``).

PyTorch is used only for device memory: ``torch_allocator()`` returns hooks
that route the library's allocations through PyTorch's caching allocator.
"""
import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbsde_gb300.so")

MAX_D = 16
MAX_IT = 64
MAX_RANKS = 64

OK = 0
ERR_INVALID_ARG = -1
ERR_STATE = -2
ERR_ILLPOSED = -3
ERR_NOMEM = -4
ERR_NOT_PD = -5
ERR_TIMEOUT = -6
ERR_CUDA = -7
ERR_EXCHANGE = -8

PREC_FP64 = 0
PREC_MIXED = 1

VOL_CONST, VOL_ABS_TANH, VOL_SIN_TANH, VOL_DUPIRE = 0, 1, 2, 3
PAYOFF_PUT, PAYOFF_CALL = 0, 1
OBSTACLE_PAYOFF, OBSTACLE_RAW = 0, 1
POLICY_FIFO, POLICY_SHORTEST, POLICY_RESPONSE_RATIO, POLICY_SIZE_LANES = 0, 1, 2, 3

_dptr = ctypes.POINTER(ctypes.c_double)

alloc_fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
free_fn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
exchange_fn = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_void_p, ctypes.c_void_p)


class bsde_create_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("alloc", alloc_fn),
                ("free", free_fn), ("alloc_user", ctypes.c_void_p), ("mem_budget", ctypes.c_size_t),
                ("precision", ctypes.c_int)]


class bsde_sigma(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("kind", ctypes.c_int), ("a", _dptr), ("a_scalar", ctypes.c_double),
                ("b", ctypes.c_double), ("kappa", _dptr), ("kappa_scalar", ctypes.c_double),
                ("s_dupire", ctypes.c_double), ("rho", ctypes.c_double), ("corr", _dptr), ("div", _dptr)]


class bsde_payoff(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("K", ctypes.c_double), ("T", ctypes.c_double), ("S0", _dptr),
                ("weights", _dptr)]


class bsde_penalty(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("obstacle", ctypes.c_int)]


class bsde_solve_params(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("N_steps", ctypes.c_int), ("eta", ctypes.c_int), ("q", ctypes.c_double),
                ("K_it", ctypes.c_int), ("seed", ctypes.c_uint64), ("k_start", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("use_graph", ctypes.c_int), ("timing", ctypes.c_int),
                ("allow_underdetermined", ctypes.c_int), ("eval_mode", ctypes.c_int),
                ("paths_tpb", ctypes.c_int), ("paths_ppt", ctypes.c_int), ("ls_mode", ctypes.c_int),
                ("gram_splits", ctypes.c_int)]


class bsde_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("d", ctypes.c_int), ("p", ctypes.c_int), ("K_it", ctypes.c_int),
                ("price", ctypes.c_double), ("delta", ctypes.c_double * MAX_D),
                ("dudx", ctypes.c_double * MAX_D), ("price_iter", ctypes.c_double * MAX_IT),
                ("resid_l2", ctypes.c_double * MAX_IT), ("resid_linf", ctypes.c_double * MAX_IT),
                ("ms_total", ctypes.c_double), ("ms_paths", ctypes.c_double), ("ms_gram", ctypes.c_double),
                ("ms_solve", ctypes.c_double), ("path_steps", ctypes.c_double),
                ("path_steps_per_s", ctypes.c_double), ("path_launches", ctypes.c_int),
                ("kernel_launches", ctypes.c_int), ("rank", ctypes.c_int)]

    def to_dict(self):
        d, K = self.d, self.K_it
        return {"status": self.status, "d": d, "p": self.p, "K_it": K, "price": self.price,
                "delta": list(self.delta[:d]), "dudx": list(self.dudx[:d]),
                "price_iter": list(self.price_iter[:K]), "resid_l2": list(self.resid_l2[:K]),
                "resid_linf": list(self.resid_linf[:K]), "ms_total": self.ms_total,
                "ms_paths": self.ms_paths, "ms_gram": self.ms_gram, "ms_solve": self.ms_solve,
                "path_steps": self.path_steps, "path_steps_per_s": self.path_steps_per_s,
                "path_launches": self.path_launches, "kernel_launches": self.kernel_launches,
                "rank": self.rank}


class bsde_peer_exchange(ctypes.Structure):
    _fields_ = [("c", ctypes.c_void_p * MAX_RANKS), ("flag", ctypes.c_void_p * MAX_RANKS),
                ("c_len", ctypes.c_size_t), ("wait_ms", ctypes.c_double), ("pushed", exchange_fn),
                ("user", ctypes.c_void_p)]


class bsde_server_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_slots", ctypes.c_int), ("mem_budget", ctypes.c_size_t),
                ("precision", ctypes.c_int), ("policy", ctypes.c_int), ("large_slots", ctypes.c_int)]


class bsde_request(ctypes.Structure):
    _fields_ = [("sigma", bsde_sigma), ("r", ctypes.c_double), ("payoff", bsde_payoff),
                ("penalty", bsde_penalty), ("n", ctypes.c_int), ("lo", ctypes.c_double * (MAX_D + 1)),
                ("hi", ctypes.c_double * (MAX_D + 1)), ("params", bsde_solve_params)]


class bsde_server_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("queued", ctypes.c_uint64), ("running", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("path_steps", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("path_steps_per_s", ctypes.c_double)]


# every exported entry point with its argument types
_SIGNATURES = {
    "bsde_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(bsde_create_opts)]),
    "bsde_destroy": (None, [ctypes.c_void_p]),
    "bsde_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "bsde_set_model": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(bsde_sigma), ctypes.c_double,
                                      ctypes.POINTER(bsde_payoff), ctypes.POINTER(bsde_penalty)]),
    "bsde_set_grid": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dptr, _dptr, ctypes.c_int]),
    "bsde_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(bsde_solve_params),
                                  ctypes.POINTER(bsde_report)]),
    "bsde_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(bsde_solve_params), ctypes.c_int, _dptr,
                                    _dptr, _dptr, _dptr, _dptr]),
    "bsde_gram_matrix": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(bsde_solve_params), ctypes.c_int,
                                        _dptr, ctypes.c_int]),
    "bsde_set_shard": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_size_t, exchange_fn, ctypes.c_void_p]),
    "bsde_set_shard_peers": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(bsde_peer_exchange)]),
    "bsde_shard_block": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    "bsde_basis_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_int)]),
    "bsde_basis_indices": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "bsde_get_coeffs": (ctypes.c_int, [ctypes.c_void_p, _dptr, ctypes.c_int]),
    "bsde_set_coeffs": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(bsde_solve_params), _dptr,
                                       ctypes.c_int]),
    "bsde_eval_price_delta": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dptr, _dptr, _dptr, _dptr]),
    "bsde_corrections_noalloc": (ctypes.c_int, [
        ctypes.POINTER(bsde_sigma), ctypes.c_double, ctypes.POINTER(bsde_payoff), ctypes.POINTER(bsde_penalty),
        _dptr, _dptr, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
        ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    "bsde_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(bsde_server_opts)]),
    "bsde_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(bsde_request),
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "bsde_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(bsde_report)]),
    "bsde_server_drain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "bsde_server_stats_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(bsde_server_stats)]),
    "bsde_server_destroy": (None, [ctypes.c_void_p]),
    "bsde_server_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
}

_LIB = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libbsde_gb300.so is not built: run __graft_entry__.build() "
                              "(nvcc for sm_103a); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


lib()  # fail loudly at import when the library is missing


# same names as the C ABI
def _export(name):
    def call(*args):
        return getattr(lib(), name)(*args)
    call.__name__ = name
    call.__doc__ = "C ABI entry point %s of include/bsde.h" % name
    return call


for _n in _SIGNATURES:
    globals()[_n] = _export(_n)


class BsdeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (status %d)" % (msg, code))
        self.code = code


def _arr(vals):
    a = (ctypes.c_double * len(vals))(*[float(v) for v in vals])
    return a


# ---------------------------------------------------------------------------
# marshalling of the workload dictionaries of workloads.py
# ---------------------------------------------------------------------------

VOL = {"const": VOL_CONST, "abs_tanh": VOL_ABS_TANH, "sin_tanh": VOL_SIN_TANH, "dupire": VOL_DUPIRE}


def model_structs(cfg):
    """(sigma, r, payoff, penalty, keep-alive) from a workload dictionary."""
    d = cfg["d"]
    vol = cfg["vol"]
    keep = []
    sg = bsde_sigma()
    sg.d = d
    sg.kind = VOL[vol["kind"]]
    a = vol.get("a", 0.0)
    if isinstance(a, (list, tuple)):
        arr = _arr(a); keep.append(arr); sg.a = ctypes.cast(arr, _dptr)
    else:
        sg.a_scalar = float(a)
    sg.b = float(vol.get("b", 0.0))
    kap = vol.get("kappa", 0.0)
    if isinstance(kap, (list, tuple)):
        arr = _arr(kap); keep.append(arr); sg.kappa = ctypes.cast(arr, _dptr)
    else:
        sg.kappa_scalar = float(kap)
    sg.s_dupire = float(vol.get("s", 0.0))
    sg.rho = float(cfg.get("rho", 0.0))
    if cfg.get("corr") is not None:
        arr = _arr([v for row in cfg["corr"] for v in row]); keep.append(arr); sg.corr = ctypes.cast(arr, _dptr)
    arr = _arr(cfg["div"]); keep.append(arr); sg.div = ctypes.cast(arr, _dptr)
    pf = bsde_payoff()
    pf.kind = PAYOFF_PUT if cfg["payoff"] == "put" else PAYOFF_CALL
    pf.K = cfg["K"]
    pf.T = cfg["T"]
    arr = _arr(cfg["S0"]); keep.append(arr); pf.S0 = ctypes.cast(arr, _dptr)
    arr = _arr(cfg["weights"]); keep.append(arr); pf.weights = ctypes.cast(arr, _dptr)
    pen = bsde_penalty()
    pen.lambda_ = cfg["lambda"]
    pen.obstacle = OBSTACLE_PAYOFF if cfg.get("obstacle", "payoff") == "payoff" else OBSTACLE_RAW
    return sg, float(cfg["r"]), pf, pen, keep


def solve_params(cfg, seed=None, K_it=None, k_start=0, refine_steps=-1, use_graph=1, timing=0,
                 allow_underdetermined=0, eval_mode=0, paths_tpb=0, paths_ppt=0, ls_mode=0, gram_splits=0):
    p = bsde_solve_params()
    p.M, p.N_steps, p.eta, p.q = cfg["M"], cfg["N"], cfg["eta"], cfg.get("q", 1.0)
    p.K_it = cfg["K_it"] if K_it is None else K_it
    p.seed = cfg["seed"] if seed is None else seed
    p.k_start, p.refine_steps, p.use_graph, p.timing = k_start, refine_steps, use_graph, timing
    p.allow_underdetermined = allow_underdetermined
    p.eval_mode = eval_mode
    p.paths_tpb, p.paths_ppt = paths_tpb, paths_ppt
    p.ls_mode = ls_mode
    p.gram_splits = gram_splits
    return p


def request(cfg, seed=None, use_graph=1, precision=None):
    """A bsde_request (and its keep-alive list) from a workload dictionary.
    With a precision, the launch shape and Gram split count tuned for the
    request's problem class (autotune cache) go into its parameters."""
    sg, r, pf, pen, keep = model_structs(cfg)
    rq = bsde_request()
    rq.sigma, rq.r, rq.payoff, rq.penalty = sg, r, pf, pen
    rq.n = cfg["n"]
    for v in range(cfg["d"] + 1):
        rq.lo[v] = cfg["lo"][v]
        rq.hi[v] = cfg["hi"][v]
    kw = {}
    if precision is not None:
        from . import autotune
        shape = autotune.lookup(cfg, precision)
        if shape:
            kw["paths_tpb"], kw["paths_ppt"] = shape
        kw["gram_splits"] = autotune.lookup_gram_splits(cfg, precision)
    rq.params = solve_params(cfg, seed=seed, use_graph=use_graph, **kw)
    return rq, keep


_TORCH_HOOKS = None


def torch_allocator():
    """(alloc, free) hooks on PyTorch's CUDA caching allocator."""
    global _TORCH_HOOKS
    if _TORCH_HOOKS is None:
        import torch

        def _alloc(nbytes, stream, user):
            try:
                dev = torch.cuda.current_device()
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, stream, user):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        _TORCH_HOOKS = (alloc_fn(_alloc), free_fn(_free))
    return _TORCH_HOOKS


class Solver:
    """One context of the C ABI set up from a workload dictionary."""

    def __init__(self, cfg, precision="mixed", device=0, stream=None, torch_memory=True, mem_budget=0,
                 launch_shape=None, allocator=None, gram_splits=0):
        self.cfg = cfg
        # (threads per CTA, paths per thread) of the path kernel, e.g. from
        # autotune.lookup()/tune(); None leaves the library's choice
        self.launch_shape = launch_shape
        # split count of the tensor-core Gram (autotune.lookup_gram_splits; 0: default)
        self.gram_splits = gram_splits
        o = bsde_create_opts()
        o.device = device
        o.stream = stream
        if allocator is not None:
            # an object with alloc(nbytes, stream) -> device address or None
            # and free(ptr, stream); the callbacks live as long as the Solver
            self._hooks = (alloc_fn(lambda nb, st, u: allocator.alloc(nb, st)),
                           free_fn(lambda ptr, st, u: allocator.free(ptr, st)))
            o.alloc, o.free = self._hooks
        elif torch_memory:
            a, f = torch_allocator()
            o.alloc, o.free = a, f
        o.mem_budget = mem_budget
        o.precision = PREC_MIXED if precision == "mixed" else PREC_FP64
        h = ctypes.c_void_p()
        rc = lib().bsde_create(ctypes.byref(h), ctypes.byref(o))
        if rc != OK:
            raise BsdeError(rc, lib().bsde_last_error(None).decode())
        self.h = h
        self._check(self.set_model(cfg))
        self._check(self.set_grid(cfg))

    def _check(self, rc):
        if rc != OK:
            raise BsdeError(rc, lib().bsde_last_error(self.h).decode())
        return rc

    def set_model(self, cfg):
        sg, r, pf, pen, keep = model_structs(cfg)
        return lib().bsde_set_model(self.h, ctypes.byref(sg), r, ctypes.byref(pf), ctypes.byref(pen))

    def set_grid(self, cfg, resample=1):
        lo, hi = _arr(cfg["lo"]), _arr(cfg["hi"])
        return lib().bsde_set_grid(self.h, cfg["n"], ctypes.cast(lo, _dptr), ctypes.cast(hi, _dptr), resample)

    def _shape(self, kw):
        if self.launch_shape and "paths_tpb" not in kw and "paths_ppt" not in kw:
            kw = dict(kw, paths_tpb=self.launch_shape[0], paths_ppt=self.launch_shape[1])
        if self.gram_splits and "gram_splits" not in kw:
            kw = dict(kw, gram_splits=self.gram_splits)
        return kw

    def solve(self, check=True, **kw):
        p = solve_params(self.cfg, **self._shape(kw))
        rep = bsde_report()
        rc = lib().bsde_solve(self.h, ctypes.byref(p), ctypes.byref(rep))
        if check:
            self._check(rc)
        return rep

    def iterate(self, k, alpha=None, check=True, **kw):
        """One iteration from alpha (None: current); returns t, x, c, alpha_next."""
        import numpy as np
        cfg = self.cfg
        p = solve_params(cfg, **self._shape(kw))
        n, d = cfg["n"], cfg["d"]
        P = self.basis_size(p.eta, p.q)
        t = np.zeros(n); x = np.zeros(d * n); c = np.zeros(n); an = np.zeros(P)
        ain = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64)
        rc = lib().bsde_iterate(self.h, ctypes.byref(p), k,
                                None if ain is None else ain.ctypes.data_as(_dptr),
                                t.ctypes.data_as(_dptr), x.ctypes.data_as(_dptr), c.ctypes.data_as(_dptr),
                                an.ctypes.data_as(_dptr))
        if check:
            self._check(rc)
        return t, x.reshape(d, n), c, an

    def gram(self, k, **kw):
        """The Gram matrix B^T B of iteration k's points (p x p), as the
        refit of a solve with these parameters would factorise it."""
        import numpy as np
        p = solve_params(self.cfg, **self._shape(kw))
        P = self.basis_size(p.eta, p.q)
        A = np.zeros((P, P))
        self._check(lib().bsde_gram_matrix(self.h, ctypes.byref(p), k, A.ctypes.data_as(_dptr), P * P))
        return A

    def set_shard(self, rank, nranks, xbuf=None, exchange=None):
        """Run the path kernel on this rank's block of points only
        (bsde_set_shard).  xbuf: a float64 CUDA tensor of at least
        nranks * ceil(n / nranks) values (the corrections of every rank);
        exchange(xbuf, nb, rank, nranks, stream) fills it with every rank's
        block, ordered on the CUDA stream `stream` (an int handle), e.g.
        torch_distributed_exchange().  nranks = 1 turns sharding off."""
        if nranks == 1:
            self._shard = None
            return self._check(lib().bsde_set_shard(self.h, 0, 1, None, 0, exchange_fn(), None))

        def _hook(c_dev, nb, rank_, nranks_, stream, user):
            try:
                exchange(xbuf, nb, rank_, nranks_, stream or 0)
                return 0
            except Exception:  # reported as BSDE_ERR_EXCHANGE
                import traceback
                traceback.print_exc()
                return 1

        cb = exchange_fn(_hook)
        self._shard = (cb, xbuf, exchange)  # keep alive while the setting holds
        return self._check(lib().bsde_set_shard(self.h, rank, nranks, xbuf.data_ptr(), xbuf.numel(), cb,
                                                None))

    def set_shard_peers(self, rank, nranks, bufs, flags, wait_ms=0.0, pushed=None):
        """Sharding with the exchange done by the devices (bsde_set_shard_peers):
        bufs[q] / flags[q] are rank q's float64 correction buffer (at least
        2 * nranks * ceil(n / nranks) values) and uint32/int32 arrival
        counters (nranks, zeroed), as tensors this device can address;
        pushed(nb, rank, nranks, stream), if given, runs on the host between
        this rank's push and its device-side wait."""
        px = bsde_peer_exchange()
        for q in range(nranks):
            px.c[q] = bufs[q].data_ptr()
            px.flag[q] = flags[q].data_ptr()
        px.c_len = min(b.numel() for b in bufs)
        px.wait_ms = wait_ms
        cb = exchange_fn()
        if pushed is not None:
            def _hook(c_dev, nb, rank_, nranks_, stream, user):
                try:
                    pushed(nb, rank_, nranks_, stream or 0)
                    return 0
                except Exception:
                    import traceback
                    traceback.print_exc()
                    return 1
            cb = exchange_fn(_hook)
        px.pushed = cb
        self._shard = (cb, bufs, flags, px)  # keep alive while the setting holds
        return self._check(lib().bsde_set_shard_peers(self.h, rank, nranks, ctypes.byref(px)))

    def basis_size(self, eta=None, q=None):
        eta = self.cfg["eta"] if eta is None else eta
        q = self.cfg.get("q", 1.0) if q is None else q
        out = ctypes.c_int()
        self._check(lib().bsde_basis_size(self.cfg["d"], eta, q, ctypes.byref(out)))
        return out.value

    def coeffs(self):
        import numpy as np
        P = self.basis_size()
        a = np.zeros(P)
        self._check(lib().bsde_get_coeffs(self.h, a.ctypes.data_as(_dptr), P))
        return a

    def set_coeffs(self, alpha, **kw):
        import numpy as np
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        p = solve_params(self.cfg, **kw)
        return self._check(lib().bsde_set_coeffs(self.h, ctypes.byref(p), a.ctypes.data_as(_dptr), len(a)))

    def eval(self, t, S):
        import numpy as np
        t = np.ascontiguousarray(t, dtype=np.float64).ravel()
        S = np.ascontiguousarray(S, dtype=np.float64).reshape(len(t), self.cfg["d"])
        price = np.zeros(len(t)); delta = np.zeros(S.shape)
        self._check(lib().bsde_eval_price_delta(self.h, len(t), t.ctypes.data_as(_dptr),
                                                S.ctypes.data_as(_dptr), price.ctypes.data_as(_dptr),
                                                delta.ctypes.data_as(_dptr)))
        return price, delta

    def close(self):
        if getattr(self, "h", None):
            lib().bsde_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shard_block(n, rank, nranks):
    """(i0, i1): the block of points rank `rank` of nranks simulates."""
    i0, i1 = ctypes.c_int(), ctypes.c_int()
    rc = lib().bsde_shard_block(n, rank, nranks, ctypes.byref(i0), ctypes.byref(i1))
    if rc != OK:
        raise BsdeError(rc, "bsde_shard_block")
    return i0.value, i1.value


def torch_distributed_exchange(group=None):
    """The exchange of a point-sharded solve over torch.distributed: an
    all-gather of every rank's block of nb corrections into xbuf (NCCL for
    CUDA tensors, ordered on the solve's stream; gloo for CPU tensors).
    Only argument marshalling: the collective is torch.distributed's."""
    import torch
    import torch.distributed as dist

    def exchange(xbuf, nb, rank, nranks, stream=0):
        out = xbuf[:nranks * nb]
        if out.is_cuda:
            with torch.cuda.stream(torch.cuda.ExternalStream(int(stream), device=out.device)):
                mine = out[rank * nb:(rank + 1) * nb].clone()
                dist.all_gather_into_tensor(out, mine, group=group)
        else:
            mine = out[rank * nb:(rank + 1) * nb].clone()
            dist.all_gather(list(out.split(nb)), mine, group=group)

    return exchange


def basis_indices(d, eta, q=1.0):
    """Multi-indices of the library's basis (host only, no GPU)."""
    import numpy as np
    P = ctypes.c_int()
    rc = lib().bsde_basis_size(d, eta, q, ctypes.byref(P))
    if rc != OK:
        raise BsdeError(rc, "bsde_basis_size")
    nu = np.zeros((P.value, d + 1), dtype=np.int32)
    rc = lib().bsde_basis_indices(d, eta, q, nu.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), P.value)
    if rc != OK:
        raise BsdeError(rc, "bsde_basis_indices")
    return nu


class Server:
    """Continuous-batching server of the C ABI (bsde_server_*): up to
    max_slots requests resident at once (each a captured graph of its whole
    solve on a stream of its own), admitted while they fit mem_budget bytes
    (0: no limit) in the order of the policy: "fifo", "shortest" (fewest
    path-steps K_it n M N first), "response_ratio" (highest
    (wait + service) / service first) or "size_lanes" (arrival order; a
    request with at least the average work waits while large_slots such
    requests run, smaller ones pass it)."""

    def __init__(self, device=0, max_slots=16, mem_budget=0, precision="mixed", policy="fifo",
                 large_slots=2):
        o = bsde_server_opts()
        o.device, o.max_slots, o.mem_budget = device, max_slots, mem_budget
        o.large_slots = large_slots
        o.policy = {"fifo": POLICY_FIFO, "shortest": POLICY_SHORTEST,
                    "response_ratio": POLICY_RESPONSE_RATIO, "size_lanes": POLICY_SIZE_LANES}[policy]
        o.precision = PREC_MIXED if precision == "mixed" else PREC_FP64
        self.precision = precision
        h = ctypes.c_void_p()
        rc = lib().bsde_server_create(ctypes.byref(h), ctypes.byref(o))
        if rc != OK:
            raise BsdeError(rc, "bsde_server_create")
        self.h = h

    def submit(self, cfg, seed=None):
        # the request's class is looked up in the autotune cache: its tuned
        # path-kernel launch shape and Gram split count, when tuned
        rq, keep = request(cfg, seed=seed, precision=self.precision)
        rid = ctypes.c_uint64()
        rc = lib().bsde_server_submit(self.h, ctypes.byref(rq), ctypes.byref(rid))
        if rc != OK:
            raise BsdeError(rc, lib().bsde_server_last_error(self.h).decode())
        return rid.value

    def poll(self, rid):
        rep = bsde_report()
        rc = lib().bsde_server_poll(self.h, rid, ctypes.byref(rep))
        if rc < 0:
            raise BsdeError(rc, lib().bsde_server_last_error(self.h).decode())
        return rep if rc == 1 else None

    def drain(self, timeout_ms=0.0):
        return lib().bsde_server_drain(self.h, timeout_ms)

    def stats(self):
        st = bsde_server_stats()
        lib().bsde_server_stats_get(self.h, ctypes.byref(st))
        return {k: getattr(st, k) for k, _ in bsde_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().bsde_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
