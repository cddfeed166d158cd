"""FP64 CPU oracle of the BSDE solver of Labart & Lelong (Algorithm 2).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline leg of bench.py import this module.  It shares no code with the
CUDA library (paper_1102_4666_gb300); the per-path arithmetic lives in the
plain C file oracle.c, the rest is numpy:

  * the multi-index sets of Section 3.2.2 (total degree, eq. hyper_set),
  * the basis matrix B_l(t_i, x_i) from numpy's Chebyshev Vandermonde matrix,
  * the least-squares extrapolation of eq. alpha (Algorithm 2) through
    numpy.linalg.lstsq (an SVD-based LAPACK solver, in the role the paper
    gives to LAPACK's dgelsy, Section 3.2.2),
  * the Picard loop of Algorithm 2 and the price / delta outputs
    (Section 5.3: V = Y = u, Delta = grad_x V).
"""
import ctypes
import math
import os

import numpy as np
from numpy.polynomial import chebyshev as npcheb

from . import build as _build

MAXD = 16
VOL_KINDS = {"const": 0, "abs_tanh": 1, "sin_tanh": 2, "dupire": 3}


class Model(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("N", ctypes.c_int), ("M", ctypes.c_int),
        ("payoff", ctypes.c_int), ("obstacle", ctypes.c_int), ("vol_kind", ctypes.c_int),
        ("T", ctypes.c_double), ("r", ctypes.c_double), ("lam", ctypes.c_double),
        ("K", ctypes.c_double),
        ("w", ctypes.c_double * MAXD), ("va", ctypes.c_double * MAXD),
        ("vb", ctypes.c_double), ("kappa", ctypes.c_double * MAXD),
        ("s_dupire", ctypes.c_double), ("div", ctypes.c_double * MAXD),
        ("C", ctypes.c_double * (MAXD * MAXD)), ("L", ctypes.c_double * (MAXD * MAXD)),
        ("lo", ctypes.c_double * (MAXD + 1)), ("hi", ctypes.c_double * (MAXD + 1)),
        ("key", ctypes.c_uint32 * 2),
    ]


class Basis(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("dp", ctypes.c_int), ("eta", ctypes.c_int),
                ("nu", ctypes.POINTER(ctypes.c_int))]


class PathInfo(ctypes.Structure):
    _fields_ = [("sstar", ctypes.c_int)] + [
        (nm, ctypes.c_double) for nm in
        ("theta", "tau", "u", "ut", "Lu", "f", "g1", "uT", "phiT", "phitau", "a")
    ] + [("XT", ctypes.c_double * MAXD), ("Xtau", ctypes.c_double * MAXD),
         ("Xs", ctypes.c_double * MAXD)]


_LIB = None


def lib():
    """The compiled oracle.c (built on first use with gcc)."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        dp_ = ctypes.POINTER(ctypes.c_double)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_uniform.argtypes = [ctypes.c_uint32]
        L.orc_uniform.restype = ctypes.c_double
        L.orc_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, dp_, dp_]
        L.orc_cholesky.argtypes = [ctypes.c_int, dp_, dp_]
        L.orc_cholesky.restype = ctypes.c_int
        L.orc_points.argtypes = [ctypes.POINTER(Model), ctypes.c_uint32, ctypes.c_int, dp_, dp_]
        L.orc_normals_path.argtypes = [ctypes.POINTER(Model), ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_int, dp_]
        L.orc_bridge_normals.argtypes = [ctypes.POINTER(Model), ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_uint32, dp_]
        L.orc_sigma.argtypes = [ctypes.POINTER(Model), ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_sigma.restype = ctypes.c_double
        L.orc_payoff.argtypes = [ctypes.POINTER(Model), dp_]
        L.orc_payoff.restype = ctypes.c_double
        L.orc_basis_eval.argtypes = [ctypes.POINTER(Model), ctypes.POINTER(Basis), dp_,
                                     ctypes.c_double, dp_, dp_, dp_, dp_, dp_]
        L.orc_path_a.argtypes = [ctypes.POINTER(Model), ctypes.POINTER(Basis), dp_, ctypes.c_double,
                                 dp_, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.POINTER(PathInfo)]
        L.orc_path_a.restype = ctypes.c_double
        L.orc_correction.argtypes = [ctypes.POINTER(Model), ctypes.POINTER(Basis), dp_, ctypes.c_int,
                                     u32p, dp_, dp_, ctypes.c_uint32, ctypes.c_int, dp_]
        L.orc_simulate_XT.argtypes = [ctypes.POINTER(Model), ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_double, dp_, ctypes.c_int, dp_, dp_, dp_]
        L.orc_samples.argtypes = [ctypes.POINTER(Model), ctypes.POINTER(Basis), dp_, ctypes.c_double,
                                  dp_, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, dp_]
        _LIB = L
    return _LIB


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------

def philox(ctr, key):
    """Philox4x32-10 of one counter (four uint32) under one key (two uint32)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def seed_key(seed):
    return [seed & 0xffffffff, (seed >> 32) & 0xffffffff]


def box_muller(w0, w1):
    z0, z1 = ctypes.c_double(), ctypes.c_double()
    lib().orc_box_muller(w0, w1, ctypes.byref(z0), ctypes.byref(z1))
    return z0.value, z1.value


def path_normals(cfg, k, i, path, count):
    z = np.zeros(count)
    lib().orc_normals_path(ctypes.byref(model(cfg)), k, i, path, count, _dptr(z))
    return z


# ---------------------------------------------------------------------------
# model
# ---------------------------------------------------------------------------

def correlation(cfg):
    d = cfg["d"]
    if "corr" in cfg and cfg["corr"] is not None:
        return np.array(cfg["corr"], dtype=np.float64).reshape(d, d)
    C = np.full((d, d), cfg["rho"])
    np.fill_diagonal(C, 1.0)
    return C


def cholesky(C):
    """Lower factor L with C = L L^T (orc_cholesky); raises if not PD."""
    d = C.shape[0]
    Cc = np.ascontiguousarray(C, dtype=np.float64)
    L = np.zeros((d, d))
    if lib().orc_cholesky(d, _dptr(Cc), _dptr(L)) != 0:
        raise ValueError("correlation matrix is not positive definite")
    return L


def model(cfg):
    d = cfg["d"]
    m = Model()
    m.d, m.N, m.M = d, cfg["N"], cfg["M"]
    m.payoff = 0 if cfg["payoff"] == "put" else 1
    m.obstacle = 0 if cfg.get("obstacle", "payoff") == "payoff" else 1
    vol = cfg["vol"]
    m.vol_kind = VOL_KINDS[vol["kind"]]
    m.T, m.r, m.lam, m.K = cfg["T"], cfg["r"], cfg["lambda"], cfg["K"]
    a = vol.get("a", 0.0)
    a = list(a) if isinstance(a, (list, tuple)) else [a] * d
    kap = vol.get("kappa", 0.0)
    kap = list(kap) if isinstance(kap, (list, tuple)) else [kap] * d
    for j in range(d):
        m.w[j] = cfg["weights"][j]
        m.va[j] = a[j]
        m.kappa[j] = kap[j]
        m.div[j] = cfg["div"][j]
    m.vb = vol.get("b", 0.0)
    m.s_dupire = vol.get("s", 0.0)
    C = correlation(cfg)
    L = cholesky(C)
    for r_ in range(d):
        for c_ in range(d):
            m.C[r_ * d + c_] = C[r_, c_]
            m.L[r_ * d + c_] = L[r_, c_]
    for v in range(d + 1):
        m.lo[v] = cfg["lo"][v]
        m.hi[v] = cfg["hi"][v]
    m.key[0], m.key[1] = seed_key(cfg["seed"])
    return m


# ---------------------------------------------------------------------------
# basis (Section 3.2.2)
# ---------------------------------------------------------------------------

def multi_index_set(dp, eta, q=1.0):
    """Multi-indices nu in N^{dp} with (sum nu_i^q)^{1/q} <= eta (eq. hyper_set;
    q = 1 gives total degree <= eta).  Graded order: total degree ascending,
    then lexicographic descending with variate 0 (time) most significant.
    The pseudo-norm test allows a relative slack of 1e-9 for q < 1."""
    by_degree = []
    for deg in range(eta + 1):
        out = []
        # all nu with |nu|_1 == deg, lexicographically descending
        def rec_exact(prefix, remaining, v):
            if v == dp - 1:
                out.append(tuple(prefix + [remaining]))
                return
            for e in range(remaining, -1, -1):
                rec_exact(prefix + [e], remaining - e, v + 1)
        rec_exact([], deg, 0)
        by_degree.extend(out)
    if q >= 1.0:
        return np.array(by_degree, dtype=np.int32).reshape(-1, dp)
    keep = []
    for nu in by_degree:
        s = sum(float(e) ** q for e in nu if e > 0)
        norm = s ** (1.0 / q) if s > 0 else 0.0
        if norm <= eta * (1.0 + 1e-9):
            keep.append(nu)
    return np.array(keep, dtype=np.int32).reshape(-1, dp)


def reduce_coords(cfg, t, x):
    """Map (t, x) to [-1,1]^{d'} (Section 3.2.2): returns xi of shape (d+1, n)."""
    lo = np.asarray(cfg["lo"], dtype=np.float64)
    hi = np.asarray(cfg["hi"], dtype=np.float64)
    Y = np.vstack([np.atleast_1d(np.asarray(t, dtype=np.float64))[None, :],
                   np.asarray(x, dtype=np.float64).reshape(cfg["d"], -1)])
    return (2.0 * Y - (lo + hi)[:, None]) / (hi - lo)[:, None]


def basis_matrix(cfg, nu, t, x):
    """B[i, l] = prod_v T_{nu_lv}(xi_v(t_i, x_i)) from numpy's Chebyshev
    Vandermonde matrices."""
    xi = reduce_coords(cfg, t, x)
    eta = int(nu.max()) if nu.size else 0
    n = xi.shape[1]
    B = np.ones((n, nu.shape[0]))
    for v in range(nu.shape[1]):
        V = npcheb.chebvander(xi[v], eta)  # (n, eta+1)
        B *= V[:, nu[:, v]]
    return B


def eval_u(cfg, nu, alpha, t, x):
    """u(t,x) and grad_x u(t,x) for arrays t (q,), x (d, q)."""
    xi = reduce_coords(cfg, t, x)
    lo = np.asarray(cfg["lo"]); hi = np.asarray(cfg["hi"])
    scale = 2.0 / (hi - lo)
    eta = int(nu.max()) if nu.size else 0
    dp = nu.shape[1]
    V = [npcheb.chebvander(xi[v], eta) for v in range(dp)]
    # derivative Vandermonde: column e holds T_e'
    Vd = []
    for v in range(dp):
        cols = []
        for e in range(eta + 1):
            c = np.zeros(eta + 1); c[e] = 1.0
            cols.append(npcheb.chebval(xi[v], npcheb.chebder(c)) if e > 0 else np.zeros_like(xi[v]))
        Vd.append(np.stack(cols, axis=1))
    B = np.ones((xi.shape[1], nu.shape[0]))
    for v in range(dp):
        B *= V[v][:, nu[:, v]]
    u = B @ alpha
    grads = []
    for j in range(1, dp):
        Bj = np.ones_like(B)
        for v in range(dp):
            Bj *= (Vd[v] if v == j else V[v])[:, nu[:, v]]
        grads.append(scale[j] * (Bj @ alpha))
    return u, np.array(grads)


def basis_struct(nu):
    nu_c = np.ascontiguousarray(nu, dtype=np.int32)
    b = Basis()
    b.p, b.dp = nu_c.shape
    b.eta = int(nu_c.max()) if nu_c.size else 0
    b.nu = nu_c.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    b._keep = nu_c
    return b


# ---------------------------------------------------------------------------
# Algorithm 2
# ---------------------------------------------------------------------------

def points(cfg, k, n=None):
    """The n random points (t_i, x_i) of iteration k: t (n,), x (d, n)."""
    n = cfg["n"] if n is None else n
    d = cfg["d"]
    t = np.zeros(n); x = np.zeros((d, n))
    m = model(cfg)
    lib().orc_points(ctypes.byref(m), k, n, _dptr(t), _dptr(x))
    return t, x


def path_detail(cfg, nu, alpha, ti, xi, k, i, path):
    m = model(cfg); b = basis_struct(nu)
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    xv = np.ascontiguousarray(xi, dtype=np.float64)
    info = PathInfo()
    lib().orc_path_a(ctypes.byref(m), ctypes.byref(b), _dptr(al), ti, _dptr(xv), k, i, path,
                     ctypes.byref(info))
    return info


def samples(cfg, nu, alpha, ti, xi, k, i, npaths=None):
    """The individual Monte Carlo samples a_m (m < npaths) of point i."""
    npaths = cfg["M"] if npaths is None else npaths
    m = model(cfg); b = basis_struct(nu)
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    xv = np.ascontiguousarray(xi, dtype=np.float64)
    a = np.zeros(npaths)
    lib().orc_samples(ctypes.byref(m), ctypes.byref(b), _dptr(al), float(ti), _dptr(xv), k, i,
                      npaths, _dptr(a))
    return a


def simulate(cfg, k, i, ti, xi, npaths):
    """X_T, X_tau (npaths, d) and tau (npaths,) of the paths of point i."""
    d = cfg["d"]
    XT = np.zeros((npaths, d)); Xtau = np.zeros((npaths, d)); tau = np.zeros(npaths)
    m = model(cfg)
    xv = np.ascontiguousarray(xi, dtype=np.float64)
    lib().orc_simulate_XT(ctypes.byref(m), k, i, float(ti), _dptr(xv), npaths, _dptr(XT),
                          _dptr(Xtau), _dptr(tau))
    return XT, Xtau, tau


def basis_eval(cfg, nu, alpha, t, x):
    """u, d_t u, grad_x u, Hessian_x u at one point by oracle.c."""
    d = cfg["d"]
    m = model(cfg); b = basis_struct(nu)
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    u, ut = ctypes.c_double(), ctypes.c_double()
    ux = np.zeros(d); uxx = np.zeros(d * d)
    lib().orc_basis_eval(ctypes.byref(m), ctypes.byref(b), _dptr(al), float(t), _dptr(xv),
                         ctypes.byref(u), ctypes.byref(ut), _dptr(ux), _dptr(uxx))
    return u.value, ut.value, ux, uxx.reshape(d, d)


def correction(cfg, nu, alpha, k, idx, t, x, nthreads=None):
    """c^k_i of eq. chat at the points with global indices idx (their
    coordinates t[idx], x[:, idx] given in the same order)."""
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    m = model(cfg); b = basis_struct(nu)
    idx_c = np.ascontiguousarray(idx, dtype=np.uint32)
    tt = np.ascontiguousarray(t, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64).reshape(cfg["d"], -1)
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    c = np.zeros(len(idx_c))
    lib().orc_correction(ctypes.byref(m), ctypes.byref(b), _dptr(al), len(idx_c),
                         idx_c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                         _dptr(tt), _dptr(xx), k, int(nthreads), _dptr(c))
    return c


def fit(B, y):
    """eq. alpha: argmin_alpha sum_i |y_i - sum_l alpha_l B_l(t_i,x_i)|^2."""
    return np.linalg.lstsq(B, y, rcond=None)[0]


def iteration(cfg, nu, alpha, k, nthreads=None):
    """One pass k -> k+1 of Algorithm 2 from alpha^k: the points, c^k, u^k at
    the points and alpha^{k+1}."""
    t, x = points(cfg, k)
    n = len(t)
    c = correction(cfg, nu, alpha, k, np.arange(n), t, x, nthreads)
    B = basis_matrix(cfg, nu, t, x)
    u = B @ alpha
    alpha_next = fit(B, u + c)
    return {"t": t, "x": x, "c": c, "u": u, "B": B, "alpha": alpha_next}


def price_delta(cfg, nu, alpha, t0=0.0, S0=None):
    """Price u(t0, log S0) and delta dV/dS_j = (du/dx_j)/S_j (Sections 5.1 and 5.3,
    Delta = grad_x V, read on the price scale)."""
    S0 = cfg["S0"] if S0 is None else S0
    x0 = np.log(np.asarray(S0, dtype=np.float64)).reshape(cfg["d"], 1)
    u, g = eval_u(cfg, nu, np.asarray(alpha), np.array([t0]), x0)
    return float(u[0]), (g[:, 0] / np.asarray(S0, dtype=np.float64))


def solve(cfg, nthreads=None, K_it=None):
    """Algorithm 2 from alpha^0 = 0 for K_it iterations."""
    nu = multi_index_set(cfg["d"] + 1, cfg["eta"], cfg.get("q", 1.0))
    alpha = np.zeros(nu.shape[0])
    hist = []
    K_it = cfg["K_it"] if K_it is None else K_it
    for k in range(K_it):
        it = iteration(cfg, nu, alpha, k, nthreads)
        dalpha = it["alpha"] - alpha
        alpha = it["alpha"]
        pr, de = price_delta(cfg, nu, alpha)
        hist.append({"price": pr, "delta": de, "resid_l2": float(np.linalg.norm(dalpha))})
    pr, de = price_delta(cfg, nu, alpha)
    return {"alpha": alpha, "nu": nu, "price": pr, "delta": de, "history": hist}
