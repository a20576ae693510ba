"""ctypes front end of the FP64 CPU oracle (oracle/nbm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the cpu_baseline / reference legs of ``bench.py``.  The product
package never imports it, and it never imports the product package.

``build()`` compiles nbm_oracle.c with gcc (FP64, OpenMP) into
``oracle/_build/libnbm_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nbm_oracle.c")
HDR = os.path.join(HERE, "nbm_oracle.h")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libnbm_oracle.so")

GEOM_SPHERE, GEOM_FLOWER, GEOM_ALL_PLUS, GEOM_ALL_MINUS, GEOM_GRID = 1, 2, 3, 4, 5

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, OpenMP); returns the library path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
             "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Problem(C.Structure):
    _fields_ = [
        ("geometry", C.c_int32), ("n_hidden", C.c_int32), ("width", C.c_int32),
        ("pad0", C.c_int32),
        ("r0", C.c_double), ("amp", C.c_double), ("lobes_theta", C.c_double),
        ("lobes_psi", C.c_double),
        ("mu_minus", C.c_double), ("mu_plus", C.c_double), ("k_minus", C.c_double),
        ("k_plus", C.c_double),
        ("h", C.c_double), ("lambda_jump", C.c_double),
        ("solution", C.c_int32), ("activation", C.c_int32),
        ("phi_n", C.c_int32), ("pad1", C.c_int32), ("phi_grid", C.POINTER(C.c_double)),
    ]

SOL_BENCH, SOL_SEC41 = 0, 1
ACT_TANH, ACT_SIN = 0, 1


class PointTerms(C.Structure):
    _fields_ = [("B", C.c_double), ("D", C.c_double), ("J", C.c_double), ("r2", C.c_double),
                ("has_jump", C.c_int32), ("cut", C.c_int32)]


class Cell(C.Structure):
    _fields_ = [("cut", C.c_int32), ("phase", C.c_int32), ("V", C.c_double * 2),
                ("A", (C.c_double * 6) * 2), ("S", C.c_double), ("centroid", C.c_double * 3),
                ("xg", C.c_double * 3)]


def make_problem(geometry=GEOM_SPHERE, n_hidden=2, width=64, r0=0.5, amp=0.1, lobes_theta=5.0,
                 lobes_psi=3.0, mu_minus=1.0, mu_plus=10.0, k_minus=0.0, k_plus=0.0, h=2.0 / 32,
                 lambda_jump=1.0, solution=SOL_BENCH, activation=ACT_TANH,
                 phi_grid=None) -> Problem:
    """phi_grid: for GEOM_GRID, the (n+1)^3 node values of the level set (x fastest)."""
    pr = Problem(geometry, n_hidden, width, 0, r0, amp, lobes_theta, lobes_psi, mu_minus,
                 mu_plus, k_minus, k_plus, h, lambda_jump, solution, activation)
    if phi_grid is not None:
        g = np.ascontiguousarray(phi_grid, dtype=np.float64).reshape(-1)
        n = round(len(g) ** (1.0 / 3.0)) - 1
        assert (n + 1) ** 3 == len(g) and n >= 1
        pr.phi_n = n
        pr.phi_grid = g.ctypes.data_as(C.POINTER(C.c_double))
        pr._phi_keep = g  # the array must outlive the problem
    return pr


_D = C.POINTER(C.c_double)
_P = C.POINTER(Problem)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            L.nbo_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
            L.nbo_phi.argtypes = [_P, _D]
            L.nbo_phi.restype = C.c_double
            L.nbo_grad_phi.argtypes = [_P, _D, _D]
            L.nbo_phase.argtypes = [_P, _D]
            L.nbo_phase.restype = C.c_int
            L.nbo_exact_u.argtypes = [_P, C.c_int, _D]
            L.nbo_exact_u.restype = C.c_double
            L.nbo_exact_grad_u.argtypes = [_P, C.c_int, _D, _D]
            L.nbo_rhs_f.argtypes = [_P, C.c_int, _D]
            L.nbo_rhs_f.restype = C.c_double
            L.nbo_mu.argtypes = [_P, C.c_int, _D]
            L.nbo_mu.restype = C.c_double
            for fn in ("nbo_alpha", "nbo_beta", "nbo_dirichlet_g"):
                getattr(L, fn).argtypes = [_P, _D]
                getattr(L, fn).restype = C.c_double
            L.nbo_cell_geometry.argtypes = [_P, _D, C.c_double, C.POINTER(Cell)]
            L.nbo_tri_fraction.argtypes = [C.c_double] * 3
            L.nbo_tri_fraction.restype = C.c_double
            L.nbo_tet_fraction.argtypes = [C.c_double] * 4
            L.nbo_tet_fraction.restype = C.c_double
            L.nbo_params_per_net.argtypes = [_P]
            L.nbo_params_per_net.restype = C.c_int64
            L.nbo_mlp_eval.argtypes = [_P, _D, _D]
            L.nbo_mlp_eval.restype = C.c_double
            L.nbo_sample_points.argtypes = [_P, C.c_uint64, C.c_int64, C.c_int64, C.c_int64, _D]
            L.nbo_point_terms_eval.argtypes = [_P, _D, _D, C.c_int, C.POINTER(PointTerms)]
            L.nbo_loss.argtypes = [_P, _D, _D, C.c_int64, _D, C.c_int]
            L.nbo_loss.restype = C.c_double
            L.nbo_loss_grad.argtypes = [_P, _D, _D, C.c_int64, _D, C.c_int]
            L.nbo_loss_grad.restype = C.c_double
            L.nbo_adam_step.argtypes = [_D, _D, _D, _D, C.c_int64, C.c_int64, C.c_double,
                                        C.c_double, C.c_double, C.c_double]
            L.nbo_train.argtypes = [_P, _D, _D, _D, C.c_int64, C.c_int, C.c_int64, C.c_int64,
                                    C.c_double, C.c_double, C.c_double, C.c_double, C.c_uint64,
                                    _D, C.c_int]
            L.nbo_default_threads.argtypes = []
            L.nbo_default_threads.restype = C.c_int
            L.nbo_eval_grid.argtypes = [_P, _D, C.c_int, _D, C.c_int]
            L.nbo_grid_assemble_dense.argtypes = [_P, C.c_int, _D, _D]
            L.nbo_grid_cg_solve.argtypes = [_P, C.c_int, C.c_double, C.c_int, _D,
                                            C.POINTER(C.c_int), _D, C.c_int]
            L.nbo_grid_error.argtypes = [_P, C.c_int, _D, _D, _D]
            L.nbo_jump_extrap.argtypes = [_P, _D, C.c_double, C.c_int, C.c_double, _D, _D, _D,
                                          C.POINTER(C.c_int)]
            L.nbo_fit_dn.argtypes = [_P, C.c_int, _D, C.c_int, _D, _D, _D]
            L.nbo_grid_solve_jump.argtypes = [_P, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                                              C.c_double, _D, C.POINTER(C.c_int), _D,
                                              C.POINTER(C.c_int), _D, C.c_int]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _vec(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().nbo_philox4x32_10(c, k, o)
    return list(o)


def phi(pr, x):
    return lib().nbo_phi(C.byref(pr), _dp(_vec(x)))


def grad_phi(pr, x):
    g = np.zeros(3)
    lib().nbo_grad_phi(C.byref(pr), _dp(_vec(x)), _dp(g))
    return g


def phase(pr, x):
    return lib().nbo_phase(C.byref(pr), _dp(_vec(x)))


def exact_u(pr, s, x):
    return lib().nbo_exact_u(C.byref(pr), s, _dp(_vec(x)))


def exact_grad_u(pr, s, x):
    g = np.zeros(3)
    lib().nbo_exact_grad_u(C.byref(pr), s, _dp(_vec(x)), _dp(g))
    return g


def mu(pr, s, x):
    return lib().nbo_mu(C.byref(pr), s, _dp(_vec(x)))


def rhs_f(pr, s, x):
    return lib().nbo_rhs_f(C.byref(pr), s, _dp(_vec(x)))


def alpha(pr, x):
    return lib().nbo_alpha(C.byref(pr), _dp(_vec(x)))


def beta(pr, x):
    return lib().nbo_beta(C.byref(pr), _dp(_vec(x)))


def cell_geometry(pr, p, h=None):
    c = Cell()
    lib().nbo_cell_geometry(C.byref(pr), _dp(_vec(p)), pr.h if h is None else h, C.byref(c))
    return {
        "cut": c.cut, "phase": c.phase, "V": np.array(list(c.V)),
        "A": np.array([list(c.A[0]), list(c.A[1])]), "S": c.S,
        "centroid": np.array(list(c.centroid)), "xg": np.array(list(c.xg)),
    }


def tri_fraction(f0, f1, f2):
    return lib().nbo_tri_fraction(f0, f1, f2)


def tet_fraction(f0, f1, f2, f3):
    return lib().nbo_tet_fraction(f0, f1, f2, f3)


def params_per_net(pr):
    return int(lib().nbo_params_per_net(C.byref(pr)))


def mlp_eval(pr, theta_net, x):
    return lib().nbo_mlp_eval(C.byref(pr), _dp(_vec(theta_net)), _dp(_vec(x)))


def sample_points(pr, seed, step, n, n_band=0):
    pts = np.zeros((n, 3))
    lib().nbo_sample_points(C.byref(pr), seed, step, n, n_band, _dp(pts))
    return pts


def point_terms(pr, theta, p, mode=0):
    t = PointTerms()
    th = _vec(theta) if theta is not None else np.zeros(1)
    lib().nbo_point_terms_eval(C.byref(pr), _dp(th), _dp(_vec(p)), mode, C.byref(t))
    return {"B": t.B, "D": t.D, "J": t.J, "r2": t.r2, "has_jump": t.has_jump, "cut": t.cut}


def loss(pr, theta, pts, n_threads=0, want_r2=False):
    pts = _vec(pts).reshape(-1, 3)
    r2 = np.zeros(len(pts)) if want_r2 else None
    L = lib().nbo_loss(C.byref(pr), _dp(_vec(theta)), _dp(pts), len(pts),
                       _dp(r2) if r2 is not None else None, n_threads)
    return (L, r2) if want_r2 else L


def loss_grad(pr, theta, pts, n_threads=0):
    pts = _vec(pts).reshape(-1, 3)
    g = np.zeros(2 * params_per_net(pr))
    L = lib().nbo_loss_grad(C.byref(pr), _dp(_vec(theta)), _dp(pts), len(pts), _dp(g), n_threads)
    return L, g


def level_problem(pr, level):
    """Copy of `pr` whose implicit cell has spacing h / 2^level."""
    q = Problem.from_buffer_copy(pr)
    q.h = pr.h / 2.0 ** level
    if hasattr(pr, "_phi_keep"):
        q._phi_keep = pr._phi_keep
    return q


# Implicit refinement (Sec. 3 and Fig. 2: implicit cells at several resolutions;
# Sec. 4.2: a base resolution implicitly refined three times).  The paper does
# not say how the levels' rows are combined; the reading taken here stacks the
# rows of every level into the point's residual vector, so that r_p^2 (and the
# loss) is the sum over the levels l = 0..levels of the single-level r_p^2 of the
# cell of spacing h / 2^l around the same point.


def loss_levels(pr, levels, theta, pts, n_threads=0, want_r2=False):
    total, r2s = 0.0, None
    for lv in range(levels + 1):
        L, r2 = loss(level_problem(pr, lv), theta, pts, n_threads, want_r2=True)
        total += L
        r2s = r2 if r2s is None else r2s + r2
    return (total, r2s) if want_r2 else total


def loss_grad_levels(pr, levels, theta, pts, n_threads=0):
    total, g = 0.0, None
    for lv in range(levels + 1):
        L, gl = loss_grad(level_problem(pr, lv), theta, pts, n_threads)
        total += L
        g = gl if g is None else g + gl
    return total, g


def adam_step(theta, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    lib().nbo_adam_step(_dp(theta), _dp(m), _dp(v), _dp(_vec(grad)), len(theta), t, lr, beta1,
                        beta2, eps)


def train(pr, theta, m, v, step0, n_steps, batch, n_band, lr=1e-3, beta1=0.9, beta2=0.999,
          eps=1e-8, seed=1, n_threads=0):
    hist = np.zeros(n_steps)
    lib().nbo_train(C.byref(pr), _dp(theta), _dp(m), _dp(v), step0, n_steps, batch, n_band, lr,
                    beta1, beta2, eps, seed, _dp(hist), n_threads)
    return hist


def default_threads():
    """Threads the oracle's parallel loops use when n_threads = 0."""
    return lib().nbo_default_threads()


def eval_grid(pr, theta, n, n_threads=0):
    u = np.zeros((n + 1) ** 3)
    lib().nbo_eval_grid(C.byref(pr), _dp(_vec(theta)), n, _dp(u), n_threads)
    return u


def grid_assemble_dense(pr, n):
    m = (n - 1) ** 3
    A = np.zeros((m, m))
    b = np.zeros(m)
    lib().nbo_grid_assemble_dense(C.byref(pr), n, _dp(A), _dp(b))
    return A, b


def grid_cg_solve(pr, n, rtol=1e-10, max_iter=10000, n_threads=0):
    u = np.zeros((n + 1) ** 3)
    it = C.c_int(0)
    rr = C.c_double(0)
    st = lib().nbo_grid_cg_solve(C.byref(pr), n, rtol, max_iter, _dp(u), C.byref(it),
                                 C.byref(rr), n_threads)
    return st, u, it.value, rr.value


def grid_error(pr, n, u):
    a = C.c_double(0)
    b = C.c_double(0)
    lib().nbo_grid_error(C.byref(pr), n, _dp(_vec(u)), C.byref(a), C.byref(b))
    return a.value, b.value


JUMP_EXACT, JUMP_EXTRAP, JUMP_FIRST_ORDER = 0, 1, 2


def jump_extrap(pr, x, h, dn_small=None):
    """Extrapolated node jump at x: (in_band, J, x_G, n, small side); dn_small
    None drops the lag term (G = beta / mu_big)."""
    J = C.c_double(0)
    xg = np.zeros(3)
    nrm = np.zeros(3)
    ss = C.c_int(0)
    rc = lib().nbo_jump_extrap(C.byref(pr), _dp(_vec(x)), h, 0 if dn_small is None else 1,
                               0.0 if dn_small is None else float(dn_small), C.byref(J), _dp(xg),
                               _dp(nrm), C.byref(ss))
    return rc == 0, J.value, xg, nrm, ss.value


def fit_dn(pr, n, u, s, xg, nrm):
    dn = C.c_double(0)
    rc = lib().nbo_fit_dn(C.byref(pr), n, _dp(_vec(u)), s, _dp(_vec(xg)), _dp(_vec(nrm)),
                          C.byref(dn))
    return (dn.value if rc == 0 else None)


def grid_solve_jump(pr, n, mode, rtol=1e-10, max_iter=10000, max_passes=10, jtol=1e-6,
                    n_threads=0):
    u = np.zeros((n + 1) ** 3)
    it = C.c_int(0)
    rr = C.c_double(0)
    ps = C.c_int(0)
    dj = C.c_double(0)
    st = lib().nbo_grid_solve_jump(C.byref(pr), n, mode, rtol, max_iter, max_passes, jtol, _dp(u),
                                   C.byref(it), C.byref(rr), C.byref(ps), C.byref(dj), n_threads)
    return st, u, it.value, rr.value, ps.value, dj.value
