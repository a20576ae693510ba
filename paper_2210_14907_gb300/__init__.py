"""GB300 (sm_103a) implementation of the fused NBM collocation-residual step.

The Neural Bootstrapping Method (arXiv 2210.14907, Sec. 3) trains two networks,
one per side of a level-set interface, on the residual of a finite-volume
discretization evaluated at random collocation points.  All compute runs in
the CUDA library ``libnbm.so`` (C ABI in ``include/nbm.h``); this module only
marshals torch tensors (device memory, streams) into those calls.  There is no
CPU fallback: importing the package without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import torch

from . import build as _build

__all__ = ["ProblemDesc", "Problem", "NBMLoss", "load_library", "config", "param_count",
           "xavier_init", "save_checkpoint", "load_checkpoint", "GEOM_SPHERE", "GEOM_FLOWER",
           "GEOM_ALL_PLUS", "GEOM_ALL_MINUS", "GEOM_GRID", "PREC_FP32", "PREC_BF16",
           "PREC_FP16", "SOL_BENCH", "SOL_SEC41", "ACT_TANH", "ACT_SIN", "JUMP_EXACT",
           "JUMP_EXTRAP", "JUMP_FIRST_ORDER", "NBMError"]

GEOM_SPHERE, GEOM_FLOWER, GEOM_ALL_PLUS, GEOM_ALL_MINUS, GEOM_GRID = 1, 2, 3, 4, 5
PREC_FP32, PREC_BF16, PREC_FP16 = 0, 1, 2
SOL_BENCH, SOL_SEC41 = 0, 1
ACT_TANH, ACT_SIN = 0, 1
JUMP_EXACT, JUMP_EXTRAP, JUMP_FIRST_ORDER = 0, 1, 2

STATUS = {0: "NBM_OK", 1: "NBM_ERR_INVALID_ARG", 2: "NBM_ERR_CUDA", 3: "NBM_ERR_NOT_CONVERGED",
          4: "NBM_ERR_NONFINITE", 5: "NBM_ERR_OOM", 6: "NBM_ERR_DEVICE_TIMEOUT"}


class NBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Desc(C.Structure):
    _fields_ = [("geometry", C.c_int32), ("n_hidden", C.c_int32), ("width", C.c_int32),
                ("precision", C.c_int32), ("r0", C.c_double), ("amp", C.c_double),
                ("lobes_theta", C.c_double), ("lobes_psi", C.c_double),
                ("mu_minus", C.c_double), ("mu_plus", C.c_double), ("k_minus", C.c_double),
                ("k_plus", C.c_double), ("h", C.c_double), ("lambda_jump", C.c_double),
                ("band_fraction", C.c_double), ("fp64_stencil", C.c_int32),
                ("refine_levels", C.c_int32), ("solution", C.c_int32),
                ("activation", C.c_int32), ("grid_jump", C.c_int32), ("reserved0", C.c_int32)]


@dataclasses.dataclass
class ProblemDesc:
    """Problem of Sec. 2 plus the NBM settings of Sec. 3 (see include/nbm.h)."""
    geometry: int = GEOM_SPHERE
    n_hidden: int = 2
    width: int = 64
    precision: int = PREC_FP32
    r0: float = 0.5
    amp: float = 0.1
    lobes_theta: float = 5.0
    lobes_psi: float = 3.0
    mu_minus: float = 1.0
    mu_plus: float = 10.0
    k_minus: float = 0.0
    k_plus: float = 0.0
    h: float = 2.0 / 32
    lambda_jump: float = 1.0
    band_fraction: float = 0.0
    fp64_stencil: int = -1
    refine_levels: int = 0  # implicit refinement: also the cells of spacing h/2, ..., h/2^levels
    solution: int = 0       # SOL_BENCH, or SOL_SEC41 (variable mu, the convergence study)
    activation: int = 0     # ACT_TANH, or ACT_SIN (FP32 path, width <= 32)
    grid_jump: int = 0      # node jump of the grid solvers: JUMP_EXACT, JUMP_EXTRAP, JUMP_FIRST_ORDER

    def to_c(self) -> _Desc:
        return _Desc(self.geometry, self.n_hidden, self.width, self.precision, self.r0,
                     self.amp, self.lobes_theta, self.lobes_psi, self.mu_minus, self.mu_plus,
                     self.k_minus, self.k_plus, self.h, self.lambda_jump, self.band_fraction,
                     self.fp64_stencil, self.refine_levels, self.solution, self.activation,
                     self.grid_jump, 0)


def config(name: str, precision: int | None = None) -> ProblemDesc:
    """The five benchmark workloads (C1..C5)."""
    if name == "C1":  # small FP32 check: sphere, 3->64->64->1, h = 2/32
        d = ProblemDesc(GEOM_SPHERE, 2, 64, PREC_FP32, mu_minus=1.0, mu_plus=10.0, h=2.0 / 32)
    elif name == "C2":  # mixed precision: 3->128^3->1, h = 2/128
        d = ProblemDesc(GEOM_SPHERE, 3, 128, PREC_BF16, mu_minus=1.0, mu_plus=10.0, h=2.0 / 128)
    elif name in ("C3", "C5"):  # flower, mu 1/100, 3->128^4->1, h = 2/256, 30 % band points
        d = ProblemDesc(GEOM_FLOWER, 4, 128, PREC_BF16, mu_minus=1.0, mu_plus=100.0,
                        h=2.0 / 256, band_fraction=0.3)
    elif name == "C4":  # fine resolution: sphere, h = 2/1024, FP64 stencil combination
        d = ProblemDesc(GEOM_SPHERE, 4, 128, PREC_BF16, mu_minus=1.0, mu_plus=10.0,
                        h=2.0 / 1024, fp64_stencil=1)
    else:
        raise ValueError(name)
    if precision is not None:
        d.precision = precision
    return d


BATCH = {"C1": 4096, "C2": 262_144, "C3": 1_048_576, "C4": 4_194_304, "C5": 1_048_576}


def param_count(d: ProblemDesc) -> int:
    H = d.width
    return 2 * (4 * H + (d.n_hidden - 1) * (H * H + H) + H + 1)


def save_checkpoint(path, desc: ProblemDesc, params, m, v, step: int, seed: int) -> None:
    """Everything a training run needs to continue bitwise: the descriptor, the
    parameters, Adam's m and v, the number of steps taken and the Philox key (the
    points of step t are drawn at counter t, so no generator state is kept)."""
    torch.save({"desc": dataclasses.asdict(desc), "params": params.detach().cpu(),
                "m": m.detach().cpu(), "v": v.detach().cpu(), "step": int(step),
                "seed": int(seed)}, path)


def load_checkpoint(path, device="cuda"):
    """Returns (desc, params, m, v, step, seed) as saved by save_checkpoint."""
    c = torch.load(path, map_location="cpu")
    return (ProblemDesc(**c["desc"]), c["params"].to(device), c["m"].to(device),
            c["v"].to(device), c["step"], c["seed"])


def xavier_init(d: ProblemDesc, seed: int = 0, device="cpu") -> torch.Tensor:
    """Glorot-uniform weights, zero biases, for both networks (flat FP32 vector)."""
    g = torch.Generator().manual_seed(seed)
    H = d.width
    parts = []
    for _ in range(2):
        dims = [(3, H)] + [(H, H)] * (d.n_hidden - 1) + [(H, 1)]
        for fan_in, fan_out in dims:
            a = (6.0 / (fan_in + fan_out)) ** 0.5
            parts.append((torch.rand(fan_in * fan_out, generator=g, dtype=torch.float64) * 2 - 1) * a)
            parts.append(torch.zeros(fan_out, dtype=torch.float64))
    return torch.cat(parts).to(torch.float32).to(device)


_lib = None


def load_library(build_if_missing: bool = True):
    """Loads libnbm.so (building it with nvcc if needed).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise ImportError(f"libnbm.so not built at {path}")
        _build.build()
    L = C.CDLL(path)
    P = C.c_void_p
    L.nbm_last_error.restype = C.c_char_p
    L.nbm_init_problem.argtypes = [C.POINTER(_Desc), C.POINTER(C.c_void_p)]
    L.nbm_destroy.argtypes = [P]
    L.nbm_param_count.argtypes = [P]
    L.nbm_param_count.restype = C.c_int64
    L.nbm_sample_points.argtypes = [P, C.c_uint64, C.c_int64, C.c_int64, P, P]
    L.nbm_residual.argtypes = [P, P, P, C.c_int64, C.c_uint64, C.c_int64, P,
                               C.POINTER(C.c_double), P]
    L.nbm_loss_grad.argtypes = [P, P, P, C.c_int64, C.c_uint64, C.c_int64, P,
                                C.POINTER(C.c_double), P]
    L.nbm_train_steps.argtypes = [P, P, P, P, C.POINTER(C.c_int64), C.c_int, C.c_int64,
                                  C.c_float, C.c_float, C.c_float, C.c_float, C.c_uint64, P, P, P]
    L.nbm_loss_grad_shard.argtypes = [P, P, P, C.c_int64, C.c_int64, C.c_int64, C.c_uint64,
                                      C.c_int64, P, P, P]
    L.nbm_adam_step.argtypes = [P, P, P, P, P, C.POINTER(C.c_int64), C.c_float, C.c_float,
                                C.c_float, C.c_float, P, P]
    L.nbm_set_level_set.argtypes = [P, P, C.c_int, P]
    L.nbm_selftest_bounded_wait.argtypes = [C.c_int64, P]
    L.nbm_profile.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.nbm_profile.restype = C.c_int
    L.nbm_eval_grid.argtypes = [P, P, C.c_int, C.c_int, P, P]
    L.nbm_eval_points.argtypes = [P, P, P, C.c_int64, C.c_int, P, P]
    L.nbm_eval_points.restype = C.c_int
    L.nbm_grid_cg_solve.argtypes = [P, C.c_int, C.c_double, C.c_int, P, C.POINTER(C.c_int),
                                    C.POINTER(C.c_double), P]
    L.nbm_grid_solve_refined.argtypes = L.nbm_grid_cg_solve.argtypes
    L.nbm_grid_last_jump_info.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_double),
                                          C.POINTER(C.c_int)]
    L.nbm_grid_node_jump.argtypes = [P, C.c_int, C.c_int, P, P, P]
    L.nbm_grid_node_jump.restype = C.c_int
    L.nbm_grid_last_jump_info.restype = C.c_int
    for fn in ("nbm_init_problem", "nbm_destroy", "nbm_sample_points", "nbm_residual",
               "nbm_loss_grad", "nbm_loss_grad_shard", "nbm_adam_step", "nbm_train_steps",
               "nbm_eval_grid", "nbm_grid_cg_solve",
               "nbm_grid_solve_refined",
               "nbm_set_level_set", "nbm_selftest_bounded_wait"):
        getattr(L, fn).restype = C.c_int
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise NBMError(rc, _lib.nbm_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(t, dtype=torch.float32):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor")
    return t


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Problem:
    """One NBM problem on the current CUDA device (owns libnbm's workspace)."""

    def __init__(self, desc: ProblemDesc):
        self.lib = load_library()
        self.desc = desc
        h = C.c_void_p()
        self._cdesc = desc.to_c()
        _check(self.lib.nbm_init_problem(C.byref(self._cdesc), C.byref(h)))
        self.handle = h
        self.P = int(self.lib.nbm_param_count(h))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.nbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_level_set(self, phi, n, stream=None):
        """Level set on a coarse mesh (GEOM_GRID): the (n+1)^3 node values, x fastest."""
        phi = _dev(phi, torch.float64)
        if phi.numel() != (n + 1) ** 3:
            raise ValueError("phi needs (n+1)^3 node values")
        _check(self.lib.nbm_set_level_set(self.handle, _ptr(phi), n, _stream(stream)))

    def sample_points(self, n, seed=1, step=1, stream=None):
        out = torch.empty(n, 3, device="cuda", dtype=torch.float32)
        _check(self.lib.nbm_sample_points(self.handle, seed, step, n, _ptr(out), _stream(stream)))
        return out

    def residual(self, params, pts=None, n=None, seed=1, step=1, want_r2=True, stream=None):
        _dev(params)
        _dev(pts)
        n = pts.shape[0] if pts is not None else n
        r2 = torch.empty(n, device="cuda", dtype=torch.float32) if want_r2 else None
        loss = C.c_double(0.0)
        _check(self.lib.nbm_residual(self.handle, _ptr(params), _ptr(pts), n, seed, step,
                                     _ptr(r2), C.byref(loss), _stream(stream)))
        return loss.value, r2

    def loss_grad(self, params, pts=None, n=None, seed=1, step=1, grad=None, stream=None,
                  sync=True):
        _dev(params)
        _dev(pts)
        n = pts.shape[0] if pts is not None else n
        if grad is None:
            grad = torch.empty(self.P, device="cuda", dtype=torch.float32)
        loss = C.c_double(0.0)
        _check(self.lib.nbm_loss_grad(self.handle, _ptr(params), _ptr(pts), n, seed, step,
                                      _ptr(grad), C.byref(loss) if sync else None,
                                      _stream(stream)))
        return (loss.value if sync else None), grad

    def loss_grad_shard(self, params, n_total, first, n, seed=1, step=1, pts=None, grad=None,
                        loss=None, stream=None):
        """Points first .. first+n-1 of the step's n_total-point batch: returns
        (loss, grad), both scaled by 1/n_total and left on the device (loss is
        a one-element FP64 tensor), so that their sums over a partition of the
        batch are the whole batch's loss and gradient.  Asynchronous."""
        _dev(params)
        _dev(pts)
        if grad is None:
            grad = torch.empty(self.P, device=params.device, dtype=torch.float32)
        if loss is None:
            loss = torch.empty(1, device=params.device, dtype=torch.float64)
        _dev(grad)
        _dev(loss, torch.float64)
        _check(self.lib.nbm_loss_grad_shard(self.handle, _ptr(params), _ptr(pts), n_total, first,
                                            n, seed, step, _ptr(grad), _ptr(loss),
                                            _stream(stream)))
        return loss, grad

    def adam_step(self, params, m, v, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                  loss=None, stream=None):
        """Adam update step+1 with the given gradient (skipped when the device
        scalar `loss` is given and not finite); returns step + 1."""
        for t in (params, m, v, grad):
            _dev(t)
        _dev(loss, torch.float64)
        st = C.c_int64(step)
        _check(self.lib.nbm_adam_step(self.handle, _ptr(params), _ptr(m), _ptr(v), _ptr(grad),
                                      C.byref(st), lr, beta1, beta2, eps, _ptr(loss),
                                      _stream(stream)))
        return st.value

    def train_steps(self, params, m, v, step, n_steps, batch, lr=1e-3, beta1=0.9, beta2=0.999,
                    eps=1e-8, seed=1, loss_hist=None, pts=None, stream=None):
        for t in (params, m, v):
            _dev(t)
        _dev(pts)
        st = C.c_int64(step)
        _check(self.lib.nbm_train_steps(self.handle, _ptr(params), _ptr(m), _ptr(v),
                                        C.byref(st), n_steps, batch, lr, beta1, beta2, eps, seed,
                                        _ptr(pts), _ptr(loss_hist), _stream(stream)))
        return st.value

    def profile(self, enable):
        """enable=True starts timing the fused kernel; enable=False returns (ms, launches)."""
        ms = C.c_double(0.0)
        n = C.c_int64(0)
        _check(self.lib.nbm_profile(self.handle, 1 if enable else 0, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def eval_grid(self, params, n, precision=PREC_FP16, out=None, stream=None):
        _dev(params)
        if out is None:
            out = torch.empty((n + 1) ** 3, device="cuda", dtype=torch.float32)
        _check(self.lib.nbm_eval_grid(self.handle, _ptr(params), n, precision, _ptr(out),
                                      _stream(stream)))
        return out

    def eval_points(self, params, pts, precision=PREC_FP32, out=None, stream=None):
        _dev(params)
        _dev(pts)
        if out is None:
            out = torch.empty(pts.shape[0], device="cuda", dtype=torch.float32)
        _check(self.lib.nbm_eval_points(self.handle, _ptr(params), _ptr(pts), pts.shape[0],
                                        precision, _ptr(out), _stream(stream)))
        return out

    def grid_cg_solve(self, n, rtol=1e-10, max_iter=20000, out=None, stream=None):
        if out is None:
            out = torch.empty((n + 1) ** 3, device="cuda", dtype=torch.float64)
        it = C.c_int(0)
        rr = C.c_double(0.0)
        rc = self.lib.nbm_grid_cg_solve(self.handle, n, rtol, max_iter, _ptr(out), C.byref(it),
                                        C.byref(rr), _stream(stream))
        if rc not in (0, 3):
            _check(rc)
        return out, it.value, rr.value, rc == 0

    @staticmethod
    def grid_jump_info():
        """(passes, max |J_new - J| of the last pass, fell_back) of this thread's
        last grid solve; passes is 1 for the exact and first-order jumps."""
        ps, dj, fb = C.c_int(0), C.c_double(0.0), C.c_int(0)
        _check(load_library().nbm_grid_last_jump_info(C.byref(ps), C.byref(dj), C.byref(fb)))
        return ps.value, dj.value, bool(fb.value)

    def grid_node_jump(self, n, mode, u=None, out=None, stream=None):
        """The grid scheme's value jump u+ - u- at the (n+1)^3 nodes for grid_jump
        mode `mode` (JUMP_EXTRAP fits the small-mu side's normal derivative
        from the node values u)."""
        _dev(u, torch.float64)
        if out is None:
            out = torch.empty((n + 1) ** 3, device="cuda", dtype=torch.float64)
        _check(self.lib.nbm_grid_node_jump(self.handle, n, mode, _ptr(u), _ptr(out),
                                           _stream(stream)))
        return out

    def grid_solve_refined(self, n, rtol=1e-10, max_iter=20000, out=None, stream=None):
        """The grid system of grid_cg_solve to the same FP64 residual test, by
        FP32 inner PCG corrections of FP64 residuals (iterative refinement)."""
        if out is None:
            out = torch.empty((n + 1) ** 3, device="cuda", dtype=torch.float64)
        it = C.c_int(0)
        rr = C.c_double(0.0)
        rc = self.lib.nbm_grid_solve_refined(self.handle, n, rtol, max_iter, _ptr(out),
                                             C.byref(it), C.byref(rr), _stream(stream))
        if rc not in (0, 3):
            _check(rc)
        return out, it.value, rr.value, rc == 0


class NBMLoss(torch.autograd.Function):
    """loss = NBMLoss.apply(problem, params, pts): mean r_p^2 of Sec. 3 as a
    differentiable function of the network parameters.

    When a gradient can be needed (grad mode on and params requiring it) the
    forward runs nbm_loss_grad, which computes the loss and libnbm's
    hand-written backward in one pass, and keeps the gradient for backward;
    otherwise it runs the forward-only nbm_residual.  The loss is not
    differentiated with respect to the collocation points: pts that require
    a gradient are refused."""

    @staticmethod
    def forward(ctx, problem, params, pts):
        if pts.requires_grad:
            raise ValueError("NBMLoss does not differentiate with respect to the collocation "
                             "points; pass pts.detach()")
        p = params.detach().contiguous()
        x = pts.detach().contiguous()
        if ctx.needs_input_grad[1]:
            loss, grad = problem.loss_grad(p, x)
            ctx.save_for_backward(grad)
        else:
            loss, _ = problem.residual(p, x, want_r2=False)
        return torch.tensor(loss, dtype=torch.float64, device=params.device)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return None, grad * gout.to(grad.dtype), None
