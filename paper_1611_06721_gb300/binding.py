"""ctypes binding of ``libmqs.so`` (argument marshalling only).

Every compute step runs in the CUDA library; this module converts numpy
arrays (host calls) or torch CUDA tensors (``*_dev`` calls) to plain pointers
and sizes.  Loading fails loudly if the compiled library is absent: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import weakref
import os
from dataclasses import dataclass, replace

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MQS_DEBUG=1 loads the debug variant (bounds-checked kernel indices, guard bytes
# after every device buffer; build it with build.build(debug=True))
DEBUG = os.environ.get("MQS_DEBUG", "") not in ("", "0")
LIB_PATH = os.path.join(HERE, "_lib_debug" if DEBUG else "_lib", "libmqs.so")

MQS_OK = 0
ERRORS = {-1: "MQS_ERR_ARG", -2: "MQS_ERR_CUDA", -3: "MQS_ERR_OOM", -4: "MQS_ERR_NOT_CONVERGED",
          -5: "MQS_ERR_BREAKDOWN", -6: "MQS_ERR_NAN", -7: "MQS_ERR_UNSTABLE", -8: "MQS_ERR_TIMEOUT",
          -9: "MQS_ERR_UNIMPLEMENTED", -10: "MQS_ERR_HALTED"}
START_ZERO, START_PREV, START_SPE, START_POD, START_CSPE = 0, 1, 2, 3, 4

EXPORTS = ("mqs_setup", "mqs_destroy", "mqs_last_error", "mqs_layout", "mqs_set_dt", "mqs_get_dt",
           "mqs_set_options", "mqs_lambda_max", "mqs_step", "mqs_step_enqueue", "mqs_step_finish",
           "mqs_get_state", "mqs_set_state", "mqs_get_state_dev", "mqs_set_state_dev", "mqs_get_solution",
           "mqs_reset_history", "pcg_solve", "pcg_solve_dev", "mqs_apply_kn", "mqs_apply_kn_dev",
           "mqs_conductor_rate", "mqs_push_history", "spe_start", "pod_basis", "pod_start", "mqs_set_stream",
           "mqs_timing_enable", "mqs_timing_get", "mqs_pcg_solve_noalloc", "mqs_selftest_barrier_timeout",
           "mqs_set_blocks", "mqs_batch_create", "mqs_batch_set_scale", "mqs_batch_step", "mqs_batch_last_ms",
           "mqs_batch_tune", "mqs_batch_destroy", "mqs_adjoint", "mqs_adjoint_ckpt", "mqs_loss",
           "mqs_solve_an", "mqs_graph_steps", "mqs_batch_graph_steps", "mqs_batch_tune_depth",
           "mqs_debug_check", "mqs_batch_set_weighting", "mqs_batch_get_weighting", "mqs_tune_pcg",
           "mqs_batch_tune_pcg", "mqs_get_options", "mqs_part_ranges")


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double)]


class Materials(C.Structure):
    _fields_ = [("sigma_cell", C.POINTER(C.c_double)), ("brauer_cell", C.POINTER(C.c_uint8)),
                ("nu0", C.c_double), ("k1", C.c_double), ("k2", C.c_double), ("k3", C.c_double)]


class Coil(C.Structure):
    _fields_ = [("plane_k", C.c_int), ("i0", C.c_int), ("j0", C.c_int), ("i1", C.c_int), ("j1", C.c_int),
                ("amplitude", C.c_double), ("freq_hz", C.c_double), ("waveform", C.c_int), ("tau", C.c_double)]


class Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("start_mode", C.c_int), ("spe_depth", C.c_int),
                ("pod_snapshots", C.c_int), ("eps_pod", C.c_double), ("eps_lin", C.c_double),
                ("dt", C.c_double), ("rhs_time", C.c_int), ("pcg_variant", C.c_int), ("precision", C.c_int),
                ("inner_tol", C.c_double), ("cspe_period", C.c_int), ("rhs_split", C.c_int), ("graph", C.c_int),
                ("cfl_factor", C.c_double), ("monitor_steps", C.c_int), ("tile_groups", C.c_int),
                ("halo_warps", C.c_int)]


class LayoutInfo(C.Structure):
    _fields_ = [("n", C.c_int), ("n_layout", C.c_long), ("n_c", C.c_long), ("n_n", C.c_long),
                ("box_lo", C.c_int * 3), ("box_hi", C.c_int * 3)]


class AdjointInfo(C.Structure):
    _fields_ = [("objective", C.c_double), ("grad_amplitude", C.c_double),
                ("forward_iterations", C.c_long), ("adjoint_iterations", C.c_long),
                ("recompute_iterations", C.c_long)]


class StepStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("rank", C.c_int), ("refinements", C.c_int),
                ("relres", C.c_double), ("start_relres", C.c_double), ("pod_info", C.c_double)]


class Timing(C.Structure):
    _fields_ = [("ms_rhs", C.c_double), ("ms_start", C.c_double), ("ms_pcg", C.c_double),
                ("ms_conductor", C.c_double), ("ms_history", C.c_double), ("launches", C.c_long),
                ("pcg_launches", C.c_long), ("steps", C.c_long)]


class DebugReport(C.Structure):
    _fields_ = [("enabled", C.c_int), ("site", C.c_int), ("index", C.c_longlong), ("faults", C.c_int),
                ("canaries_bad", C.c_int), ("buffers", C.c_int)]


class PcgInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("relres", C.c_double),
                ("start_relres", C.c_double)]


_lib = None
_live = weakref.WeakSet()     # open solvers (the debug check visits their buffers)


def load():
    """Load libmqs.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1611_06721_gb300.build.build("
                           f"{'debug=True' if DEBUG else ''}) (the library has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P, D, I, L, V = C.POINTER, C.c_double, C.c_int, C.c_long, C.c_void_p
    H = V
    sig = {
        "mqs_setup": ([P(Grid), P(Materials), P(C.c_uint8), P(Coil), P(Options), P(H)], I),
        "mqs_destroy": ([H], I),
        "mqs_last_error": ([H, C.c_char_p, C.c_size_t], I),
        "mqs_layout": ([H, P(LayoutInfo)], I),
        "mqs_set_dt": ([H, D], I),
        "mqs_get_dt": ([H, P(D), P(D)], I),
        "mqs_set_options": ([H, P(Options)], I),
        "mqs_lambda_max": ([H, P(D), D, D, I, P(D), P(I)], I),
        "mqs_step": ([H, I, P(StepStats)], I),
        "mqs_step_enqueue": ([H, I], I),
        "mqs_step_finish": ([H, I, P(StepStats)], I),
        "mqs_get_state": ([H, P(D), C.c_size_t, P(D), P(L)], I),
        "mqs_set_state": ([H, P(D), C.c_size_t, D, L], I),
        "mqs_get_state_dev": ([H, V, C.c_size_t, V], I),
        "mqs_set_state_dev": ([H, V, C.c_size_t, V], I),
        "mqs_get_solution": ([H, P(D)], I),
        "mqs_reset_history": ([H], I),
        "pcg_solve": ([H, P(D), P(D), D, I, P(PcgInfo)], I),
        "pcg_solve_dev": ([H, V, V, D, I, P(PcgInfo), V], I),
        "mqs_apply_kn": ([H, P(D), P(D)], I),
        "mqs_apply_kn_dev": ([H, V, V, V], I),
        "mqs_conductor_rate": ([H, P(D), P(D), P(D)], I),
        "mqs_push_history": ([H, P(D)], I),
        "spe_start": ([H, P(D), P(D), P(I)], I),
        "pod_basis": ([H, P(I), P(D), P(D)], I),
        "pod_start": ([H, P(D), P(D), P(I)], I),
        "mqs_set_stream": ([H, V], I),
        "mqs_timing_enable": ([H, I], I),
        "mqs_timing_get": ([H, P(Timing)], I),
        "mqs_pcg_solve_noalloc": ([I, D, D, V, V, V, D, I, P(PcgInfo), V], I),
        "mqs_selftest_barrier_timeout": ([C.c_longlong], I),
        "mqs_part_ranges": ([I, I, I, P(I)], I),
        "mqs_set_blocks": ([H, I], I),
        "mqs_batch_create": ([P(H), I, D, P(V)], I),
        "mqs_batch_set_scale": ([V, D], I),
        "mqs_batch_step": ([V, I, P(StepStats)], I),
        "mqs_batch_last_ms": ([V, P(D)], I),
        "mqs_batch_tune": ([V, I, P(D)], I),
        "mqs_batch_destroy": ([V], I),
        "mqs_adjoint": ([H, I, P(D), P(AdjointInfo)], I),
        "mqs_adjoint_ckpt": ([H, I, I, P(D), P(AdjointInfo)], I),
        "mqs_loss": ([H, I, P(D)], I),
        "mqs_solve_an": ([H, P(D), P(PcgInfo)], I),
        "mqs_graph_steps": ([H, P(C.c_long)], I),
        "mqs_batch_graph_steps": ([V, P(C.c_long)], I),
        "mqs_batch_tune_depth": ([V, I, P(I), I, P(I)], I),
        "mqs_debug_check": ([H, P(DebugReport)], I),
        "mqs_batch_set_weighting": ([V, I], I),
        "mqs_batch_get_weighting": ([V, P(I)], I),
        "mqs_tune_pcg": ([H, I, P(I)], I),
        "mqs_batch_tune_pcg": ([V, I, P(I)], I),
        "mqs_get_options": ([H, P(Options)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _dev_ptrs(*specs):
    """Device pointers of torch tensors, after checking that each is what the library
    reads or writes there.  specs: (tensor, name, dtype, numel[, align]) tuples.  First
    every tensor's dtype, element count and layout, then that each is a CUDA tensor on
    the current device and aligned: ValueError on the first mismatch, before any launch."""
    import torch
    for sp in specs:
        t, name, dtype, numel = sp[:4]
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor, got {type(t).__name__}")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
        if t.numel() != numel:
            raise ValueError(f"{name} must hold {numel} values, got {t.numel()}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    out = []
    for sp in specs:
        t, name = sp[0], sp[1]
        align = sp[4] if len(sp) > 4 else 8
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is "
                             f"cuda:{torch.cuda.current_device()}")
        if t.data_ptr() % align:
            raise ValueError(f"{name} must be {align}-byte aligned")
        out.append(C.c_void_p(t.data_ptr()))
    return out if len(out) > 1 else out[0]


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


class MqsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


@dataclass
class SolverOptions:
    tol: float = 1e-10
    maxit: int = 100000
    start_mode: int = START_ZERO
    spe_depth: int = 8
    pod_snapshots: int = 20
    eps_pod: float = 1e-4
    eps_lin: float = 1e-10
    dt: float = 0.0
    rhs_time: int = 0
    pcg_variant: int = 0
    precision: int = 0
    inner_tol: float = 0.0
    cspe_period: int = 0
    rhs_split: int = 0
    graph: int = 1          # steady-state SPE steps from CUDA graphs (bitwise the same results)
    cfl_factor: float = 0.0  # > 0 with dt <= 0: setup sets dt = cfl_factor * 2 / lambda_max (eq. (CFL))
    monitor_steps: int = 0   # instability monitor window (0: 8 steps; < 0: finiteness test only)
    tile_groups: int = 0     # stencil groups per block of the FP64 one-reduction pass (0/2 or 3)
    halo_warps: int = 0      # halo warps per tile group of that pass (0/1, or 2 with two groups)

    def c(self):
        return Options(self.tol, self.maxit, self.start_mode, self.spe_depth, self.pod_snapshots,
                       self.eps_pod, self.eps_lin, self.dt, self.rhs_time, self.pcg_variant, self.precision,
                       self.inner_tol, self.cspe_period, self.rhs_split, self.graph, self.cfl_factor,
                       self.monitor_steps, self.tile_groups, self.halo_warps)


class Solver:
    """One handle of the library: grid, materials, coil and options."""

    def __init__(self, n, h, sigma_cell, brauer_cell, nu0, k1, k2, k3, coil, options: SolverOptions,
                 conductor_mask=None):
        self.lib = load()
        self._sigma = _f64(sigma_cell, n ** 3)
        self._brauer = None if brauer_cell is None else np.ascontiguousarray(brauer_cell, dtype=np.uint8).reshape(-1)
        mat = Materials(_dp(self._sigma),
                        None if self._brauer is None else self._brauer.ctypes.data_as(C.POINTER(C.c_uint8)),
                        nu0, k1, k2, k3)
        mask = None
        if conductor_mask is not None:
            self._mask = np.ascontiguousarray(conductor_mask, dtype=np.uint8).reshape(-1)
            mask = self._mask.ctypes.data_as(C.POINTER(C.c_uint8))
        self.options = options
        h_ = C.c_void_p()
        rc = self.lib.mqs_setup(C.byref(Grid(n, n, n, h)), C.byref(mat), mask, C.byref(Coil(*coil)),
                                C.byref(options.c()), C.byref(h_))
        if rc != MQS_OK:
            raise MqsError(rc, "mqs_setup failed (see stderr)")
        self.h = h_
        _live.add(self)
        info = LayoutInfo()
        self._check(self.lib.mqs_layout(self.h, C.byref(info)))
        self.n = info.n
        self.n_layout = info.n_layout
        self.n_c = info.n_c
        self.n_n = info.n_n

    @classmethod
    def from_problem(cls, p, options: SolverOptions, conductor_mask=None):
        coil = (p.coil_k, p.coil_i0, p.coil_j0, p.coil_i1, p.coil_j1, p.amplitude, p.freq, p.waveform, p.tau)
        return cls(p.N, p.h, p.sigma_cell, p.brauer_cell, p.nu0, p.k1, p.k2, p.k3, coil, options,
                   conductor_mask)

    def _check(self, rc, allow=()):
        if rc != MQS_OK and rc not in allow:
            buf = C.create_string_buffer(512)
            self.lib.mqs_last_error(self.h, buf, 512)
            raise MqsError(rc, buf.value.decode())
        return rc

    def close(self):
        batch = getattr(self, "_batch", None)
        batch = batch() if batch is not None else None
        if batch is not None:
            batch.close()               # a batch must end before the handles it steps
        if getattr(self, "h", None):
            self.lib.mqs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration ---------------------------------------------------------------
    def set_dt(self, dt):
        self._check(self.lib.mqs_set_dt(self.h, dt))

    def get_dt(self):
        return self.dt_lambda()[0]

    def dt_lambda(self):
        """(dt, lambda_max of eq. (CFL) found on this handle, 0 if none) (mqs_get_dt)."""
        d, lam = C.c_double(), C.c_double()
        self._check(self.lib.mqs_get_dt(self.h, C.byref(d), C.byref(lam)))
        return d.value, lam.value

    def set_options(self, options: SolverOptions):
        self._check(self.lib.mqs_set_options(self.h, C.byref(options.c())))
        self.options = options

    def reset_history(self):
        self._check(self.lib.mqs_reset_history(self.h))

    def lambda_max(self, v0, pcg_tol=1e-12, rtol=1e-8, maxit=2000):
        v0 = _f64(v0, self.n_c)
        lam, it = C.c_double(), C.c_int()
        self._check(self.lib.mqs_lambda_max(self.h, _dp(v0), pcg_tol, rtol, maxit, C.byref(lam), C.byref(it)))
        return lam.value, it.value

    def set_stream(self, stream):
        """Route later work to a cudaStream_t given as an int (0 = own stream)."""
        self._check(self.lib.mqs_set_stream(self.h, C.c_void_p(stream)))

    def timing_enable(self, on=True):
        self._check(self.lib.mqs_timing_enable(self.h, 1 if on else 0))

    def timing_get(self):
        t = Timing()
        self._check(self.lib.mqs_timing_get(self.h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in Timing._fields_}

    def graph_steps(self):
        """Steps replayed from (or captured into) a CUDA graph since setup."""
        v = C.c_long()
        self._check(self.lib.mqs_graph_steps(self.h, C.byref(v)))
        return v.value

    # -- time stepping -----------------------------------------------------------------
    def step(self, nsteps, allow_fail=False):
        st = (StepStats * max(nsteps, 1))()
        rc = self.lib.mqs_step(self.h, nsteps, st)
        if not allow_fail:
            self._check(rc)
        return rc, [st[q] for q in range(nsteps)]

    def mqs_step(self, nsteps):
        return self.step(nsteps)[1]

    def step_enqueue(self, nsteps):
        """Issue nsteps steps on the handle's stream without waiting (mqs_step_enqueue)."""
        self._check(self.lib.mqs_step_enqueue(self.h, nsteps))

    def step_finish(self, nsteps, allow_fail=False):
        """Wait for enqueued steps: (rc, per-step stats) as step() returns (mqs_step_finish)."""
        st = (StepStats * max(nsteps, 1))()
        rc = self.lib.mqs_step_finish(self.h, nsteps, st)
        if not allow_fail:
            self._check(rc)
        return rc, [st[q] for q in range(nsteps)]

    def adjoint(self, nsteps, checkpoint_every=0):
        """Gradient of the eddy-current loss J over nsteps steps from the current state
        (mqs_adjoint, or mqs_adjoint_ckpt with checkpoints every `checkpoint_every` steps
        and recomputation in between): returns (J, dJ/dsigma per cell as an (N, N, N)
        array indexed [k, j, i], dJ/d amplitude, AdjointInfo)."""
        g = np.zeros(self.n ** 3)
        info = AdjointInfo()
        if checkpoint_every > 0:
            self._check(self.lib.mqs_adjoint_ckpt(self.h, nsteps, checkpoint_every, _dp(g), C.byref(info)))
        else:
            self._check(self.lib.mqs_adjoint(self.h, nsteps, _dp(g), C.byref(info)))
        return info.objective, g.reshape(self.n, self.n, self.n), info.grad_amplitude, info

    def solve_an(self):
        """a_n^m of eq. (anm) for the current state (mqs_solve_an): (layout vector, PcgInfo)."""
        a = np.empty(self.n_layout)
        info = PcgInfo()
        self._check(self.lib.mqs_solve_an(self.h, _dp(a), C.byref(info)))
        return a, info

    def loss(self, nsteps):
        """The eddy-current loss J over nsteps steps from the current state (mqs_loss)."""
        v = C.c_double()
        self._check(self.lib.mqs_loss(self.h, nsteps, C.byref(v)))
        return v.value

    def tune_pcg(self, trials=2):
        """The fastest PCG kernel form for this grid, precision and block count
        (mqs_tune_pcg); sets it and returns (pcg_variant, tile_groups, halo_warps)."""
        v = C.c_int()
        self._check(self.lib.mqs_tune_pcg(self.h, trials, C.byref(v)))
        self._sync_options()
        return self.pcg_form()

    def pcg_form(self):
        """(pcg_variant, tile_groups, halo_warps) of the options in use."""
        o = self.options
        return o.pcg_variant, o.tile_groups, o.halo_warps

    def _sync_options(self):
        o = Options()
        self._check(self.lib.mqs_get_options(self.h, C.byref(o)))
        self.options = replace(self.options, pcg_variant=o.pcg_variant, tile_groups=o.tile_groups,
                               halo_warps=o.halo_warps)

    def set_blocks(self, nblk):
        """Persistent blocks of this handle's PCG kernels (0 = one per SM)."""
        self._check(self.lib.mqs_set_blocks(self.h, nblk))

    def get_state(self, out=None):
        """(a_c, t, m).  out (optional): a C-contiguous float64 array of n_c values (pinned
        host memory, for one) that receives a_c and is returned."""
        if out is None:
            a = np.empty(self.n_c)
        else:
            if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
                    and out.flags.writeable and out.size == self.n_c):
                raise ValueError(f"out must be a writeable C-contiguous float64 array of {self.n_c} values")
            a = out
        t, m = C.c_double(), C.c_long()
        self._check(self.lib.mqs_get_state(self.h, _dp(a), a.size, C.byref(t), C.byref(m)))
        return a, t.value, m.value

    def set_state(self, a_c, t=0.0, m=0):
        a = _f64(a_c, self.n_c)
        self._check(self.lib.mqs_set_state(self.h, _dp(a), a.size, t, m))

    def get_state_dev(self, out, stream=0):
        """a_c into the float64 CUDA tensor `out` (n_c values)."""
        import torch
        ptr = _dev_ptrs((out, "out", torch.float64, self.n_c))
        self._check(self.lib.mqs_get_state_dev(self.h, ptr, self.n_c, C.c_void_p(stream)))

    def set_state_dev(self, a, stream=0):
        """a_c from the float64 CUDA tensor `a` (n_c values)."""
        import torch
        ptr = _dev_ptrs((a, "a", torch.float64, self.n_c))
        self._check(self.lib.mqs_set_state_dev(self.h, ptr, self.n_c, C.c_void_p(stream)))

    def get_solution(self):
        w = np.empty(self.n_layout)
        self._check(self.lib.mqs_get_solution(self.h, _dp(w)))
        return w

    # -- stand-alone operations -------------------------------------------------------
    def pcg_solve(self, b, x0=None, tol=1e-10, maxit=100000, allow_fail=False):
        b = _f64(b, self.n_layout)
        x = np.zeros(self.n_layout) if x0 is None else _f64(x0, self.n_layout).copy()
        info = PcgInfo()
        rc = self.lib.pcg_solve(self.h, _dp(b), _dp(x), tol, maxit, C.byref(info))
        if not allow_fail:
            self._check(rc)
        return x, info

    def pcg_solve_dev(self, b, x, tol=1e-10, maxit=100000, stream=0, allow_fail=False):
        """pcg_solve_dev on float64 CUDA tensors of n_layout values (x: start in, solution out)."""
        import torch
        pb, px = _dev_ptrs((b, "b", torch.float64, self.n_layout), (x, "x", torch.float64, self.n_layout))
        info = PcgInfo()
        rc = self.lib.pcg_solve_dev(self.h, pb, px, tol, maxit, C.byref(info), C.c_void_p(stream))
        if not allow_fail:
            self._check(rc)
        return info

    def apply_kn(self, x):
        x = _f64(x, self.n_layout)
        y = np.empty(self.n_layout)
        self._check(self.lib.mqs_apply_kn(self.h, _dp(x), _dp(y)))
        return y

    def apply_kn_dev(self, x, y, stream=0):
        """y = K_n x on float64 CUDA tensors of n_layout values."""
        import torch
        px, py = _dev_ptrs((x, "x", torch.float64, self.n_layout), (y, "y", torch.float64, self.n_layout))
        self._check(self.lib.mqs_apply_kn_dev(self.h, px, py, C.c_void_p(stream)))

    def conductor_rate(self, a_c, w):
        a = _f64(a_c, self.n_c)
        w = _f64(w, self.n_layout)
        F = np.empty(self.n_c)
        self._check(self.lib.mqs_conductor_rate(self.h, _dp(a), _dp(w), _dp(F)))
        return F

    def push_history(self, w):
        w = _f64(w, self.n_layout)
        self._check(self.lib.mqs_push_history(self.h, _dp(w)))

    def spe_start(self, b):
        b = _f64(b, self.n_layout)
        x0 = np.empty(self.n_layout)
        r = C.c_int()
        self._check(self.lib.spe_start(self.h, _dp(b), _dp(x0), C.byref(r)))
        return x0, r.value

    def pod_basis(self):
        k, info = C.c_int(), C.c_double()
        sig = np.zeros(self.options.pod_snapshots)
        self._check(self.lib.pod_basis(self.h, C.byref(k), _dp(sig), C.byref(info)))
        return k.value, sig, info.value

    def pod_start(self, b):
        b = _f64(b, self.n_layout)
        x0 = np.empty(self.n_layout)
        k = C.c_int()
        self._check(self.lib.pod_start(self.h, _dp(b), _dp(x0), C.byref(k)))
        return x0, k.value


def debug_check(solvers=None):
    """mqs_debug_check over the recorded index faults and the guard bytes of every
    open solver's buffers (or of `solvers`).  Returns a dict: enabled (0 in the
    release library), site and index of the first fault (site 0: none), faults,
    canaries_bad and buffers summed over the solvers."""
    lib = load()
    rep = DebugReport()
    rc = lib.mqs_debug_check(None, C.byref(rep))
    if rc != MQS_OK:
        raise MqsError(rc, "mqs_debug_check failed")
    out = {"enabled": rep.enabled, "site": rep.site, "index": rep.index, "faults": rep.faults,
           "canaries_bad": 0, "buffers": 0}
    for sv in list(_live if solvers is None else solvers):
        if not getattr(sv, "h", None):
            continue
        r = DebugReport()
        rc = lib.mqs_debug_check(sv.h, C.byref(r))
        if rc != MQS_OK:
            raise MqsError(rc, "mqs_debug_check failed")
        out["canaries_bad"] += r.canaries_bad
        out["buffers"] += r.buffers
        if r.faults and not out["faults"]:
            out.update(site=r.site, index=r.index)
        out["faults"] += r.faults
    return out


def part_ranges(n, nblk, groups=2):
    """Plane-tile ranges of the one-reduction PCG pass's tile groups (mqs_part_ranges,
    host only): an (nblk * groups, 2) int array of [first, end) per part."""
    groups = groups or 2                      # 0: the default two groups, as in the library
    if n < 1 or nblk < 1 or groups < 1:
        raise ValueError("n, nblk and groups must be positive")
    out = np.zeros(2 * nblk * groups, dtype=np.int32)
    rc = load().mqs_part_ranges(n, nblk, groups, out.ctypes.data_as(C.POINTER(C.c_int)))
    if rc != 0:
        raise MqsError(rc, f"mqs_part_ranges({n}, {nblk}, {groups}) failed")
    return out.reshape(-1, 2)


def pcg_solve_noalloc(n, h, nu0, cell_mask, b, x, tol=1e-10, maxit=100000, stream=0):
    """mqs_pcg_solve_noalloc on torch CUDA tensors (cell_mask uint8 n^3, b and
    x float64 layout vectors of 3 n^3 values, x 16-byte aligned); x is overwritten.
    Returns (status, PcgInfo).  The tensors are checked before the call."""
    import torch
    n3 = int(n) ** 3
    pm, pb, px = _dev_ptrs((cell_mask, "cell_mask", torch.uint8, n3, 1), (b, "b", torch.float64, 3 * n3),
                           (x, "x", torch.float64, 3 * n3, 16))
    lib = load()
    info = PcgInfo()
    rc = lib.mqs_pcg_solve_noalloc(n, h, nu0, pm, pb, px, tol, maxit, C.byref(info), C.c_void_p(stream))
    return rc, info


class Batch:
    """Several solvers advanced together on one GPU (mqs_batch_*): each on its own
    stream, PCG block counts proportional to the unknowns.  The solvers stay
    owned by the caller and must outlive the batch."""

    def __init__(self, solvers, blocks_scale=2.0):
        self.lib = load()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[sv.h for sv in self.solvers])
        b = C.c_void_p()
        rc = self.lib.mqs_batch_create(arr, len(self.solvers), blocks_scale, C.byref(b))
        if rc != MQS_OK:
            raise MqsError(rc, "mqs_batch_create failed")
        self.b = b
        for sv in self.solvers:
            sv._batch = weakref.ref(self)

    def _check(self, rc):
        if rc != MQS_OK:
            msgs = []
            for q, sv in enumerate(self.solvers):
                buf = C.create_string_buffer(512)
                self.lib.mqs_last_error(sv.h, buf, 512)
                if buf.value:
                    msgs.append(f"[{q}] {buf.value.decode()}")
            raise MqsError(rc, "; ".join(msgs))
        return rc

    def step(self, nsteps, allow_fail=False):
        """nsteps steps of every solver; returns (rc, stats[nsteps][count])."""
        cnt = len(self.solvers)
        st = (StepStats * max(nsteps * cnt, 1))()
        rc = self.lib.mqs_batch_step(self.b, nsteps, st)
        if not allow_fail:
            self._check(rc)
        return rc, [[st[s * cnt + q] for q in range(cnt)] for s in range(nsteps)]

    def last_ms(self):
        v = C.c_double()
        self._check(self.lib.mqs_batch_last_ms(self.b, C.byref(v)))
        return v.value

    def graph_steps(self):
        """Batch steps replayed from (or captured into) a CUDA graph."""
        v = C.c_long()
        self._check(self.lib.mqs_batch_graph_steps(self.b, C.byref(v)))
        return v.value

    def set_scale(self, blocks_scale):
        self._check(self.lib.mqs_batch_set_scale(self.b, blocks_scale))

    def tune(self, trial_steps):
        v = C.c_double()
        self._check(self.lib.mqs_batch_tune(self.b, trial_steps, C.byref(v)))
        return v.value

    def tune_pcg(self, trials=2):
        """mqs_batch_tune_pcg: the PCG kernel form per (grid size, precision) group;
        returns every solver's (pcg_variant, tile_groups, halo_warps)."""
        out = (C.c_int * len(self.solvers))()
        self._check(self.lib.mqs_batch_tune_pcg(self.b, trials, out))
        for sv in self.solvers:
            sv._sync_options()
        return [sv.pcg_form() for sv in self.solvers]

    def set_weighting(self, by_work):
        """Block shares by unknowns (False) or unknowns x last iterations (True)."""
        self._check(self.lib.mqs_batch_set_weighting(self.b, int(by_work)))

    def weighting(self):
        v = C.c_int()
        self._check(self.lib.mqs_batch_get_weighting(self.b, C.byref(v)))
        return bool(v.value)

    def tune_depth(self, trial_steps, depths=(4, 8, 16)):
        """SPE depth per grid size (mqs_batch_tune_depth); returns every solver's depth."""
        ds = (C.c_int * len(depths))(*depths)
        out = (C.c_int * len(self.solvers))()
        self._check(self.lib.mqs_batch_tune_depth(self.b, trial_steps, ds, len(depths), out))
        for sv, d in zip(self.solvers, out):
            if sv.options.start_mode == START_SPE:
                sv.options = replace(sv.options, spe_depth=int(d))
        return list(out)

    def close(self):
        if getattr(self, "b", None):
            self.lib.mqs_batch_destroy(self.b)
            self.b = None
            for sv in self.solvers:
                sv._batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eddy_loss(sigma_cell, amplitude, problem, options: SolverOptions, nsteps, checkpoint_every=0):
    """The eddy-current loss J over `nsteps` steps from rest as a differentiable torch
    function of the cell conductivities (tensor [N, N, N] indexed [k, j, i]) and the coil
    amplitude (0-d tensor); dt, the edge classes and the waveform come from `problem` /
    `options` and stay fixed.  The forward call runs mqs_adjoint (J and both gradients
    at once; checkpoints every `checkpoint_every` steps when positive), backward scales
    the stored gradients.  The conducting region (and so the edge classes) is the one of
    `problem` (its cells with sigma > 0); a conductivity that reaches 0 or below inside
    it raises MqsError."""
    import torch
    cmask = (np.asarray(problem.sigma_cell) > 0).astype(np.uint8)

    class _EddyLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, sig, amp):
            sg = sig.detach().to("cpu", torch.float64).numpy()
            p = problem.with_(sigma_cell=sg, amplitude=float(amp))
            # the conducting region stays the problem's own: a conductivity driven to 0
            # inside it is refused by mqs_setup instead of silently changing the edge classes
            s = Solver.from_problem(p, options, conductor_mask=cmask)
            try:
                J, g, gI, _ = s.adjoint(nsteps, checkpoint_every)
            finally:
                s.close()
            ctx.save_for_backward(torch.from_numpy(g).to(sig.device, sig.dtype),
                                  torch.tensor(gI, dtype=amp.dtype, device=amp.device))
            return torch.tensor(J, dtype=torch.float64, device=sig.device)

        @staticmethod
        def backward(ctx, gout):
            g, gI = ctx.saved_tensors
            return gout.to(g.dtype) * g, gout.to(gI.dtype) * gI

    return _EddyLoss.apply(sigma_cell, amplitude)
