"""Python binding of the C ABI: MGSolver owns one context and its workspace.

PyTorch provides the device memory (the workspace and the vectors) and the
stream; every computation happens in the CUDA library.
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import MgOpts, load_library

PRECISION = {"fp64": 0, "mixed": 1, "df64": 2}
OVERLAP_MODE = {"layers": 0, "width": 1, "max": 2}
PROFILE = {"quintic": 0, "linear": 1, "quintic_halves": 2, "quintic_normalised": 3}
WEIGHT_DELTA = {"default": 0, "node": 1, "mid": 2, "strip": 3}
FDM_OPERANDS = {"fp32": 0, "bf16": 1, "fp8": 2}


class MGError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_lib.STATUS_NAMES.get(status, status), message))
        self.status = status


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class MGSolver:
    """Polynomial multigrid for the SIPG Poisson problem on a periodic box.

    lengths (lx, ly, lz), counts (nx, ny, nz), order P (power of two), penalty
    mu/mu_min (paper: 2), overlap N_O node layers; see include/mgdg.h.
    widths: three sequences of element widths for a graded mesh
    (mg_setup_graded); lengths and counts are then taken from them and may be
    None."""

    def __init__(self, lengths, counts, P, penalty=2.0, overlap=1, precision="fp64", overlap_mode="layers",
                 overlap_frac=0.08, weight_profile="quintic", ns_pre=1, ns_post=1, ns_growth=1, device="cuda",
                 stream=None, tensor_cores=False, outer_df64=False, weight_delta="default", autotune=False,
                 fdm_bf16=False, fdm_operands="fp32", persistent="auto", widths=None):
        self.lib = load_library()
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        opts = MgOpts()
        self.lib.mg_default_opts(ctypes.byref(opts))
        opts.overlap_mode = OVERLAP_MODE[overlap_mode]
        opts.overlap_frac = float(overlap_frac)
        opts.weight_profile = PROFILE[weight_profile]
        opts.weight_delta = WEIGHT_DELTA[weight_delta]
        opts.autotune = 1 if autotune else 0
        # operand precision study of the FP32 smoother (fdm_bf16=True is fdm_operands="bf16")
        opts.fdm_operands = FDM_OPERANDS["bf16" if fdm_bf16 else fdm_operands]
        opts.persistent = {"auto": 0, "always": 1, "never": 2}[persistent]  # grouped launches of solve_batch
        opts.ns_pre, opts.ns_post, opts.ns_growth = int(ns_pre), int(ns_post), int(ns_growth)
        opts.precision = PRECISION[precision]
        opts.fdm_tensor_cores = {False: 0, True: 1, "auto": 2}[tensor_cores]
        opts.outer_df64 = {False: 0, True: 1, "all": 2}[outer_df64]
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        opts.stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.opts = opts
        ctx = ctypes.c_void_p()
        if widths is not None:
            self.widths = tuple(np.ascontiguousarray(w, dtype=np.float64) for w in widths)
            counts = tuple(len(w) for w in self.widths)
            lengths = tuple(float(w.sum()) for w in self.widths)
            hp = [w.ctypes.data_as(ctypes.c_void_p) for w in self.widths]
            st = self.lib.mg_setup_graded(hp[0], hp[1], hp[2], int(counts[0]), int(counts[1]), int(counts[2]), int(P),
                                          float(penalty), int(overlap), ctypes.byref(opts), ctypes.byref(ctx))
            if st != 0:
                raise MGError(st, "mg_setup_graded rejected the arguments")
        else:
            self.widths = None
            st = self.lib.mg_setup(float(lengths[0]), float(lengths[1]), float(lengths[2]), int(counts[0]),
                                   int(counts[1]), int(counts[2]), int(P), float(penalty), int(overlap),
                                   ctypes.byref(opts), ctypes.byref(ctx))
            if st != 0:
                raise MGError(st, "mg_setup rejected the arguments")
        self.ctx = ctx
        self.P = int(P)
        self.lengths = tuple(float(v) for v in lengths)
        self.counts = tuple(int(v) for v in counts)
        size = ctypes.c_size_t()
        self._check(self.lib.mg_workspace_size(ctx, ctypes.byref(size)))
        self.workspace_bytes = size.value
        self.workspace = torch.empty(size.value + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self._check(self.lib.mg_bind_workspace(ctx, ctypes.c_void_p(self._ws_ptr), ctypes.c_size_t(size.value)))

    # -- helpers --------------------------------------------------------------
    def _check(self, st):
        if st != 0:
            msg = self.lib.mg_last_error(self.ctx)
            raise MGError(st, msg.decode() if msg else "")
        return st

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.mg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_levels(self):
        return self.lib.mg_num_levels(self.ctx)

    @property
    def L(self):
        return self.num_levels - 1

    def num_dofs(self, level=None):
        return int(self.lib.mg_num_dofs(self.ctx, self.L if level is None else level))

    def fdm_tensor_cores(self, level):
        """1 if the FP32 smoother of `level` runs its contractions on the tensor cores."""
        return int(self.lib.mg_level_fdm_tensor_cores(self.ctx, level))

    def kernel_variants(self, level):
        """Kernel variants of single solves on `level` (mg_level_kernel_variant):
        {"fdm", "sipg", "scatter"} -> 0 parameter-space / element-aligned
        kernels, 1 the alternative, 2 (FP32 smoother) the split form."""
        return {k: int(self.lib.mg_level_kernel_variant(self.ctx, level, i))
                for i, k in enumerate(("fdm", "sipg", "scatter"))}

    def layers(self, level, direction=None):
        """N_O of a level: of the x direction, or of `direction` (0, 1, 2)."""
        if direction is None:
            return int(self.lib.mg_level_layers(self.ctx, level))
        return int(self.lib.mg_level_layers_dir(self.ctx, level, int(direction)))

    def _vec(self, t, level, dtype=torch.float64, name="vector"):
        n = self.num_dofs(level)
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dtype or not t.is_contiguous() \
                or t.numel() != n:
            raise ValueError("%s must be a contiguous %s tensor of %d values on %s" % (name, dtype, n, self.device))
        return t

    def empty(self, level=None, dtype=torch.float64):
        return torch.empty(self.num_dofs(level), dtype=dtype, device=self.device)

    def zeros(self, level=None, dtype=torch.float64):
        return torch.zeros(self.num_dofs(level), dtype=dtype, device=self.device)

    # -- entry points (same names as the C ABI) ---------------------------------
    def node_coords(self, level=None):
        level = self.L if level is None else level
        x, y, z = (self.empty(level) for _ in range(3))
        self._check(self.lib.mg_node_coords(self.ctx, level, _ptr(x), _ptr(y), _ptr(z)))
        return x, y, z

    def rhs(self, f_nodal):
        self._vec(f_nodal, self.L, name="f_nodal")
        b = self.empty()
        self._check(self.lib.mg_rhs(self.ctx, _ptr(f_nodal), _ptr(b)))
        return b

    def apply_sipg(self, u, level=None, out=None):
        level = self.L if level is None else level
        if u.dtype == torch.float32:
            self._vec(u, level, torch.float32, "u")
            out = self.empty(level, torch.float32) if out is None else out
            self._check(self.lib.mg_apply_sipg_f32(self.ctx, level, _ptr(u), _ptr(out)))
            return out
        self._vec(u, level, name="u")
        out = self.empty(level) if out is None else self._vec(out, level, name="out")
        self._check(self.lib.mg_apply_sipg(self.ctx, level, _ptr(u), _ptr(out)))
        return out

    def apply_sipg_df64(self, u, level=None, out=None):
        """A_l u with double-float arithmetic (FP64 vectors); see mg_apply_sipg_df64."""
        level = self.L if level is None else level
        self._vec(u, level, name="u")
        out = self.empty(level) if out is None else self._vec(out, level, name="out")
        self._check(self.lib.mg_apply_sipg_df64(self.ctx, level, _ptr(u), _ptr(out)))
        return out

    def residual(self, u, f, level=None, out=None):
        level = self.L if level is None else level
        self._vec(u, level, name="u")
        self._vec(f, level, name="f")
        out = self.empty(level) if out is None else self._vec(out, level, name="out")
        self._check(self.lib.mg_residual(self.ctx, level, _ptr(u), _ptr(f), _ptr(out)))
        return out

    def smooth(self, u, f, level=None, nsteps=1):
        level = self.L if level is None else level
        if u.dtype == torch.float32:
            self._vec(u, level, torch.float32, "u")
            self._vec(f, level, torch.float32, "f")
            self._check(self.lib.mg_smooth_f32(self.ctx, level, _ptr(u), _ptr(f), int(nsteps)))
            return u
        self._vec(u, level, name="u")
        self._vec(f, level, name="f")
        self._check(self.lib.mg_smooth(self.ctx, level, _ptr(u), _ptr(f), int(nsteps)))
        return u

    def smooth_df64(self, u, f, level=None, nsteps=1):
        """Schwarz steps on FP64 vectors with double-float arithmetic (mg_smooth_df64)."""
        level = self.L if level is None else level
        self._vec(u, level, name="u")
        self._vec(f, level, name="f")
        self._check(self.lib.mg_smooth_df64(self.ctx, level, _ptr(u), _ptr(f), int(nsteps)))
        return u

    def restrict_residual(self, u, f, level=None):
        level = self.L if level is None else level
        self._vec(u, level, name="u")
        self._vec(f, level, name="f")
        fc = self.empty(level - 1)
        self._check(self.lib.mg_restrict_residual(self.ctx, level, _ptr(u), _ptr(f), _ptr(fc)))
        return fc

    def prolongate(self, uc, u, level=None):
        level = self.L if level is None else level
        self._vec(uc, level - 1, name="u_c")
        self._vec(u, level, name="u")
        self._check(self.lib.mg_prolongate(self.ctx, level, _ptr(uc), _ptr(u)))
        return u

    def coarse_solve(self, f0):
        self._vec(f0, 0, name="f0")
        u0 = self.empty(0)
        self._check(self.lib.mg_coarse_solve(self.ctx, _ptr(f0), _ptr(u0)))
        return u0

    def vcycle_df64(self, u, f):
        """One V-cycle on FP64 vectors with the multigrid in double-float arithmetic."""
        self._vec(u, self.L, name="u")
        self._vec(f, self.L, name="f")
        self._check(self.lib.mg_vcycle_df64(self.ctx, _ptr(u), _ptr(f)))
        return u

    def vcycle(self, u, f):
        if u.dtype == torch.float32:
            self._vec(u, self.L, torch.float32, "u")
            self._vec(f, self.L, torch.float32, "f")
            self._check(self.lib.mg_vcycle_f32(self.ctx, _ptr(u), _ptr(f)))
            return u
        self._vec(u, self.L, name="u")
        self._vec(f, self.L, name="f")
        self._check(self.lib.mg_vcycle(self.ctx, _ptr(u), _ptr(f)))
        return u

    def solve(self, f, u=None, tol=1e-10, maxit=200, use_cg=False, raise_on_noconv=True):
        """Solve A u = f in place on u (zeros if None).  Returns (u, iterations,
        relative residual, residual-norm history as numpy array)."""
        self._vec(f, self.L, name="f")
        u = self.zeros() if u is None else self._vec(u, self.L, name="u")
        its = ctypes.c_int()
        rel = ctypes.c_double()
        hist = np.zeros(maxit + 1)
        st = self.lib.mg_solve(self.ctx, _ptr(u), _ptr(f), float(tol), int(maxit), int(bool(use_cg)),
                               ctypes.byref(its), ctypes.byref(rel), hist.ctypes.data_as(ctypes.c_void_p))
        if st != 0 and (raise_on_noconv or st != _lib.MG_ENOCONV):
            self._check(st)
        return u, its.value, rel.value, hist[:its.value + 1]

    def solve_host(self, f_host, u_host=None, tol=1e-10, maxit=200, use_cg=False):
        """mg_solve_host: numpy / pinned-CPU-tensor buffers in, solution out."""
        n = self.num_dofs()
        f_host = np.ascontiguousarray(f_host, dtype=np.float64) if not isinstance(f_host, torch.Tensor) else f_host
        if u_host is None:
            u_host = np.zeros(n)
        its = ctypes.c_int()
        rel = ctypes.c_double()
        hist = np.zeros(maxit + 1)
        fp = f_host.data_ptr() if isinstance(f_host, torch.Tensor) else f_host.ctypes.data
        up = u_host.data_ptr() if isinstance(u_host, torch.Tensor) else u_host.ctypes.data
        st = self.lib.mg_solve_host(self.ctx, ctypes.c_void_p(up), ctypes.c_void_p(fp), float(tol), int(maxit),
                                    int(bool(use_cg)), ctypes.byref(its), ctypes.byref(rel),
                                    hist.ctypes.data_as(ctypes.c_void_p))
        self._check(st)
        return u_host, its.value, rel.value, hist[:its.value + 1]

    # -- instrumentation ------------------------------------------------------
    def kernel_launches(self):
        return int(self.lib.mg_kernel_launches(self.ctx))

    def batch_launches(self):
        """Kernels launched by the batched solves this solver led (first in the list)."""
        return int(self.lib.mg_batch_launches(self.ctx))

    def profile(self, enable=True):
        self._check(self.lib.mg_profile(self.ctx, int(bool(enable))))

    PROFILE_KINDS = {"fdm": 0, "scatter": 1, "sipg": 2, "restrict": 3, "prolong": 4, "coarse": 5, "vector": 6,
                     "outer": 7}

    def profile_result(self, kind, level=-1):
        """(total ms, number of kernel groups) recorded for one kind / level."""
        ms = ctypes.c_double()
        cnt = ctypes.c_longlong()
        self._check(self.lib.mg_profile_result(self.ctx, self.PROFILE_KINDS[kind], int(level), ctypes.byref(ms),
                                               ctypes.byref(cnt)))
        return ms.value, cnt.value

    def get_table(self, level, direction, what):
        """Copy a 1D setup table to a numpy array (see mg_get_table)."""
        cap = 1 << 16
        buf = np.zeros(cap)
        cnt = ctypes.c_int()
        self._check(self.lib.mg_get_table(self.ctx, int(level), int(direction), int(what),
                                          buf.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(cnt)))
        return buf[:cnt.value].copy()

    def get_line_table(self, level, direction, line, what):
        """Copy a table of one element line of a graded mesh (see mg_get_line_table)."""
        cap = 1 << 16
        buf = np.zeros(cap)
        cnt = ctypes.c_int()
        self._check(self.lib.mg_get_line_table(self.ctx, int(level), int(direction), int(line), int(what),
                                               buf.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(cnt)))
        return buf[:cnt.value].copy()


def solve_batch(solvers, fs, us=None, tol=1e-10, maxit=200):
    """mg_solve_batch: MG-CG solves of several problems (one MGSolver each,
    distinct) advanced together, every sweep one launch for all of them, on
    the first solver's stream.  Returns (us, iterations, relative residuals,
    statuses), one entry per problem; raises only for argument or CUDA
    errors (per-problem outcomes are in the statuses, 0 = converged)."""
    n = len(solvers)
    if n != len(fs):
        raise ValueError("one right-hand side per solver")
    for s, f in zip(solvers, fs):
        s._vec(f, s.L, name="f")
    us = [s.zeros() for s in solvers] if us is None else [s._vec(u, s.L, name="u") for s, u in zip(solvers, us)]
    P = ctypes.c_void_p
    ctxs = (P * n)(*[s.ctx for s in solvers])
    up = (P * n)(*[_ptr(u) for u in us])
    fp = (P * n)(*[_ptr(f) for f in fs])
    its = (ctypes.c_int * n)()
    rel = (ctypes.c_double * n)()
    st = (ctypes.c_int * n)()
    lib = solvers[0].lib
    solvers[0]._check(lib.mg_solve_batch(ctypes.cast(ctxs, P), n, ctypes.cast(up, P), ctypes.cast(fp, P),
                                         float(tol), int(maxit), ctypes.cast(its, P), ctypes.cast(rel, P),
                                         ctypes.cast(st, P)))
    return us, list(its), list(rel), list(st)
