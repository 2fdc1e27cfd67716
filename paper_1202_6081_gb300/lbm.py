"""Python binding of liblbm.so (include/lbm.h).

The module-level functions carry the C-ABI names and only marshal arguments
(ctypes pointers from torch tensors, the current CUDA stream); every step of
the method runs in the library's CUDA kernels.  There is no CPU fallback: if
liblbm.so is missing or no GPU is present the calls raise.

``Solver`` is a convenience owner of the two state buffers (torch uint8
tensors sized by ``lbm_state_bytes``) around one context.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_D3Q15 = 15
LBM_D3Q27 = 27
LBM_STORE_F32 = 0
LBM_STORE_F16 = 1
LBM_STORE_BF16 = 2
LBM_WALL_Y = 1
LBM_WALL_Z = 2
LBM_INPLACE = 4
LBM_F32_SR = 8
STORAGE = {"f32": LBM_STORE_F32, "f16": LBM_STORE_F16, "bf16": LBM_STORE_BF16}

LBM_OK = 0
_STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ESTATE", 4: "LBM_ECUDA",
           5: "LBM_ENONFINITE", 6: "LBM_EUNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class LBMError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = "%s failed: %s" % (where, _STATUS.get(status, str(status)))
        if detail:
            msg += " (%s)" % detail
        super().__init__(msg)


def load():
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblbm.so not found at %s: build it with "
                               "paper_1202_6081_gb300.build.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        ctx_pp = ctypes.POINTER(ctypes.c_void_p)
        sigs = {
            "lbm_create": ([ip, ip, ip, ip, dp, dp, ctypes.c_uint, ip, ctx_pp], ip),
            "lbm_destroy": ([vp], None),
            "lbm_state_bytes": ([vp], ctypes.c_size_t),
            "lbm_row_pitch": ([vp], ip),
            "lbm_bind": ([vp, vp, vp, vp], ip),
            "lbm_set_force": ([vp, dp], ip),
            "lbm_set_omega": ([vp, dp], ip),
            "lbm_init_equilibrium": ([vp, vp, vp, vp], ip),
            "lbm_set_state": ([vp, vp, vp], ip),
            "lbm_get_state": ([vp, vp, vp], ip),
            "lbm_step": ([vp, ip, vp], ip),
            "lbm_macroscopic": ([vp, vp, vp, vp], ip),
            "lbm_conservation": ([vp, dp, vp], ip),
            "lbm_status_string": ([ip], ctypes.c_char_p),
            "lbm_last_cuda_error": ([vp], ctypes.c_char_p),
            "lbm_set_force_field": ([vp, vp], ip),
            "lbm_adjoint_bytes": ([vp], ctypes.c_size_t),
            "lbm_current_state": ([vp], vp),
            "lbm_step_into": ([vp, vp, vp, vp], ip),
            "lbm_adjoint_step": ([vp, vp, vp, vp, vp, vp], ip),
            "lbm_kinetic_energy": ([vp, vp, dp, vp], ip),
            "lbm_kinetic_energy_seed": ([vp, vp, vp, vp, vp], ip),
            "lbm_conservation_noalloc": ([vp, vp, vp], ip),
            "lbm_macroscopic_seed": ([vp, vp, vp, vp, vp, vp, vp], ip),
            "lbm_set_graph_steps": ([vp, ip], ip),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def exported_symbols():
    """Names of every entry point the header declares, as loaded."""
    lib = load()
    names = []
    for n in ("lbm_create", "lbm_destroy", "lbm_state_bytes", "lbm_row_pitch", "lbm_bind",
              "lbm_set_force", "lbm_set_force_field", "lbm_set_omega", "lbm_init_equilibrium",
              "lbm_set_state", "lbm_get_state", "lbm_step", "lbm_macroscopic",
              "lbm_conservation", "lbm_status_string", "lbm_last_cuda_error",
              "lbm_adjoint_bytes", "lbm_current_state", "lbm_step_into", "lbm_adjoint_step",
              "lbm_kinetic_energy", "lbm_kinetic_energy_seed", "lbm_conservation_noalloc",
              "lbm_macroscopic_seed", "lbm_set_graph_steps"):
        getattr(lib, n)
        names.append(n)
    return names


def _check(status, where, ctx=None):
    if status != LBM_OK:
        detail = ""
        if ctx is not None and status == 4:
            detail = load().lbm_last_cuda_error(ctx).decode()
        raise LBMError(status, where, detail)


def _darr(values, n):
    arr = (ctypes.c_double * n)(*[float(v) for v in values])
    return arr


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---- C-ABI functions (same names, same argument order) --------------------

def lbm_create(lattice, nx, ny, nz, omega, force=None, bc_flags=0, storage=LBM_STORE_F32):
    lib = load()
    Q = int(lattice)
    om = _darr(omega, Q)
    F = _darr(force, 3) if force is not None else None
    ctx = ctypes.c_void_p()
    _check(lib.lbm_create(Q, nx, ny, nz, om, F, bc_flags, storage, ctypes.byref(ctx)),
           "lbm_create")
    return ctx


def lbm_destroy(ctx):
    load().lbm_destroy(ctx)


def lbm_state_bytes(ctx):
    return int(load().lbm_state_bytes(ctx))


def lbm_row_pitch(ctx):
    return int(load().lbm_row_pitch(ctx))


def lbm_bind(ctx, f_a, f_b, force_field=None):
    _check(load().lbm_bind(ctx, _ptr(f_a), _ptr(f_b), _ptr(force_field)), "lbm_bind", ctx)


def lbm_set_force(ctx, force):
    _check(load().lbm_set_force(ctx, _darr(force, 3) if force is not None else None),
           "lbm_set_force", ctx)


def lbm_set_omega(ctx, omega, Q):
    _check(load().lbm_set_omega(ctx, _darr(omega, Q)), "lbm_set_omega", ctx)


def lbm_init_equilibrium(ctx, rho, u, stream=None):
    _check(load().lbm_init_equilibrium(ctx, _ptr(rho), _ptr(u), _stream(stream)),
           "lbm_init_equilibrium", ctx)


def lbm_set_state(ctx, f, stream=None):
    _check(load().lbm_set_state(ctx, _ptr(f), _stream(stream)), "lbm_set_state", ctx)


def lbm_get_state(ctx, f, stream=None):
    _check(load().lbm_get_state(ctx, _ptr(f), _stream(stream)), "lbm_get_state", ctx)


def lbm_step(ctx, nsteps, stream=None):
    _check(load().lbm_step(ctx, int(nsteps), _stream(stream)), "lbm_step", ctx)


def lbm_macroscopic(ctx, rho, u, stream=None):
    _check(load().lbm_macroscopic(ctx, _ptr(rho), _ptr(u), _stream(stream)),
           "lbm_macroscopic", ctx)


def lbm_conservation(ctx, stream=None):
    out = (ctypes.c_double * 4)()
    _check(load().lbm_conservation(ctx, out, _stream(stream)), "lbm_conservation", ctx)
    return np.array(list(out))


def lbm_status_string(status):
    return load().lbm_status_string(int(status)).decode()


def lbm_set_force_field(ctx, force_field):
    _check(load().lbm_set_force_field(ctx, _ptr(force_field)), "lbm_set_force_field", ctx)


def lbm_adjoint_bytes(ctx):
    return int(load().lbm_adjoint_bytes(ctx))


def lbm_current_state(ctx):
    return load().lbm_current_state(ctx)


def lbm_step_into(ctx, f_in, f_out, stream=None):
    _check(load().lbm_step_into(ctx, _ptr(f_in), _ptr(f_out), _stream(stream)), "lbm_step_into",
           ctx)


def lbm_adjoint_step(ctx, f_t, lam_next, lam_out, dJdF=None, stream=None):
    _check(load().lbm_adjoint_step(ctx, _ptr(f_t), _ptr(lam_next), _ptr(lam_out), _ptr(dJdF),
                                   _stream(stream)), "lbm_adjoint_step", ctx)


def lbm_kinetic_energy(ctx, f=None, stream=None):
    out = ctypes.c_double()
    _check(load().lbm_kinetic_energy(ctx, _ptr(f), ctypes.byref(out), _stream(stream)),
           "lbm_kinetic_energy", ctx)
    return float(out.value)


def lbm_conservation_noalloc(ctx, out, stream=None):
    """Asynchronous conservation sums into the device tensor `out` (4 FP64:
    sum (rho - 1), sum rho u) without any allocation by the library."""
    if not (torch.is_tensor(out) and out.is_cuda and out.dtype == torch.float64
            and out.numel() >= 4 and out.is_contiguous()):
        raise ValueError("lbm_conservation_noalloc: out must be a contiguous CUDA float64 "
                         "tensor of at least 4 elements")
    _check(load().lbm_conservation_noalloc(ctx, _ptr(out), _stream(stream)),
           "lbm_conservation_noalloc", ctx)


def lbm_kinetic_energy_seed(ctx, f, lam_out, dJdF=None, stream=None):
    _check(load().lbm_kinetic_energy_seed(ctx, _ptr(f), _ptr(lam_out), _ptr(dJdF),
                                          _stream(stream)), "lbm_kinetic_energy_seed", ctx)


def lbm_set_graph_steps(ctx, steps):
    _check(load().lbm_set_graph_steps(ctx, int(steps)), "lbm_set_graph_steps", ctx)


def lbm_macroscopic_seed(ctx, f, g_rho, g_u, lam_out, dJdF=None, stream=None):
    _check(load().lbm_macroscopic_seed(ctx, _ptr(f), _ptr(g_rho), _ptr(g_u), _ptr(lam_out),
                                       _ptr(dJdF), _stream(stream)), "lbm_macroscopic_seed", ctx)


# ---- convenience owner ----------------------------------------------------

class Solver:
    """One grid on the current CUDA device.

    shape = (nz, ny, nx); omega: Q relaxation rates (0..3 ignored); force:
    uniform F (3,) or a per-cell field [3, nz, ny, nx] (device FP32 tensor or
    array); walls: OR of LBM_WALL_Y / LBM_WALL_Z; storage: "f32", "f16" or
    "bf16"; inplace: one state buffer with in-place (AA) streaming (nx
    even; no step_into / adjoint); sr32: stochastically rounded FP32 update
    (LBM_F32_SR; FP32 storage, not in place)."""

    def __init__(self, Q, shape, omega, force=(0.0, 0.0, 0.0), walls=0, storage="f32",
                 device=None, inplace=False, sr32=False):
        self.Q = int(Q)
        self.shape = tuple(int(s) for s in shape)
        nz, ny, nx = self.shape
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.storage = storage
        self.walls = walls
        self.inplace = bool(inplace)
        self.omega = np.asarray(omega, dtype=np.float64)
        with torch.cuda.device(self.device):
            field = None
            uniform = (0.0, 0.0, 0.0)
            F = np.asarray(force.cpu() if torch.is_tensor(force) else force)
            if F.ndim == 1:
                uniform = tuple(float(v) for v in F)
            else:
                field = torch.as_tensor(F, dtype=torch.float32).reshape(3, nz, ny, nx)
                field = field.to(self.device).contiguous()
            self.force_field = field
            flags = walls | (LBM_INPLACE if self.inplace else 0) | (LBM_F32_SR if sr32 else 0)
            self.ctx = lbm_create(self.Q, nx, ny, nz, self.omega, uniform, flags, STORAGE[storage])
            nbytes = lbm_state_bytes(self.ctx)
            self.buffers = [torch.empty(nbytes, dtype=torch.uint8, device=self.device)
                            for _ in range(1 if self.inplace else 2)]
            lbm_bind(self.ctx, self.buffers[0], self.buffers[1] if len(self.buffers) > 1 else None,
                     field)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and _lib is not None:
            try:
                torch.cuda.synchronize(self.device)
            except Exception:
                pass
            _lib.lbm_destroy(ctx)
            self.ctx = None

    @property
    def ncells(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    def _dev64(self, a, shape):
        t = torch.as_tensor(a, dtype=torch.float64)
        return t.reshape(shape).to(self.device).contiguous()

    def init_equilibrium(self, rho, u, stream=None):
        r = self._dev64(rho, self.shape)
        v = self._dev64(u, (3,) + self.shape)
        lbm_init_equilibrium(self.ctx, r, v, stream)
        self._keep = (r, v)  # alive until the stream has consumed them

    def set_state(self, f, stream=None):
        t = self._dev64(f, (self.Q,) + self.shape)
        lbm_set_state(self.ctx, t, stream)
        self._keep = (t,)

    def get_state(self, stream=None):
        out = torch.empty((self.Q,) + self.shape, dtype=torch.float64, device=self.device)
        lbm_get_state(self.ctx, out, stream)
        return out

    def step(self, nsteps=1, stream=None):
        lbm_step(self.ctx, nsteps, stream)

    def set_graph_steps(self, steps):
        """Steps per CUDA graph in step() (even; 0 = one launch per step)."""
        lbm_set_graph_steps(self.ctx, steps)

    def macroscopic(self, stream=None):
        rho = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        u = torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)
        lbm_macroscopic(self.ctx, rho, u, stream)
        return rho, u

    def conservation(self, stream=None):
        return lbm_conservation(self.ctx, stream)

    def set_force(self, force):
        lbm_set_force(self.ctx, force)

    def set_omega(self, omega):
        self.omega = np.asarray(omega, dtype=np.float64)
        lbm_set_omega(self.ctx, self.omega, self.Q)

    def set_force_field(self, field):
        """Bind a device FP32 force field [3, nz, ny, nx] (None: uniform)."""
        if field is not None:
            nz, ny, nx = self.shape
            assert field.dtype == torch.float32 and field.is_contiguous()
            assert tuple(field.shape) == (3, nz, ny, nx) and field.device == self.device
        self.force_field = field
        lbm_set_force_field(self.ctx, field)

    # ---- state buffers (checkpoints) and the adjoint --------------------

    def new_state_buffer(self):
        return torch.empty(lbm_state_bytes(self.ctx), dtype=torch.uint8, device=self.device)

    def current_buffer(self):
        """The bound buffer tensor holding the current state."""
        p = lbm_current_state(self.ctx)
        for b in self.buffers:
            if b.data_ptr() == p:
                return b
        raise RuntimeError("no current state")

    def load_buffer(self, src):
        """Make the state in buffer `src` the current state."""
        self.current_buffer().copy_(src)

    def step_into(self, src, dst, stream=None):
        lbm_step_into(self.ctx, src, dst, stream)

    def new_adjoint_field(self):
        n = lbm_adjoint_bytes(self.ctx) // 4
        return torch.zeros(n, dtype=torch.float32, device=self.device)

    def adjoint_step(self, f_t, lam_next, lam_out, dJdF=None, stream=None):
        lbm_adjoint_step(self.ctx, f_t, lam_next, lam_out, dJdF, stream)

    def kinetic_energy(self, buf=None, stream=None):
        return lbm_kinetic_energy(self.ctx, buf, stream)

    def kinetic_energy_seed(self, buf, lam_out, dJdF=None, stream=None):
        lbm_kinetic_energy_seed(self.ctx, buf, lam_out, dJdF, stream)

    def macroscopic_seed(self, buf, g_rho, g_u, lam_out, dJdF=None, stream=None):
        """lam_out = dJ/df of the state in `buf` for J(rho, u) with the given
        gradients (dense FP32 tensors, or None for zero)."""
        g_rho = None if g_rho is None else g_rho.to(self.device, torch.float32).contiguous()
        g_u = None if g_u is None else g_u.to(self.device, torch.float32).contiguous()
        lbm_macroscopic_seed(self.ctx, buf, g_rho, g_u, lam_out, dJdF, stream)
        self._keep = (g_rho, g_u)

    def adjoint_view(self, lam):
        """Dense [Q, nz, ny, nx] view of a pitched adjoint field."""
        nz, ny, nx = self.shape
        px = lbm_row_pitch(self.ctx)
        return lam.view(self.Q, nz, ny, px)[..., :nx]
