"""ctypes binding of libgblb (C ABI in include/lb.h).

Functions keep the C names and only marshal arguments; every numerical step runs in the
CUDA library.  ``Simulation`` is a convenience wrapper that binds a torch-owned device
workspace and torch's current stream to a context.  Importing this module raises if the
library has not been built (``python -c "import __graft_entry__ as g; g.build()"``): there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libgblb.so")
if not os.path.exists(_LIBPATH):
    raise ImportError(f"{_LIBPATH} is missing: build it with __graft_entry__.build() (needs nvcc)")
_lib = C.CDLL(_LIBPATH)

LB_OK, LB_ERR_ARG, LB_ERR_CUDA, LB_ERR_OOM, LB_ERR_FENE, LB_ERR_NONFINITE, LB_ERR_TIMEOUT, LB_ERR_STATE = range(8)
LB_FP64, LB_FP32, LB_BF16, LB_FP16 = range(4)
LB_NOBS = 20

_dp = C.POINTER(C.c_double)
_vp = C.c_void_p
_SIGS = {
    "lb_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                            C.c_double, C.c_double, C.c_uint64, C.c_int]),
    "lb_add_chain": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                               C.c_double, _dp, _dp, C.c_double, C.c_int]),
    "lb_set_options": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _dp, C.c_int]),
    "lb_set_stream": (C.c_int, [_vp, _vp]),
    "lb_set_md_substeps": (C.c_int, [_vp, C.c_int]),
    "lb_batch_accumulate": (C.c_int, [_vp]),
    "lb_workspace_size": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "lb_bind_workspace": (C.c_int, [_vp, _vp, C.c_size_t]),
    "lb_step": (C.c_int, [_vp, C.c_int64]),
    "lb_sync": (C.c_int, [_vp]),
    "lb_get_populations": (C.c_int, [_vp, _dp, C.c_size_t]),
    "lb_set_populations": (C.c_int, [_vp, _dp, C.c_size_t]),
    "lb_get_beads": (C.c_int, [_vp, _dp, _dp, C.c_size_t]),
    "lb_get_beads_async": (C.c_int, [_vp, _dp, _dp, C.c_size_t, C.POINTER(C.c_int64)]),
    "lb_wait": (C.c_int, [_vp, C.c_int64]),
    "lb_get_observables": (C.c_int, [_vp, _dp, C.c_size_t]),
    "lb_set_obs_stride": (C.c_int, [_vp, C.c_int]),
    "lb_record_trajectory": (C.c_int, [_vp, _vp, C.c_int, C.c_int]),
    "lb_trajectory_frames": (C.c_int, [_vp, C.POINTER(C.c_int64)]),
    "lb_analysis_msd": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp]),
    "lb_analysis_rouse_modes": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp]),
    "lb_analysis_rouse_correlation": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp]),
    "lb_analysis_static_sk": (C.c_int, [_vp, C.c_int, C.c_int, _vp, C.c_int, _vp, _vp]),
    "lb_analysis_dynamic_sk": (C.c_int, [_vp, C.c_int, C.c_int, _vp, C.c_int, C.c_int, C.c_int, _vp, _vp]),
    "lb_analysis_inverse_radius": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp]),
    "lb_bd_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                               C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                               C.c_uint64, _dp, C.c_int]),
    "lb_bd_set_stream": (C.c_int, [_vp, _vp]),
    "lb_bd_step": (C.c_int, [_vp, C.c_int64]),
    "lb_bd_sync": (C.c_int, [_vp]),
    "lb_bd_get_beads": (C.c_int, [_vp, _dp, C.c_size_t]),
    "lb_bd_get_step": (C.c_int64, [_vp]),
    "lb_bd_destroy": (None, [_vp]),
    "lb_reset_reference": (C.c_int, [_vp]),
    "lb_save": (C.c_int, [_vp, C.c_char_p]),
    "lb_load": (C.c_int, [_vp, C.c_char_p]),
    "lb_get_step": (C.c_int64, [_vp]),
    "lb_adjoint_displacement": (C.c_int, [_vp, C.c_int64, C.c_int, _dp, _dp, C.c_size_t, _dp]),
    "lb_set_timing": (C.c_int, [_vp, C.c_int]),
    "lb_get_timing": (C.c_int, [_vp, _dp, C.POINTER(C.c_int64)]),
    "lb_destroy": (None, [_vp]),
    "lb_strerror": (C.c_char_p, [C.c_int]),
    "lb_last_error": (C.c_size_t, [C.c_char_p, C.c_size_t]),
    "lb_philox4x32_10": (C.c_int, [_vp, C.c_int64, C.c_uint32, C.c_uint32, _vp, _vp]),
    "lb_cell_index_f32": (C.c_int, [_vp, C.c_int64, C.c_float, C.c_int, _vp, _vp]),
    "lb_debug_coupling_cells": (C.c_int, [_vp, C.POINTER(C.c_int32), _dp, C.c_size_t]),
    "lb_fluid_sums_noalloc": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double, _dp, _vp]),
    "lb_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_uint64), C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_double, C.c_double, _dp, C.c_int, C.c_int]),
    "lb_batch_set_stream": (C.c_int, [_vp, _vp]),
    "lb_batch_workspace_size": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "lb_batch_bind_workspace": (C.c_int, [_vp, _vp, C.c_size_t]),
    "lb_batch_set_shape": (C.c_int, [_vp, C.c_int, C.c_int]),
    "lb_batch_set_options": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
    "lb_batch_autotune": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lb_batch_step": (C.c_int, [_vp, C.c_int64]),
    "lb_batch_sync": (C.c_int, [_vp]),
    "lb_batch_get_populations": (C.c_int, [_vp, C.c_int, _dp, C.c_size_t]),
    "lb_batch_get_beads": (C.c_int, [_vp, C.c_int, _dp, _dp, C.c_size_t]),
    "lb_batch_get_observables": (C.c_int, [_vp, C.c_int, _dp, C.c_size_t]),
    "lb_batch_nodes": (C.c_int64, [_vp]),
    "lb_batch_destroy": (None, [_vp]),
}
LB_NOALLOC_MAX_L = 256
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def library_path() -> str:
    return _LIBPATH


class LBError(RuntimeError):
    def __init__(self, code: int, where: str):
        detail = lb_last_error()
        super().__init__(f"{where}: {lb_strerror(code)} (status {code})" + (f": {detail}" if detail else ""))
        self.code = code
        self.detail = detail


def _check(code: int, where: str) -> None:
    if code != LB_OK:
        raise LBError(code, where)


def _dbuf(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _out64(a, need: int, where: str):
    """Pointer to a caller's output array after checking that the library may write `need`
    doubles into it (None passes through): the C side only knows the capacity it is told."""
    if a is None:
        return None
    if (not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous
            or not a.flags.writeable):
        raise ValueError(f"{where}: output must be a writable C-contiguous float64 numpy array")
    if a.size < need:
        raise ValueError(f"{where}: output holds {a.size} values, {need} are written")
    return a.ctypes.data_as(_dp)


# --- C functions, same names -----------------------------------------------------------
def lb_strerror(code: int) -> str:
    return _lib.lb_strerror(code).decode()


def lb_last_error() -> str:
    """The message of this thread's last failing call (and clears it); '' when none."""
    buf = C.create_string_buffer(512)
    _lib.lb_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def lb_create(L, rho, eta, eta_b, kT, h, a, seed, precision):
    ctx = _vp()
    _check(_lib.lb_create(C.byref(ctx), int(L), rho, eta, eta_b, kT, h, a, int(seed), int(precision)), "lb_create")
    return ctx


def lb_add_chain(ctx, N, m, zeta, k_fene, R0, eps, sigma, x0=None, v0=None, bond=0.97, saw=1):
    x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).reshape(-1)
    v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64).reshape(-1)
    for name, arr in (("x0", x0), ("v0", v0)):
        if arr is not None and arr.size != 3 * int(N):
            raise ValueError(f"lb_add_chain: {name} must hold 3 N = {3 * int(N)} values, got {arr.size}")
    _check(_lib.lb_add_chain(ctx, int(N), m, zeta, k_fene, R0, eps, sigma, _dbuf(x0), _dbuf(v0), bond, int(saw)),
           "lb_add_chain")


def lb_set_options(ctx, noise_fluid=1, noise_beads=1, stress_only=0, ext_bead_force=None, counter_force_fluid=0):
    ext = None if ext_bead_force is None else np.ascontiguousarray(ext_bead_force, dtype=np.float64).reshape(-1)
    if ext is not None and ext.size != 3:
        raise ValueError("lb_set_options: ext_bead_force must hold 3 values")
    _check(_lib.lb_set_options(ctx, int(noise_fluid), int(noise_beads), int(stress_only), _dbuf(ext),
                               int(counter_force_fluid)), "lb_set_options")


def lb_set_md_substeps(ctx, n: int):
    _check(_lib.lb_set_md_substeps(ctx, int(n)), "lb_set_md_substeps")


def lb_batch_accumulate(b):
    _check(_lib.lb_batch_accumulate(b), "lb_batch_accumulate")


def lb_set_stream(ctx, stream_handle: int):
    _check(_lib.lb_set_stream(ctx, _vp(stream_handle) if stream_handle else None), "lb_set_stream")


def lb_workspace_size(ctx) -> int:
    n = C.c_size_t()
    _check(_lib.lb_workspace_size(ctx, C.byref(n)), "lb_workspace_size")
    return n.value


def lb_bind_workspace(ctx, device_ptr: int, nbytes: int):
    _check(_lib.lb_bind_workspace(ctx, _vp(device_ptr), nbytes), "lb_bind_workspace")


def lb_step(ctx, n: int):
    _check(_lib.lb_step(ctx, int(n)), "lb_step")


def lb_sync(ctx):
    _check(_lib.lb_sync(ctx), "lb_sync")


def lb_get_populations(ctx, out: np.ndarray):
    _check(_lib.lb_get_populations(ctx, _out64(out, 0, "lb_get_populations"), out.size), "lb_get_populations")


def lb_set_populations(ctx, arr: np.ndarray):
    arr = np.ascontiguousarray(arr, dtype=np.float64)
    _check(_lib.lb_set_populations(ctx, _dbuf(arr), arr.size), "lb_set_populations")


def lb_get_beads(ctx, x: np.ndarray | None, v: np.ndarray | None, cap: int):
    _check(_lib.lb_get_beads(ctx, _out64(x, cap, "lb_get_beads"), _out64(v, cap, "lb_get_beads"), cap),
           "lb_get_beads")


def lb_get_beads_async(ctx, x: np.ndarray, v, cap: int) -> int:
    """Enqueue a bead read-back into x (and v) without waiting; returns the ticket for
    lb_wait.  The arrays must stay alive (and should be pinned) until then."""
    t = C.c_int64()
    _check(_lib.lb_get_beads_async(ctx, _out64(x, cap, "lb_get_beads_async"),
                                   _out64(v, cap, "lb_get_beads_async"), cap, C.byref(t)),
           "lb_get_beads_async")
    return t.value


def lb_wait(ctx, ticket: int):
    _check(_lib.lb_wait(ctx, int(ticket)), "lb_wait")


def lb_get_observables(ctx) -> np.ndarray:
    out = np.zeros(LB_NOBS)
    _check(_lib.lb_get_observables(ctx, _dbuf(out), out.size), "lb_get_observables")
    return out


def lb_set_obs_stride(ctx, stride: int):
    _check(_lib.lb_set_obs_stride(ctx, int(stride)), "lb_set_obs_stride")


def lb_record_trajectory(ctx, traj_ptr: int, capacity: int, stride: int):
    _check(_lib.lb_record_trajectory(ctx, traj_ptr, int(capacity), int(stride)), "lb_record_trajectory")


def lb_trajectory_frames(ctx) -> int:
    n = C.c_int64()
    _check(_lib.lb_trajectory_frames(ctx, C.byref(n)), "lb_trajectory_frames")
    return n.value


def lb_analysis_msd(traj_ptr, T, N, max_lag, i0, i1, out_ptr, stream):
    _check(_lib.lb_analysis_msd(traj_ptr, T, N, max_lag, i0, i1, out_ptr, stream), "lb_analysis_msd")


def lb_analysis_rouse_modes(traj_ptr, T, N, P, X_ptr, stream):
    _check(_lib.lb_analysis_rouse_modes(traj_ptr, T, N, P, X_ptr, stream), "lb_analysis_rouse_modes")


def lb_analysis_rouse_correlation(X_ptr, T, P, max_lag, c_ptr, stream):
    _check(_lib.lb_analysis_rouse_correlation(X_ptr, T, P, max_lag, c_ptr, stream), "lb_analysis_rouse_correlation")


def lb_analysis_static_sk(traj_ptr, T, N, k_ptr, nk, S_ptr, stream):
    _check(_lib.lb_analysis_static_sk(traj_ptr, T, N, k_ptr, nk, S_ptr, stream), "lb_analysis_static_sk")


def lb_analysis_inverse_radius(traj_ptr, T, N, out_ptr, stream):
    _check(_lib.lb_analysis_inverse_radius(traj_ptr, T, N, out_ptr, stream), "lb_analysis_inverse_radius")


def lb_analysis_dynamic_sk(traj_ptr, T, N, k_ptr, nk, max_lag, origin_stride, S_ptr, stream):
    _check(_lib.lb_analysis_dynamic_sk(traj_ptr, T, N, k_ptr, nk, max_lag, origin_stride, S_ptr, stream),
           "lb_analysis_dynamic_sk")


def lb_reset_reference(ctx):
    _check(_lib.lb_reset_reference(ctx), "lb_reset_reference")


def lb_save(ctx, path: str):
    _check(_lib.lb_save(ctx, path.encode()), "lb_save")


def lb_load(ctx, path: str):
    _check(_lib.lb_load(ctx, path.encode()), "lb_load")


def lb_adjoint_displacement(ctx, T: int, K: int, N: int):
    """(O, dO/dx0 (N,3), dO/dzeta) for O = sum_b |x_b(T) - x_b(0)|^2, noise held fixed."""
    obj = C.c_double()
    gz = C.c_double()
    gx = np.zeros((N, 3))
    _check(_lib.lb_adjoint_displacement(ctx, int(T), int(K), C.byref(obj), _dbuf(gx), gx.size, C.byref(gz)),
           "lb_adjoint_displacement")
    return obj.value, gx, gz.value


def lb_get_step(ctx) -> int:
    return int(_lib.lb_get_step(ctx))


def lb_set_timing(ctx, enable: bool):
    _check(_lib.lb_set_timing(ctx, int(enable)), "lb_set_timing")


def lb_get_timing(ctx):
    ms = C.c_double()
    n = C.c_int64()
    _check(_lib.lb_get_timing(ctx, C.byref(ms), C.byref(n)), "lb_get_timing")
    return ms.value, n.value


def lb_destroy(ctx):
    _lib.lb_destroy(ctx)


def lb_philox4x32_10(ctr_dev_ptr: int, n: int, k0: int, k1: int, out_dev_ptr: int, stream: int = 0):
    _check(_lib.lb_philox4x32_10(_vp(ctr_dev_ptr), n, k0, k1, _vp(out_dev_ptr), _vp(stream) if stream else None),
           "lb_philox4x32_10")


def lb_debug_coupling_cells(ctx, N: int, substeps: int = 1):
    """Test hook: (corner nodes (substeps, N, 8) int32, stored coordinates (N, 3)) of the last
    step's coupling, as the bead kernel used them."""
    cap = max(8 * N * substeps, 3 * N)
    nodes = np.empty(cap, dtype=np.int32)
    xs = np.empty(cap, dtype=np.float64)
    _check(_lib.lb_debug_coupling_cells(ctx, nodes.ctypes.data_as(C.POINTER(C.c_int32)), _dbuf(xs), cap),
           "lb_debug_coupling_cells")
    return nodes[:8 * N * substeps].reshape(substeps, N, 8), xs[:3 * N].reshape(N, 3)


def lb_cell_index_f32(x_dev_ptr: int, n: int, a: float, L: int, out_dev_ptr: int, stream: int = 0):
    _check(_lib.lb_cell_index_f32(_vp(x_dev_ptr), n, a, L, _vp(out_dev_ptr), _vp(stream) if stream else None),
           "lb_cell_index_f32")


def lb_fluid_sums_noalloc(pop_dev_ptr: int, L: int, a: float, h: float, stream: int = 0) -> np.ndarray:
    """Mass and momentum of a device population field (19 L^3 FP64) without any device
    allocation: the library's fixed scratch array holds the partial sums."""
    out = np.zeros(4)
    _check(_lib.lb_fluid_sums_noalloc(_vp(pop_dev_ptr), int(L), a, h, _dbuf(out), _vp(stream) if stream else None),
           "lb_fluid_sums_noalloc")
    return out


def lb_batch_create(L, N, seeds, rho, eta, eta_b, kT, h, a, m, zeta, k_fene, R0, eps, sigma, x0, precision,
                    md_substeps=1):
    R = len(L)
    Ls = (C.c_int * R)(*[int(v) for v in L])
    Ns = (C.c_int * R)(*[int(v) for v in N])
    Ss = (C.c_uint64 * R)(*[int(v) for v in seeds])
    xa = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).reshape(-1)
    if xa is not None and xa.size != 3 * sum(int(v) for v in N):
        raise ValueError(f"lb_batch_create: x0 must hold 3 sum(N) = {3 * sum(int(v) for v in N)} values")
    b = _vp()
    _check(_lib.lb_batch_create(C.byref(b), R, Ls, Ns, Ss, rho, eta, eta_b, kT, h, a, m, zeta, k_fene, R0, eps,
                                sigma, _dbuf(xa), int(precision), int(md_substeps)), "lb_batch_create")
    return b


def lb_batch_set_stream(b, stream_handle: int):
    _check(_lib.lb_batch_set_stream(b, _vp(stream_handle) if stream_handle else None), "lb_batch_set_stream")


def lb_batch_workspace_size(b) -> int:
    n = C.c_size_t()
    _check(_lib.lb_batch_workspace_size(b, C.byref(n)), "lb_batch_workspace_size")
    return n.value


def lb_batch_bind_workspace(b, device_ptr: int, nbytes: int):
    _check(_lib.lb_batch_bind_workspace(b, _vp(device_ptr), nbytes), "lb_batch_bind_workspace")


def lb_batch_set_shape(b, threads: int, blocks_per_sm: int):
    _check(_lib.lb_batch_set_shape(b, int(threads), int(blocks_per_sm)), "lb_batch_set_shape")


def lb_batch_set_options(b, noise_fluid=1, noise_beads=1, stress_only=0):
    _check(_lib.lb_batch_set_options(b, int(noise_fluid), int(noise_beads), int(stress_only)), "lb_batch_set_options")


def lb_batch_autotune(b):
    t, k = C.c_int(), C.c_int()
    _check(_lib.lb_batch_autotune(b, C.byref(t), C.byref(k)), "lb_batch_autotune")
    return t.value, k.value


def lb_batch_step(b, n: int):
    _check(_lib.lb_batch_step(b, int(n)), "lb_batch_step")


def lb_batch_sync(b):
    _check(_lib.lb_batch_sync(b), "lb_batch_sync")


def lb_batch_get_populations(b, r: int, out: np.ndarray):
    _check(_lib.lb_batch_get_populations(b, int(r), _out64(out, 0, "lb_batch_get_populations"), out.size),
           "lb_batch_get_populations")


def lb_batch_get_beads(b, r: int, x, v, cap: int):
    _check(_lib.lb_batch_get_beads(b, int(r), _out64(x, cap, "lb_batch_get_beads"),
                                   _out64(v, cap, "lb_batch_get_beads"), cap), "lb_batch_get_beads")


def lb_batch_get_observables(b, r: int) -> np.ndarray:
    out = np.zeros(LB_NOBS)
    _check(_lib.lb_batch_get_observables(b, int(r), _dbuf(out), out.size), "lb_batch_get_observables")
    return out


def lb_batch_nodes(b) -> int:
    return int(_lib.lb_batch_nodes(b))


def lb_batch_destroy(b):
    _lib.lb_batch_destroy(b)


class Batch:
    """R replicas (box sizes L[r], chains N[r] with positions X0[r]) on the current device,
    workspace in a torch tensor, work on torch's current stream."""

    def __init__(self, L, N, seeds, X0, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=0.01, a=1.0, m=1.0, zeta=20.8,
                 k_fene=30.0, R0=1.5, eps=1.0, sigma=1.0, precision=LB_FP32, md_substeps=1, stress_only=False):
        import torch

        self.L = [int(v) for v in L]
        self.N = [int(v) for v in N]
        xs = [np.asarray(x, dtype=np.float64).reshape(-1) for x, n in zip(X0, self.N) if n > 0]
        x0 = np.concatenate(xs) if xs else None
        self.b = lb_batch_create(self.L, self.N, seeds, rho, eta, eta_b, kT, h, a, m, zeta, k_fene, R0, eps,
                                 sigma, x0, precision, md_substeps)
        lb_batch_set_stream(self.b, torch.cuda.current_stream().cuda_stream)
        nbytes = lb_batch_workspace_size(self.b)
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        lb_batch_bind_workspace(self.b, self._ws.data_ptr(), nbytes)
        if stress_only:
            lb_batch_set_options(self.b, 1, 1, 1)

    def step(self, n=1):
        lb_batch_step(self.b, n)

    def sync(self):
        lb_batch_sync(self.b)

    def populations(self, r):
        out = np.empty((19, self.L[r], self.L[r], self.L[r]))
        lb_batch_get_populations(self.b, r, out)
        return out

    def beads(self, r):
        x = np.empty((self.N[r], 3))
        v = np.empty((self.N[r], 3))
        lb_batch_get_beads(self.b, r, x, v, 3 * self.N[r])
        return x, v

    def observables(self, r):
        return lb_batch_get_observables(self.b, r)

    def accumulate(self):
        lb_batch_accumulate(self.b)

    def close(self):
        if self.b:
            lb_batch_destroy(self.b)
            self.b = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- convenience wrapper ---------------------------------------------------------------
class Simulation:
    """One fluid box (+ optional chain) on the current CUDA device, with its workspace in a
    torch tensor and its work on torch's current stream."""

    def __init__(self, L, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=0.01, a=1.0, seed=1, precision=LB_FP32,
                 torch_workspace=True):
        self.L = int(L)
        self.N = 0
        self.ctx = lb_create(L, rho, eta, eta_b, kT, h, a, seed, precision)
        self._ws = None
        self._torch_workspace = torch_workspace
        self._bound = False

    def add_chain(self, N, m=1.0, zeta=20.8, k_fene=30.0, R0=1.5, eps=1.0, sigma=1.0, x0=None, v0=None,
                  bond=0.97, saw=1):
        lb_add_chain(self.ctx, N, m, zeta, k_fene, R0, eps, sigma, x0, v0, bond, saw)
        self.N = int(N)

    def set_options(self, **kw):
        lb_set_options(self.ctx, **kw)

    def set_md_substeps(self, n: int):
        lb_set_md_substeps(self.ctx, n)

    def _bind(self):
        if self._bound:
            return
        import torch

        lb_set_stream(self.ctx, torch.cuda.current_stream().cuda_stream)
        if self._torch_workspace:
            nbytes = lb_workspace_size(self.ctx)
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            lb_bind_workspace(self.ctx, self._ws.data_ptr(), nbytes)
        self._bound = True

    def step(self, n=1):
        self._bind()
        lb_step(self.ctx, n)

    def sync(self):
        self._bind()
        lb_sync(self.ctx)

    def populations(self) -> np.ndarray:
        self._bind()
        out = np.empty((19, self.L, self.L, self.L))
        lb_get_populations(self.ctx, out)
        return out

    def set_populations(self, arr):
        self._bind()
        lb_set_populations(self.ctx, arr)

    def beads(self):
        self._bind()
        x = np.empty((self.N, 3))
        v = np.empty((self.N, 3))
        lb_get_beads(self.ctx, x, v, 3 * self.N)
        return x, v

    def observables(self) -> np.ndarray:
        self._bind()
        return lb_get_observables(self.ctx)

    def record_trajectory(self, stride: int, capacity: int):
        """Record the unwrapped bead positions now and after every `stride` steps into a
        device ring of `capacity` frames (a torch float64 tensor owned by this object)."""
        import torch

        self._bind()
        self._traj = torch.empty((int(capacity), self.N, 3), dtype=torch.float64, device="cuda")
        lb_record_trajectory(self.ctx, self._traj.data_ptr(), capacity, stride)

    def trajectory(self):
        """The recorded frames, oldest first, as a (T, N, 3) float64 CUDA tensor."""
        import torch

        self.sync()
        n = lb_trajectory_frames(self.ctx)
        cap = self._traj.shape[0]
        if n <= cap:
            return self._traj[:n]
        return torch.roll(self._traj, -(n % cap), dims=0)

    def save(self, path: str):
        self._bind()
        lb_save(self.ctx, path)

    def load(self, path: str):
        self._bind()
        lb_load(self.ctx, path)

    def close(self):
        if self.ctx:
            lb_destroy(self.ctx)
            self.ctx = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- Brownian dynamics (Sec. II C) --------------------------------------------------------
def lb_bd_create(replicas, N, kT, zeta, eta_s, dt, k_fene, R0, eps, sigma, hi, degree, power_iters, seed, x0,
                 precision):
    b = _vp()
    x = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1)
    if x.size != replicas * N * 3:
        raise ValueError("x0 must hold replicas x N x 3 positions")
    _check(_lib.lb_bd_create(C.byref(b), int(replicas), int(N), kT, zeta, eta_s, dt, k_fene, R0, eps, sigma,
                             int(hi), int(degree), int(power_iters), int(seed), _dbuf(x), int(precision)),
           "lb_bd_create")
    return b


def lb_bd_set_stream(b, stream):
    _check(_lib.lb_bd_set_stream(b, stream), "lb_bd_set_stream")


def lb_bd_step(b, n):
    _check(_lib.lb_bd_step(b, int(n)), "lb_bd_step")


def lb_bd_sync(b):
    _check(_lib.lb_bd_sync(b), "lb_bd_sync")


def lb_bd_get_beads(b, out: np.ndarray):
    _check(_lib.lb_bd_get_beads(b, _out64(out, 0, "lb_bd_get_beads"), out.size), "lb_bd_get_beads")


def lb_bd_get_step(b) -> int:
    return _lib.lb_bd_get_step(b)


def lb_bd_destroy(b):
    _lib.lb_bd_destroy(b)


class BD:
    """Brownian-dynamics chains with hydrodynamic interaction (Sec. II C) on the current CUDA
    device, on torch's current stream.  Parameters in the units the caller chooses; the
    defaults are the paper's production chain in MD/LB units with zeta = zeta_eff (Sec. II D)
    and the time step 0.005 tau_k."""

    def __init__(self, x0, kT=1.2, zeta=None, eta_s=0.864 * 2.8, dt=None, k_fene=7.0, R0=2.0, eps=1.0, sigma=1.0,
                 hi=True, degree=20, power_iters=20, seed=1, precision=LB_FP32):
        import torch

        x0 = np.asarray(x0, dtype=np.float64)
        if x0.ndim == 2:
            x0 = x0[None]
        self.R, self.N = x0.shape[0], x0.shape[1]
        if zeta is None:
            zeta = zeta_eff(20.8, eta_s)
        if dt is None:
            dt = 0.005 * zeta / (4.0 * k_fene)
        self.b = lb_bd_create(self.R, self.N, kT, zeta, eta_s, dt, k_fene, R0, eps, sigma, int(hi), degree,
                              power_iters, seed, x0, precision)
        lb_bd_set_stream(self.b, torch.cuda.current_stream().cuda_stream)

    def step(self, n=1):
        lb_bd_step(self.b, n)

    def sync(self):
        lb_bd_sync(self.b)

    def beads(self) -> np.ndarray:
        out = np.empty((self.R, self.N, 3))
        lb_bd_get_beads(self.b, out)
        return out

    def close(self):
        if self.b:
            lb_bd_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zeta_eff(zeta_bare: float, eta_s: float, a: float = 1.0, g: float = 25.0) -> float:
    """Long-time friction of a point particle coupled to the LB fluid (Sec. II D): 1/zeta_eff =
    1/zeta_bare + 1/(g eta_s a), g ~ 25 for linear interpolation to the nearest nodes."""
    return 1.0 / (1.0 / zeta_bare + 1.0 / (g * eta_s * a))
