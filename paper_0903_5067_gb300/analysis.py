"""Chain observables of Sec. III A/B on the GPU: g1, g2, g3, Rouse modes and their time
correlation, S(k) and S(k, t), from a (T, N, 3) float64 CUDA tensor of unwrapped bead
positions (``Simulation.trajectory()``).  Argument marshalling only: the sums run in the
library's kernels (``lb_analysis_*`` in include/lb.h), on torch's current stream."""
from __future__ import annotations

import numpy as np

from . import lb


def _check_traj(traj):
    import torch

    if not (isinstance(traj, torch.Tensor) and traj.is_cuda and traj.dtype == torch.float64 and traj.dim() == 3
            and traj.shape[2] == 3):
        raise ValueError("trajectory must be a (T, N, 3) float64 CUDA tensor")
    return traj.contiguous()


def _stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


def inner_pair(N: int):
    """The two innermost monomers of an N-bead chain (0-based), used by g1 and g2."""
    return (N - 1) // 2, N // 2


def msd(traj, max_lag: int, pair=None):
    """g1, g2, g3 at lags 0..max_lag (numpy arrays)."""
    import torch

    traj = _check_traj(traj)
    T, N, _ = traj.shape
    i0, i1 = inner_pair(N) if pair is None else pair
    out = torch.empty((3, max_lag + 1), dtype=torch.float64, device=traj.device)
    lb.lb_analysis_msd(traj.data_ptr(), T, N, max_lag, i0, i1, out.data_ptr(), _stream())
    g = out.cpu().numpy()
    return g[0], g[1], g[2]


def rouse_modes(traj, P: int | None = None):
    """X_p(t), p = 1..P (default N-1), as a (T, P, 3) float64 CUDA tensor."""
    import torch

    traj = _check_traj(traj)
    T, N, _ = traj.shape
    P = N - 1 if P is None else P
    X = torch.empty((T, P, 3), dtype=torch.float64, device=traj.device)
    lb.lb_analysis_rouse_modes(traj.data_ptr(), T, N, P, X.data_ptr(), _stream())
    return X


def rouse_correlation(X, max_lag: int):
    """c[p-1, lag] = <X_p(t0+lag).X_p(t0)> and <X_p^2> = c[:, 0] (numpy)."""
    import torch

    X = _check_traj(X)
    T, P, _ = X.shape
    c = torch.empty((P, max_lag + 1), dtype=torch.float64, device=X.device)
    lb.lb_analysis_rouse_correlation(X.data_ptr(), T, P, max_lag, c.data_ptr(), _stream())
    c = c.cpu().numpy()
    return c, c[:, 0].copy()


def static_sk(traj, ks):
    """S(k) for the wave numbers ks (numpy)."""
    import torch

    traj = _check_traj(traj)
    T, N, _ = traj.shape
    k = torch.as_tensor(np.asarray(ks, dtype=np.float64), device=traj.device)
    S = torch.empty(k.numel(), dtype=torch.float64, device=traj.device)
    lb.lb_analysis_static_sk(traj.data_ptr(), T, N, k.data_ptr(), k.numel(), S.data_ptr(), _stream())
    return S.cpu().numpy()


def dynamic_sk(traj, ks, max_lag: int, origin_stride: int = 1):
    """S(k, lag) for the wave numbers ks and lags 0..max_lag (numpy, (nk, max_lag+1))."""
    import torch

    traj = _check_traj(traj)
    T, N, _ = traj.shape
    k = torch.as_tensor(np.asarray(ks, dtype=np.float64), device=traj.device)
    S = torch.empty((k.numel(), max_lag + 1), dtype=torch.float64, device=traj.device)
    lb.lb_analysis_dynamic_sk(traj.data_ptr(), T, N, k.data_ptr(), k.numel(), max_lag, origin_stride, S.data_ptr(),
                              _stream())
    return S.cpu().numpy()


def inverse_radius(traj) -> float:
    """<1/R_H> = (1/N^2) sum_{i != j} <1/r_ij> over the frames."""
    import torch

    traj = _check_traj(traj)
    T, N, _ = traj.shape
    out = torch.empty(1, dtype=torch.float64, device=traj.device)
    lb.lb_analysis_inverse_radius(traj.data_ptr(), T, N, out.data_ptr(), _stream())
    return float(out.item())
