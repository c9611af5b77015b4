"""Shared helpers for the GPU parity tests: device upload with optional x padding and
the tolerance measures the parity bar is stated in."""
import numpy as np
import torch

# FP64 parity bar: max-norm error relative to the reference's max norm.
TOL_F64 = 1e-12


def to_dev(a: np.ndarray, pad: int = 0, dtype=torch.float64) -> torch.Tensor:
    """Uploads a vertex array; pad > 0 gives each x-row `pad` extra elements (pitch)."""
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dtype)
    if pad:
        shape = list(t.shape)
        buf = torch.full(shape[:-1] + [shape[-1] + pad], float("nan"), dtype=dtype)
        buf[..., :shape[-1]] = t
        return buf.cuda()[..., :shape[-1]]
    return t.cuda()


def to_host(t: torch.Tensor) -> np.ndarray:
    return t.detach().to(torch.float64).cpu().numpy()


def rel_err(got, ref) -> float:
    d = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(got - ref))) / (d if d > 0 else 1.0)


def apply_err(got, ref, u, h) -> float:
    """Apply/residual error: max-norm difference over max(|y_ref|_inf, |A|_inf |u|_inf
    * 1e-3), |A|_inf = (16/3)/h^2, guarding against cancellation on smooth inputs."""
    denom = max(float(np.max(np.abs(ref))), (16.0 / 3.0) / h ** 2 * float(np.max(np.abs(u))) * 1e-3)
    return float(np.max(np.abs(got - ref))) / (denom if denom > 0 else 1.0)
