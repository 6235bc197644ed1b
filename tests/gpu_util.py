"""Helpers shared by the GPU tests: move oracle/generator arrays to column-major CUDA tensors."""
import numpy as np
import torch


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.float64)


def rhs_dev(rhs):
    return to_dev(rhs.U), to_dev(rhs.s), to_dev(rhs.V)
