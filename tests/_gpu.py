"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
fetch results as numpy arrays."""
import numpy as np
import torch

from paper_1903_00227_gb300 import wrs


def to_device(w: np.ndarray) -> torch.Tensor:
    if w.dtype == np.uint32:
        return torch.from_numpy(w.view(np.int32).copy()).cuda()
    return torch.from_numpy(np.ascontiguousarray(w)).cuda()


def gpu_build(w: np.ndarray, table: "wrs.AliasTable | None" = None):
    t = table or wrs.AliasTable(len(w))
    t.build(to_device(w))
    return t


def gpu_samples(t, k: int, seed: int, stream_id: int = 0) -> np.ndarray:
    out = t.sample(k, seed, stream_id)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)
