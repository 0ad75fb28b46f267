"""Shared helpers for the tests: numpy <-> torch device buffers."""
import numpy as np


def to_dev(x: np.ndarray, word_bytes: int):
    import torch
    dt = np.uint32 if word_bytes == 4 else np.uint64
    return torch.from_numpy(np.ascontiguousarray(x.astype(dt))).cuda()


def from_dev(t) -> np.ndarray:
    return t.cpu().numpy().astype(np.uint64)


def empty_dev(n: int, word_bytes: int):
    import torch
    return torch.empty(n, dtype=torch.uint32 if word_bytes == 4 else torch.uint64, device="cuda")


def bitrev(i: int, k: int) -> int:
    return int(format(i, f"0{k}b")[::-1], 2) if k else 0
