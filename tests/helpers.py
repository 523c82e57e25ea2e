"""Shared helpers of the GPU tests: moving tuples between numpy and CUDA, reading
library views, and multiset comparisons for orders the method leaves open."""
import numpy as np

U64 = (1 << 64) - 1


def to_dev(a: np.ndarray):
    import torch

    a = np.ascontiguousarray(a, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64)).to("cuda")


def from_dev_ptr(ptr: int, n: int, width: int = 2, dtype=np.uint64) -> np.ndarray:
    """Copy n rows of `width` 64-bit (or 32-bit) values from a device pointer."""
    import torch

    if n == 0:
        return np.zeros((0, width), dtype=dtype) if width > 1 else np.zeros(0, dtype=dtype)
    itemsize = np.dtype(dtype).itemsize
    nbytes = n * width * itemsize
    host = torch.empty(nbytes, dtype=torch.uint8)
    dev = torch.cuda.current_device()
    t = _wrap(ptr, nbytes, dev)
    host.copy_(t)
    arr = host.numpy().view(dtype)
    return arr.reshape(n, width) if width > 1 else arr


def _wrap(ptr: int, nbytes: int, dev: int):
    """A uint8 CUDA tensor aliasing [ptr, ptr+nbytes) (read only use)."""
    import torch

    class _CAI:
        def __init__(self):
            self.__cuda_array_interface__ = {
                "shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3, "strides": None,
            }

    return torch.as_tensor(_CAI(), device=f"cuda:{dev}")


def sort_tuples(a: np.ndarray) -> np.ndarray:
    """Rows sorted by (col0, col1): a canonical form of a multiset of pairs."""
    if len(a) == 0:
        return a
    order = np.lexsort((a[:, 1], a[:, 0]))
    return a[order]


def same_multiset(a: np.ndarray, b: np.ndarray) -> bool:
    return a.shape == b.shape and bool((sort_tuples(a) == sort_tuples(b)).all())


def random_tuples(rng, n, domain, extremes=False):
    keys = rng.integers(0, domain, n, dtype=np.uint64) if domain < (1 << 63) else rng.integers(
        0, U64, n, dtype=np.uint64, endpoint=True)
    if extremes and n:
        idx = rng.integers(0, n, max(1, n // 50))
        keys[idx] = rng.choice(np.array([0, U64, U64 - 1, 1], dtype=np.uint64), len(idx))
    pay = rng.integers(0, U64, n, dtype=np.uint64, endpoint=True)
    return np.stack([keys, pay], axis=1)
