"""Oracle: storage rounding of H and S values.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Mixed-precision forms store H and S in FP32 or BF16. Their results are compared
with the oracle run on the same stored values, so the oracle needs the same
rounding, written here from its definition:

* FP32: round-to-nearest-even of the FP64 value (IEEE 754 conversion);
* BF16: round-to-nearest-even of the FP64 value to FP32, then
  round-to-nearest-even of that FP32 value to its upper 16 bits
  (1 sign, 8 exponent, 7 mantissa bits). Values here are finite and far from
  the overflow range.
"""
from __future__ import annotations

import numpy as np


def round_fp32(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_bf16(x: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_storage(x: np.ndarray, storage: str) -> np.ndarray:
    if storage == "fp64":
        return np.asarray(x, dtype=np.float64)
    if storage == "fp32":
        return round_fp32(x)
    if storage == "bf16":
        return round_bf16(x)
    raise ValueError(storage)
