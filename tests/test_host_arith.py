"""Integer arithmetic the sweep kernels rely on, checked on the CPU.

The blocked forward finds the run of an entry (or pair) f of a row as
floor(f / q) for a divisor q fixed per row, by one high multiply with
m = ceil(2^32 / q) (Granlund & Montgomery, division by invariant integers).
The floor is exact while f (q - 1) < 2^32; rows hold far fewer entries.
"""
import numpy as np


def _div_high(f: np.ndarray, q: int) -> np.ndarray:
    m = (0xFFFFFFFF // q) + 1
    return (f.astype(np.uint64) * np.uint64(m)) >> np.uint64(32)


def test_high_multiply_division_exact_in_range():
    f = np.arange(1 << 21, dtype=np.uint64)
    for q in range(2, 65):
        assert np.array_equal(_div_high(f, q), f // np.uint64(q)), q
    # the largest numerators of the stated bound
    for q in (3, 9, 17, 31, 64):
        hi = (1 << 32) // (q - 1) - 1
        f = np.arange(max(hi - 4096, 0), hi + 1, dtype=np.uint64)
        assert np.array_equal(_div_high(f, q), f // np.uint64(q)), q
