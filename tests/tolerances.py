"""Tolerances shared by several GPU parity test files (see the docstring of
tests/test_gpu_parity.py for their derivation)."""
import numpy as np

# FP32 operator, row by row: |dy_i| <= MF32_ROW_C * 2^-24 * (|K| (|u| + ||u||_inf))_i
MF32_ROW_C = 64.0


def mf32_row_bound(ref_row, u_cols, u_inf):
    """The row-wise bound of the FP32 tiled operator for one row of K
    (ref_row, on the columns u_cols) and an FP32 input of max norm u_inf."""
    return MF32_ROW_C * 2.0 ** -24 * (np.abs(ref_row) @ (np.abs(u_cols) + u_inf))
