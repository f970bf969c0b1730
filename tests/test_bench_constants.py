"""The per-matrix figures bench.py divides by are re-derived here (CPU):
algorithmic FP64 operations from the oracle's counting scalar on the mixed
workload recipe, and algorithmic bytes from the record layouts."""

import numpy as np

import bench
import oracle
from paper_1806_06698_gb300 import inputs


def test_flops_per_matrix_matches_the_oracle_count():
    A, _ = inputs.mixed(1 << 15, seed=inputs.SEED_BASE + 1)
    ops = oracle.count_ops(A).astype(np.float64)
    mean = ops.sum(axis=1).mean()
    assert abs(mean - bench.FLOPS_PER_MATRIX_F64) <= 0.03 * bench.FLOPS_PER_MATRIX_F64, mean


def test_bytes_per_matrix():
    # packed input (6) + eigenvalues (3) + eigenvectors (9), 8 bytes each
    assert bench.BYTES_PER_MATRIX_F64 == (6 + 3 + 9) * 8
