"""Pins for the FP64 oracle GEMM (CPU only).

Each check compares the oracle with something other than itself: closed
forms, exact integer arithmetic, exact rational arithmetic, a hand-computed
worked example, and the standard rounding-error bound.  Together they fail on
a dropped term, a wrong sign, a wrong index or a transposed operand.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return rows


def test_hand_computed_2x3x4():
    r = _read_golden("gemm_2x3x4.txt")
    A = np.array(r[0:2]); B = np.array(r[2:5]); alpha, beta = r[5]
    C0 = np.array(r[6:8]); expect = np.array(r[8:10])
    got = oracle.gemm(A, B, alpha=alpha, beta=beta, C0=C0)
    assert np.array_equal(got, expect)


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (3, 5, 7), (64, 33, 17), (130, 70, 257)])
def test_all_ones_every_entry_is_k(m, n, k):
    C = oracle.gemm(np.ones((m, k)), np.ones((k, n)))
    assert C.shape == (m, n)
    assert np.all(C == k)


@pytest.mark.parametrize("m,n", [(5, 9), (64, 64), (33, 130)])
def test_identity_is_exact(m, n):
    A = W.uniform(m, n, seed=11)
    assert np.array_equal(oracle.gemm(A, np.eye(n)), A.astype(np.float64))
    assert np.array_equal(oracle.gemm(np.eye(m), A), A.astype(np.float64))


def test_permutation_is_exact():
    m, k, n = 17, 23, 19
    A = W.uniform(m, k, seed=12)
    B = W.uniform(k, n, seed=13)
    g = W.rng(14)
    pr = g.permutation(m); pc = g.permutation(n)
    P_rows = np.eye(m)[pr]              # (P A)[i] = A[pr[i]]
    P_cols = np.eye(n)[:, pc]           # (B P)[:, j] = B[:, pc[j]]
    assert np.array_equal(oracle.gemm(P_rows, A), A[pr].astype(np.float64))
    assert np.array_equal(oracle.gemm(B, P_cols), B[:, pc].astype(np.float64))


@pytest.mark.parametrize("m,n,k", [(7, 5, 3), (40, 24, 130), (33, 65, 4096)])
def test_integer_matrices_exact(m, n, k):
    A = W.integer_matrix(m, k, seed=21)
    B = W.integer_matrix(k, n, seed=22)
    exact = A.astype(np.int64) @ B.astype(np.int64)       # exact integer product
    assert np.array_equal(oracle.gemm(A, B), exact.astype(np.float64))


def test_alpha_beta_exact_on_integers():
    m, n, k = 9, 11, 13
    A = W.integer_matrix(m, k, seed=31)
    B = W.integer_matrix(k, n, seed=32)
    C0 = W.integer_matrix(m, n, seed=33)
    exact = 3 * (A.astype(np.int64) @ B.astype(np.int64)) - 2 * C0.astype(np.int64)
    got = oracle.gemm(A, B, alpha=3.0, beta=-2.0, C0=C0)
    assert np.array_equal(got, exact.astype(np.float64))


def test_beta_zero_does_not_read_c0():
    A = np.ones((2, 2)); B = np.ones((2, 2))
    C0 = np.full((2, 2), np.nan)
    got = oracle.gemm(A, B, alpha=1.0, beta=0.0, C0=C0)
    assert np.all(got == 2.0)


def test_non_square_orientation():
    # A (2x3) with distinct entries against B (3x2): a transposed operand or a
    # swapped index would give a different (or ill-shaped) result.
    A = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]])
    B = np.array([[7.0, 8.0], [9.0, 10.0], [11.0, 12.0]])
    assert np.array_equal(oracle.gemm(A, B), np.array([[58.0, 64.0], [139.0, 154.0]]))


def test_brute_force_rational_within_rounding_bound():
    # Exact rational sums on small random float inputs; the fp64 result must
    # lie within the classical bound |fl(s) - s| <= gamma_k * sum|a||b|,
    # gamma_k = k u / (1 - k u), u = 2^-53 (Higham, Accuracy and Stability of
    # Numerical Algorithms, Sec. 3.1).
    m, n, k = 4, 5, 6
    A = W.uniform(m, k, seed=41); B = W.uniform(k, n, seed=42)
    got = oracle.gemm(A, B)
    u = 2.0 ** -53
    gamma = k * u / (1 - k * u)
    for i in range(m):
        for j in range(n):
            s = sum(Fraction(float(A[i, p])) * Fraction(float(B[p, j])) for p in range(k))
            mag = sum(abs(float(A[i, p]) * float(B[p, j])) for p in range(k))
            assert abs(Fraction(got[i, j]) - s) <= Fraction(gamma * mag)


def test_rows_match_full_and_closed_form():
    m, n, k = 50, 40, 30
    A = W.uniform(m, k, seed=51); B = W.uniform(k, n, seed=52)
    C0 = W.uniform(m, n, seed=53)
    full = oracle.gemm(A, B, alpha=1.5, beta=0.5, C0=C0)
    rows = W.sample_rows(m, 7, seed=54)
    part = oracle.gemm_rows(A, B, rows, alpha=1.5, beta=0.5, C0=C0)
    assert np.array_equal(part, full[rows])
    ones = oracle.gemm_rows(np.ones((m, k)), np.ones((k, n)), rows)
    assert np.all(ones == k)


def test_empty_shapes():
    assert oracle.gemm(np.zeros((0, 3)), np.zeros((3, 4))).shape == (0, 4)
    assert np.all(oracle.gemm(np.zeros((2, 0)), np.zeros((0, 3))) == 0)


def test_shape_mismatch_raises():
    with pytest.raises(ValueError):
        oracle.gemm(np.ones((2, 3)), np.ones((4, 2)))


def test_threads_reported():
    assert oracle.num_threads() >= 1
