"""Pins of the oracle's block-DROP step (P_T of Appendix C; DROP of ref. CEHN08, Sec. III-D).

Reading used: x_j += lambda/s_j * sum_{i in block} a_ij (b_i - <a_i,x>)/||a_i||^2,
s_j = number of rows of the block with a_ij != 0.  Pins: exact projection for one-row
blocks, the one-row closed form, fixed points, convergence to numpy's least-squares
solution on a consistent system, a hand-computed block (tests/golden), degenerate rows.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _csr_from_dense(A):
    rows, cols, vals = [], [], []
    rp = [0]
    for i in range(A.shape[0]):
        nz = np.nonzero(A[i])[0]
        cols.extend(nz.tolist()); vals.extend(A[i, nz].tolist())
        rp.append(len(cols))
    return np.array(rp, np.int64), np.array(cols, np.int32), np.array(vals, np.float64)


def _random_sparse(M, V, per_row, rng):
    A = np.zeros((M, V))
    for i in range(M):
        idx = rng.choice(V, size=per_row, replace=False)
        A[i, idx] = rng.uniform(0.1, 1.5, size=per_row)
    return A


def test_one_row_block_is_exact_hyperplane_projection():
    rng = np.random.default_rng(0)
    V = 36
    A = _random_sparse(1, V, 9, rng)
    rp, c, v = _csr_from_dense(A)
    b = np.array([3.7])
    x0 = rng.normal(size=V)
    x1, ss = oracle.drop_block(rp, c, v, b, 0, 1, x0, 1.0)
    assert A[0] @ x1 == pytest.approx(3.7, rel=1e-13)
    d = x1 - x0   # parallel to a_i
    assert np.allclose(d, (d @ A[0]) / (A[0] @ A[0]) * A[0], atol=1e-14)
    # projection is the nearest point of the hyperplane: equals the textbook formula
    proj = x0 + (3.7 - A[0] @ x0) / (A[0] @ A[0]) * A[0]
    np.testing.assert_allclose(x1, proj, rtol=1e-13, atol=1e-14)
    assert ss == pytest.approx((3.7 - A[0] @ x0) ** 2, rel=1e-13)


@pytest.mark.parametrize("lam", [0.3, 1.0, 1.9])
def test_one_row_closed_form(lam):
    rng = np.random.default_rng(1)
    V = 20
    A = _random_sparse(1, V, 5, rng)
    rp, c, v = _csr_from_dense(A)
    b = np.array([-1.25])
    x0 = rng.normal(size=V)
    x1, _ = oracle.drop_block(rp, c, v, b, 0, 1, x0, lam)
    r = (b[0] - A[0] @ x0) / (A[0] @ A[0])
    np.testing.assert_allclose(x1, x0 + lam * r * A[0], rtol=1e-13, atol=1e-14)
    # relaxed projection moves the residual by the factor (1 - lam)
    assert b[0] - A[0] @ x1 == pytest.approx((1 - lam) * (b[0] - A[0] @ x0), rel=1e-10, abs=1e-12)


def test_hand_computed_block():
    g = json.load(open(os.path.join(GOLD, "drop_3voxel_4row.json")))
    V = g["V"]
    A = np.zeros((len(g["rows"]), V))
    for i, row in enumerate(g["rows"]):
        for j, a in row:
            A[i, j] = a
    rp, c, v = _csr_from_dense(A)
    b = np.array(g["b"])
    for case in g["cases"]:
        x1, ss = oracle.drop_sweep(rp, c, v, b, case["block_ptr"], case["x0"], case["lambda"])
        np.testing.assert_allclose(x1, case["x1"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(ss, case["resid_ss"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_solution_is_fixed_point(lam):
    rng = np.random.default_rng(2)
    V, M = 30, 50
    A = _random_sparse(M, V, 6, rng)
    rp, c, v = _csr_from_dense(A)
    xs = rng.uniform(0, 2, size=V)
    b = A @ xs
    x1, ss = oracle.drop_sweep(rp, c, v, b, [0, 13, 37, 50], xs, lam)
    np.testing.assert_allclose(x1, xs, rtol=1e-13, atol=1e-14)
    assert np.all(ss < 1e-24)


@pytest.mark.parametrize("B", [1, 4, 60])
def test_consistent_system_converges_to_least_squares(B):
    rng = np.random.default_rng(3)
    V, M = 36, 60            # 6x6x1 image, full column rank
    A = _random_sparse(M, V, 10, rng)
    assert np.linalg.matrix_rank(A) == V
    rp, c, v = _csr_from_dense(A)
    xs = rng.uniform(0, 2, size=V)
    b = A @ xs
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    bp = np.minimum(np.arange(B + 1) * -(-M // B), M)
    x = np.zeros(V)
    # fully simultaneous blocks (B=1) converge more slowly than sequential ones
    for it in range(100000):
        x_new, ss = oracle.drop_sweep(rp, c, v, b, bp, x, 1.0)
        done = np.max(np.abs(x_new - x)) < 1e-13
        x = x_new
        if done:
            break
    np.testing.assert_allclose(x, x_ls, rtol=0, atol=1e-8)
    assert np.linalg.norm(A @ x - b) < 1e-7 * np.linalg.norm(b)


def test_degenerate_rows_and_voxels():
    # a zero-norm row contributes nothing; voxels hit by no row keep their value;
    # an empty block is the identity
    A = np.array([[1.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0], [0.0, 2.0, 0.0, 0.0]])
    rp, c, v = _csr_from_dense(A)
    b = np.array([1.0, 5.0, 4.0])
    x0 = np.array([0.0, 0.0, 7.0, -3.0])
    x1, ss = oracle.drop_block(rp, c, v, b, 0, 3, x0, 1.0)
    np.testing.assert_allclose(x1, [1.0, 2.0, 7.0, -3.0], atol=1e-15)
    assert ss == pytest.approx(1 + 25 + 16)
    x2, ss2 = oracle.drop_block(rp, c, v, b, 1, 1, x0, 1.0)
    np.testing.assert_array_equal(x2, x0)
    assert ss2 == 0.0
    # explicit zeros stored in a row do not count towards s_j
    rp2 = np.array([0, 2, 3], np.int64)
    c2 = np.array([0, 1, 1], np.int32)
    v2 = np.array([1.0, 0.0, 1.0])
    x3, _ = oracle.drop_block(rp2, c2, v2, np.array([1.0, 1.0]), 0, 2, np.zeros(2), 1.0)
    np.testing.assert_allclose(x3, [1.0, 1.0], atol=1e-15)


def test_block_at_matches_full_block():
    rng = np.random.default_rng(4)
    V, M = 64, 200
    A = _random_sparse(M, V, 7, rng)
    rp, c, v = _csr_from_dense(A)
    b = rng.uniform(1, 3, size=M)
    x0 = rng.uniform(0, 1, size=V)
    for r0, r1 in [(0, 200), (37, 91), (5, 6)]:
        full, _ = oracle.drop_block(rp, c, v, b, r0, r1, x0, 0.7)
        vox = rng.choice(V, size=17, replace=False)
        at = oracle.drop_block_at(rp, c, v, b, r0, r1, x0, 0.7, vox)
        np.testing.assert_array_equal(at, full[vox])


def test_blocks_are_sequential_rows_inside_are_simultaneous():
    # two identical rows in one block act like one row (s_j = 2, averaged), but in
    # two blocks the second sees the first's result (a plain sequential projection)
    A = np.array([[1.0, 1.0], [1.0, 1.0]])
    rp, c, v = _csr_from_dense(A)
    b = np.array([2.0, 2.0])
    x_one, _ = oracle.drop_sweep(rp, c, v, b, [0, 2], [0.0, 0.0], 1.0)
    np.testing.assert_allclose(x_one, [1.0, 1.0], atol=1e-15)
    x_two, _ = oracle.drop_sweep(rp, c, v, b, [0, 1, 2], [0.0, 0.0], 0.5)
    # block 0: r = 2/2 = 1, x = 0.5*(1,1) = (0.5,0.5); block 1: r = (2-1)/2, x += 0.5*0.5
    np.testing.assert_allclose(x_two, [0.75, 0.75], atol=1e-15)
