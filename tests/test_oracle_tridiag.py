"""Pins of the oracle's tridiagonal solvers and of its PDD / PPT algebra (Sec. 3.2)."""
import os

import numpy as np
import pytest

from oracle import ns_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "partition_n12_p4.txt")


def _rand_dd(rng, n, margin=1.0):
    a = rng.uniform(-1, 1, n)
    c = rng.uniform(-1, 1, n)
    b = (np.abs(a) + np.abs(c) + margin) * rng.choice([-1, 1], n)
    return a, b, c


def test_thomas_closed_form():
    # [2 -1 0; -1 2 -1; 0 -1 2] x = [1 0 1]  ->  x = [1 1 1]
    x = O.thomas(np.array([0, -1, -1.0]), np.array([2, 2, 2.0]), np.array([-1, -1, 0.0]),
                 np.array([1.0, 0.0, 1.0]))
    np.testing.assert_allclose(x, [1, 1, 1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64])
def test_thomas_vs_dense_lu(n):
    rng = np.random.default_rng(n)
    a, b, c = _rand_dd(rng, n)
    d = rng.standard_normal((4, n))
    x = O.thomas(a, b, c, d)
    A = O.tridiag_dense(a, b, c)
    ref = np.linalg.solve(A, d.T).T          # LAPACK LU with partial pivoting
    np.testing.assert_allclose(x, ref, rtol=1e-13, atol=1e-13)
    assert np.abs(A @ x.T - d.T).max() <= 1e-14 * np.abs(d).max() * 10


@pytest.mark.parametrize("n", [3, 4, 8, 33])
def test_cyclic_vs_dense_lu(n):
    rng = np.random.default_rng(100 + n)
    a, b, c = _rand_dd(rng, n)
    d = rng.standard_normal((3, n))
    x = O.thomas_cyclic(a, b, c, d)
    A = O.tridiag_dense(a, b, c, cyclic=True)
    ref = np.linalg.solve(A, d.T).T
    np.testing.assert_allclose(x, ref, rtol=1e-12, atol=1e-13)


def test_complex_rhs():
    rng = np.random.default_rng(5)
    a, b, c = _rand_dd(rng, 9)
    d = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    x = O.thomas(a, b, c, d)
    np.testing.assert_allclose(O.tridiag_dense(a, b, c) @ x, d, atol=1e-13)


def _load_golden():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _example():
    rng = np.random.default_rng(12)
    n = 12
    a = rng.uniform(0.2, 0.9, n)
    c = rng.uniform(0.2, 0.9, n)
    b = a + c + rng.uniform(0.5, 1.5, n)
    return a, b, c


def test_partition_matches_printed_example():
    """The oracle's A~, V, E, Y, Z, P, Z-bar reproduce the n=12, p=4 matrices of Sec. 3.2."""
    a, b, c = _example()
    n, p, m = 12, 4, 3
    A, At, V, E = O.partition_matrices(a, b, c, p)
    g = _load_golden()
    sym = {"one": 1.0}
    for j in range(n):
        sym["a%d" % (j + 1)] = a[j]
        sym["c%d" % (j + 1)] = c[j]
    Y = np.linalg.solve(At, V)
    # spikes by partition, from the Y column layout
    for r in g:
        if r[0] == "Y":
            col, r0, r1, kind, part = int(r[1]), int(r[2]), int(r[3]), r[4], int(r[5])
            spike = Y[r0 - 1:r1, col - 1]
            sym["%s1%d" % (kind, part)] = spike[0]
            sym["%sm%d" % (kind, part)] = spike[-1]
            rest = np.delete(Y[:, col - 1], np.arange(r0 - 1, r1))
            assert np.all(rest == 0.0), "spike leaks outside partition"
    DA = A - At
    exp = np.zeros((n, n))
    for r in g:
        if r[0] == "DA":
            exp[int(r[1]) - 1, int(r[2]) - 1] = sym[r[3]]
    np.testing.assert_array_equal(DA, exp)
    expV = np.zeros_like(V)
    for r in g:
        if r[0] == "V":
            expV[int(r[1]) - 1, int(r[2]) - 1] = sym[r[3]]
    np.testing.assert_array_equal(V, expV)
    expE = np.zeros((2 * (p - 1), n))
    for r in g:
        if r[0] == "ET":
            expE[int(r[1]) - 1, int(r[2]) - 1] = 1.0
    np.testing.assert_array_equal(E.T, expE)
    Z = np.eye(2 * (p - 1)) + E.T @ Y
    expZ = np.zeros_like(Z)
    for r in g:
        if r[0] == "Z":
            expZ[int(r[1]) - 1, int(r[2]) - 1] = sym[r[3]]
    np.testing.assert_allclose(Z, expZ, rtol=0, atol=1e-15)
    P = O.swap_permutation(2 * (p - 1))
    expP = np.zeros_like(P)
    for r in g:
        if r[0] == "P":
            expP[int(r[1]) - 1, int(r[2]) - 1] = 1.0
    np.testing.assert_array_equal(P, expP)
    np.testing.assert_array_equal(P @ P, np.eye(2 * (p - 1)))
    Zb = P + E.T @ Y @ P
    expZb = np.zeros_like(Zb)
    for r in g:
        if r[0] == "ZB":
            expZb[int(r[1]) - 1, int(r[2]) - 1] = sym[r[3]]
    np.testing.assert_allclose(Zb, expZb, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n,p,cyclic", [(12, 4, False), (12, 4, True), (64, 8, False),
                                        (64, 8, True), (30, 5, False), (16, 1, True)])
def test_ppt_is_exact(n, p, cyclic):
    """PPT makes no approximation (Sec. 3.2): equals dense LU on a general system."""
    rng = np.random.default_rng(n * 7 + p)
    a, b, c = _rand_dd(rng, n, margin=0.05)
    d = rng.standard_normal(n)
    ref = np.linalg.solve(O.tridiag_dense(a, b, c, cyclic), d)
    x = O.ppt_solve(a, b, c, d, p, cyclic)
    np.testing.assert_allclose(x, ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("cyclic", [False, True])
def test_pdd_machine_accuracy_on_adi_rows(cyclic):
    """|b| = |a| + |c| + 1 (ADI rows, Sec. 3.2): PDD matches the exact solution
    to machine accuracy once partitions are a few rows long."""
    n, p = 256, 32
    for r in (1e-3, 1e-1, 1.0):
        a = np.full(n, -r)
        c = np.full(n, -r)
        b = 1.0 + 2.0 * r + np.zeros(n)
        assert np.allclose(np.abs(b), np.abs(a) + np.abs(c) + 1.0)
        d = np.random.default_rng(3).standard_normal(n)
        ref = np.linalg.solve(O.tridiag_dense(a, b, c, cyclic), d)
        x = O.pdd_solve(a, b, c, d, p, cyclic)
        drop = O.pdd_dropped_coupling(a, b, c, p, cyclic)
        err = np.abs(x - ref).max() / np.abs(ref).max()
        assert err <= max(4 * drop, 1e-15) * 50, (r, err, drop)
        if drop < 1e-17:          # dropped coupling below round-off
            assert err < 1e-14


def test_pdd_inaccurate_on_weakly_dominant_poisson_rows():
    """|b| = |a| + |c| + eps with eps ~ 1e-8 (low Poisson modes, Sec. 3.2): PDD
    visibly wrong, PPT exact."""
    n, p = 64, 4
    a = np.full(n, 1.0)
    c = np.full(n, 1.0)
    b = -(a + c) - 1e-8
    d = np.random.default_rng(4).standard_normal(n)
    d -= d.mean()
    ref = np.linalg.solve(O.tridiag_dense(a, b, c), d)
    xpdd = O.pdd_solve(a, b, c, d, p)
    xppt = O.ppt_solve(a, b, c, d, p)
    scale = np.abs(ref).max()
    assert np.abs(xpdd - ref).max() / scale > 1e-3
    assert np.abs(xppt - ref).max() / scale < 1e-6   # limited by cond(A) ~ 1e8


def test_pdd_dropped_coupling_decay_closed_form():
    """For constant rows (-r, 1+2r, -r) the dropped coupling decays like lam^m with
    lam = ((1+2r) - sqrt(1+4r)) / (2r), the smaller root of r t^2 - (1+2r) t + r = 0."""
    r = 0.5
    lam = ((1 + 2 * r) - np.sqrt(1 + 4 * r)) / (2 * r)
    drops = []
    for m in (4, 6, 8):
        n = 4 * m
        a = np.full(n, -r)
        c = np.full(n, -r)
        b = np.full(n, 1 + 2 * r)
        drops.append(O.pdd_dropped_coupling(a, b, c, 4))
    np.testing.assert_allclose(drops[1] / drops[0], lam ** 2, rtol=1e-3)
    np.testing.assert_allclose(drops[2] / drops[1], lam ** 2, rtol=1e-3)
