"""Pins for the oracle's query-guided instance labels (Sec. 3.3): the whole
chain recomputed with scipy's logistic function, multivariate normal density
and softmax; rows are distributions; query order only permutes columns; the
closed cases of a Gaussian at a query centre with an orthogonal feature and
of Gaussians far from every query."""
import numpy as np
import pytest
from scipy import special, stats

import oracle as O
from paper_2604_10951_gb300 import scenes


def _inputs(n=60, nq=16, dim=32, seed=0):
    sc = scenes.room_scene(n=4000, C=4, seed=seed)
    f_ins, f_q, p_q, prec = scenes.room_queries(sc.means, nq, dim, seed)
    idx = np.random.default_rng(seed).choice(sc.n, n, replace=False)
    return f_ins[idx].astype(np.float64), sc.means[idx].astype(np.float64), f_q.astype(np.float64), \
        p_q.astype(np.float64), prec.astype(np.float64)


def _cov(prec_row):
    xx, yy, zz, xy, xz, yz = prec_row
    return np.linalg.inv(np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]))


def test_labels_match_scipy_density_logistic_and_softmax():
    f_ins, means, f_q, p_q, prec = _inputs()
    got = O.query_labels(f_ins, means, f_q, p_q, prec)
    S = special.expit(f_ins @ f_q.T)
    D = np.empty_like(S)
    for q in range(f_q.shape[0]):
        mvn = stats.multivariate_normal(mean=p_q[q], cov=_cov(prec[q]))
        D[:, q] = mvn.pdf(means) / mvn.pdf(p_q[q])
    want = special.softmax(S * D, axis=1)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-15)
    assert D.max() > 0.5 and D.min() < 0.05  # the proximity term varies over the inputs


def test_rows_are_distributions_and_query_order_permutes_columns():
    f_ins, means, f_q, p_q, prec = _inputs(n=200, nq=32, seed=1)
    l = O.query_labels(f_ins, means, f_q, p_q, prec)
    np.testing.assert_allclose(l.sum(1), 1.0, atol=1e-14)
    assert (l > 0).all()
    perm = np.random.default_rng(2).permutation(f_q.shape[0])
    lp = O.query_labels(f_ins, means, f_q[perm], p_q[perm], prec[perm])
    np.testing.assert_allclose(lp, l[:, perm], rtol=1e-14)  # the softmax sum in another order


def test_closed_cases():
    dim, nq = 16, 4
    rng = np.random.default_rng(3)
    f_q = rng.normal(size=(nq, dim))
    p_q = rng.uniform(-1, 1, (nq, 3))
    prec = np.tile([4.0, 2.0, 1.0, 0.0, 0.0, 0.0], (nq, 1))
    # a Gaussian at query 0's centre with a feature orthogonal to every query
    # feature: S = 1/2 for all queries, D = 1 for query 0
    f = rng.normal(size=dim)
    Q, _ = np.linalg.qr(f_q.T)
    f -= Q @ (Q.T @ f)
    l = O.query_labels(f[None], p_q[:1], f_q, p_q, prec)[0]
    d = p_q[0] - p_q
    quad = 4 * d[:, 0] ** 2 + 2 * d[:, 1] ** 2 + d[:, 2] ** 2
    A = 0.5 * np.exp(-0.5 * quad)
    np.testing.assert_allclose(l, np.exp(A) / np.exp(A).sum(), rtol=1e-12)
    assert np.argmax(l) == 0
    # far from every query: D underflows to 0, so the labels are uniform
    far = O.query_labels(rng.normal(size=(3, dim)), np.full((3, 3), 1e3), f_q, p_q, prec)
    np.testing.assert_allclose(far, 1.0 / nq, rtol=1e-15)
