"""Pin of the oracle's Kalman log-likelihood: for small T it must equal the
log-density of the joint Gaussian of y_{1:T} written out from the model
(x_0 ~ N(m0, p0), x_t = a x_{t-1} + N(0,q), y_t = x_t + N(0,r))."""
import numpy as np
import pytest

import oracle


def joint_gaussian_loglik(a, q, r, y, m0, p0):
    T, D = y.shape
    var = np.zeros(T + 1)
    var[0] = p0
    for t in range(1, T + 1):
        var[t] = a * a * var[t - 1] + q
    C = np.zeros((T, T))
    for s in range(1, T + 1):
        for t in range(s, T + 1):
            C[s - 1, t - 1] = C[t - 1, s - 1] = a ** (t - s) * var[s]
    C += r * np.eye(T)
    mean = np.array([a ** t * m0 for t in range(1, T + 1)])
    sign, logdet = np.linalg.slogdet(C)
    assert sign > 0
    ll = 0.0
    Ci = np.linalg.inv(C)
    for d in range(D):
        e = y[:, d] - mean
        ll += -0.5 * (T * np.log(2 * np.pi) + logdet + e @ Ci @ e)
    return ll


@pytest.mark.parametrize("a,q,r,m0,p0", [(0.9, 0.1, 0.5, 0.0, 1.0), (0.8, 0.3, 0.2, 1.5, 0.7), (-0.5, 1.0, 1.0, 0.0, 2.0)])
def test_kalman_matches_joint_gaussian(a, q, r, m0, p0):
    rng = np.random.default_rng(3)
    y = rng.standard_normal((9, 4))
    assert oracle.kalman_loglik(a, q, r, y, m0, p0) == pytest.approx(joint_gaussian_loglik(a, q, r, y, m0, p0),
                                                                     rel=1e-10, abs=1e-9)
