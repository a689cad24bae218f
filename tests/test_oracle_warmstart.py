"""Pins of the warm-start oracle (oracle/warmstart.py) to facts outside itself: a normal-table
value of Phi, finite differences (brute force) for every gradient entry, the closed form of
Adam's first step, and the identity R Z = D - HA W of the exact solve of S Z = D
(Eq. matvec_decomp with W = HA^T Z/(N-1))."""
import math

import numpy as np
import pytest

import oracle
from oracle import warmstart as ws


def test_gelu_values():
    # x Phi(x) with Phi(1.959964) = 0.975 (standard normal table) and Phi(0) = 1/2
    x = 1.959963984540054
    assert abs(ws.gelu(np.array(x)) / x - 0.975) < 1e-12
    assert ws.gelu(np.array(0.0)) == 0.0
    xs = np.linspace(-6, 6, 101)
    assert np.allclose(ws.gelu(xs) - ws.gelu(-xs), xs, atol=1e-15, rtol=0)   # x(Phi(x) + Phi(-x)) = x
    assert abs(ws.gelu_grad(np.array(0.0)) - 0.5) < 1e-15


def test_gelu_grad_finite_difference():
    xs = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (ws.gelu(xs + h) - ws.gelu(xs - h)) / (2 * h)
    assert np.max(np.abs(fd - ws.gelu_grad(xs))) < 1e-8


def _tiny(seed=0, shape=(5, 4, 2, 3), B=7):
    rng = np.random.default_rng(seed)
    P = ws.param_count(*shape)
    theta = rng.standard_normal(P) * 0.7
    Ws, mu_in, sd_in, mu_out, sd_out = ws.unpack(theta, *shape)
    # standardisation entries: positive scales
    off = P - 2 * shape[0] - 2 * shape[3]
    theta[off + shape[0]:off + 2 * shape[0]] = rng.uniform(0.5, 2.0, shape[0])
    theta[P - shape[3]:] = rng.uniform(0.5, 2.0, shape[3])
    X = rng.standard_normal((B, shape[0])) * 2
    T = rng.standard_normal((B, shape[3]))
    return theta, shape, X, T


def test_param_count_layout():
    assert ws.param_count(5, 4, 2, 3) == (4 * 5 + 4) + (4 * 4 + 4) + (3 * 4 + 3) + 2 * 5 + 2 * 3
    assert ws.param_count(1088, 512, 3, 64) == 1088 * 512 + 512 + 2 * (512 * 512 + 512) + 512 * 64 + 64 + 2 * 1088 + 2 * 64


def test_loss_grad_matches_finite_differences():
    theta, shape, X, T = _tiny()
    L, g = ws.loss_grad(theta, shape, X, T)
    h = 1e-6
    trained = ws.param_count(*shape) - 2 * shape[0] - 2 * shape[3]
    fd = np.zeros(trained)
    for k in range(trained):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (ws.loss_grad(tp, shape, X, T)[0] - ws.loss_grad(tm, shape, X, T)[0]) / (2 * h)
    assert np.max(np.abs(fd - g[:trained])) < 1e-7 * max(1.0, np.max(np.abs(fd)))
    assert np.all(g[trained:] == 0)


def test_loss_with_zero_weights_is_bias_fit():
    theta, shape, X, T = _tiny(1)
    Ws, mu_in, sd_in, mu_out, sd_out = ws.unpack(theta, *shape)
    W, b = Ws[-1]
    theta2 = theta.copy()
    # zero the output weights: the prediction is the output bias for every row
    off = sum(o * i + o for i, o in ws.layer_dims(*shape)[:-1])
    o, i = ws.layer_dims(*shape)[-1][1], ws.layer_dims(*shape)[-1][0]
    theta2[off:off + o * i] = 0.0
    L, _ = ws.loss_grad(theta2, shape, X, T)
    t_std = (T - mu_out) / sd_out
    assert abs(L - np.mean((b[None, :] - t_std) ** 2)) < 1e-14
    Y = ws.forward(theta2, shape, X)
    assert np.allclose(Y, mu_out + sd_out * b, rtol=1e-15, atol=1e-15)


def test_adam_first_steps_closed_form():
    # bias correction makes every step of a constant gradient exactly lr * g / (|g| + eps)
    g = np.array([3.0, -0.25, 1e-3])
    theta = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    lr, eps = 1e-2, 1e-8
    for step in (1, 2, 3):
        theta, m, v = ws.adam(theta, g, m, v, step, lr, eps=eps)
        assert np.allclose(theta, -step * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    # and it minimises a quadratic
    th, m, v = np.array([5.0]), np.zeros(1), np.zeros(1)
    for step in range(1, 3001):
        th, m, v = ws.adam(th, th.copy(), m, v, step, 0.05)
    assert abs(th[0]) < 1e-2


def test_standardization():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((50, 4)) * [1, 2, 3, 0] + [0, 1, -2, 7]
    T = rng.standard_normal((50, 2))
    mx, sx, mt, st = ws.standardization(X, T)
    assert np.allclose(mx, X.mean(0)) and np.allclose(sx[:3], X.std(0)[:3]) and sx[3] == 1.0
    assert np.allclose(mt, T.mean(0)) and np.allclose(st, T.std(0))


def test_sketch_indices():
    assert ws.sketch_indices(10, 4).tolist() == [0, 2, 5, 7]
    assert ws.sketch_indices(3, 6).tolist() == [0, 0, 1, 1, 2, 2]


def _small_problem(seed=3, n=300, N=12, m=80):
    rng = np.random.default_rng(seed)
    Xf = rng.standard_normal((n, N)) + rng.standard_normal(n)[:, None]
    rowptr = np.arange(m + 1, dtype=np.int32)
    col = np.sort(rng.choice(n, m, replace=False)).astype(np.int32)
    w = np.ones(m)
    r = rng.uniform(0.5, 1.5, m)
    y = rng.standard_normal(m)
    E = rng.standard_normal((m, N)) * np.sqrt(r)[:, None]
    return Xf, rowptr, col, w, r, y, E


def test_exact_target_decodes_to_exact_solution():
    Xf, rowptr, col, w, r, y, E = _small_problem()
    N = Xf.shape[1]
    Xa, info = oracle.cgd_enkf(Xf, rowptr, col, w, r, y, E, tol=1e-14)
    HA, D, Z = info["Zhat"], info["D"], info["Z"]
    # Z from an explicit dense solve of S Z = D (not from CG)
    S = HA @ HA.T / (N - 1) + np.diag(r)
    Zd = np.linalg.solve(S, D)
    assert np.max(np.abs(Z - Zd)) < 1e-9 * np.max(np.abs(Zd))
    W = HA.T @ Zd / (N - 1)
    Z0 = ws.decode(HA, D, r, W)
    assert np.max(np.abs(Z0 - Zd)) < 1e-10 * np.max(np.abs(Zd))
    # and the features' g satisfies (I + HA^T R^-1 HA/(N-1)) c_j = g_j for c_j = W e_j
    F, s = ws.features(HA, D, r, 16)
    g = F[:, 16:].T * s[None, :]
    G = np.eye(N) + HA.T @ (HA / r[:, None]) / (N - 1)
    assert np.max(np.abs(G @ W - g)) < 1e-10 * np.max(np.abs(g))
    T = ws.targets(W, s)
    assert np.allclose(T * s[:, None], W.T)


def test_decoded_residual_lies_in_span_of_HA():
    Xf, rowptr, col, w, r, y, E = _small_problem(4)
    N = Xf.shape[1]
    _, info = oracle.cgd_enkf(Xf, rowptr, col, w, r, y, E, tol=1e-12)
    HA, D = info["Zhat"], info["D"]
    C = np.random.default_rng(0).standard_normal((N, N))
    Z0 = ws.decode(HA, D, r, C)
    res = D - (HA @ (HA.T @ Z0) / (N - 1) + r[:, None] * Z0)
    coef, *_ = np.linalg.lstsq(HA, res, rcond=None)
    assert np.max(np.abs(HA @ coef - res)) < 1e-10 * np.max(np.abs(res))
    # and it equals the N x N form the decoder uses
    assert np.max(np.abs(ows_start_residual(HA, D, r, C) - res)) < 1e-10 * np.max(np.abs(res))


def ows_start_residual(HA, D, r, C):
    return ws.start_residual(HA, D, r, C)


def _gelu_by_hand(z):
    """z Phi(z) with Phi written out through math.erf (independent of the oracle's gelu)."""
    return z * 0.5 * (1.0 + math.erf(z / math.sqrt(2.0)))


def _theta(layers, mu_in, sd_in, mu_out, sd_out):
    """Flat parameter vector in the library's layout from explicit (W, b) pairs."""
    parts = []
    for W, b in layers:
        parts += [np.asarray(W, np.float64).ravel(), np.asarray(b, np.float64)]
    parts += [np.asarray(v, np.float64) for v in (mu_in, sd_in, mu_out, sd_out)]
    return np.concatenate(parts)


def test_forward_one_hidden_layer_evaluated_by_hand():
    # 2 inputs with non-trivial standardisation, 2 GELU hidden units, 1 linear output:
    # a = (x - mu_in)/sd_in = ((3 - 1)/2, (-1 - 2)/0.5) = (1, -6)
    # z1 = 0.5*1 + 0.25*(-6) + 0.2 = -0.8,  z2 = -1*1 + 0.1*(-6) - 0.3 = -1.9
    # y_std = 2 gelu(z1) - 3 gelu(z2) + 0.7,  Y = 10 + 4 y_std
    W1, b1 = [[0.5, 0.25], [-1.0, 0.1]], [0.2, -0.3]
    W2, b2 = [[2.0, -3.0]], [0.7]
    theta = _theta([(W1, b1), (W2, b2)], [1.0, 2.0], [2.0, 0.5], [10.0], [4.0])
    assert theta.size == ws.param_count(2, 2, 1, 1)
    y_std = 2.0 * _gelu_by_hand(-0.8) - 3.0 * _gelu_by_hand(-1.9) + 0.7
    expect = 10.0 + 4.0 * y_std
    Y = ws.forward(theta, (2, 2, 1, 1), np.array([[3.0, -1.0]]))
    assert Y.shape == (1, 1)
    assert abs(Y[0, 0] - expect) <= 1e-14 * abs(expect)
    # the slips this must catch give other values: GELU on the output layer, sd multiplied
    # instead of divided, the output scale and shift swapped
    wrong = [10.0 + 4.0 * _gelu_by_hand(y_std),
             10.0 + 4.0 * (2.0 * _gelu_by_hand(0.5 * 4 + 0.25 * -1.5 + 0.2)
                           - 3.0 * _gelu_by_hand(-1.0 * 4 + 0.1 * -1.5 - 0.3) + 0.7),
             4.0 + 10.0 * y_std]
    assert all(abs(Y[0, 0] - v) > 1e-3 for v in wrong)


def test_forward_two_hidden_layers_evaluated_by_hand():
    # two hidden layers of width 2 (order matters: W1 then W2), x = (0.5, 4), mu_in = (-0.5, 2),
    # sd_in = (0.25, 4): a = (4, 0.5)
    W1, b1 = [[0.3, -0.2], [0.1, 0.4]], [0.0, -1.0]
    W2, b2 = [[1.5, -0.5], [-2.0, 1.0]], [0.1, 0.2]
    W3, b3 = [[0.75, -1.25]], [-0.05]
    theta = _theta([(W1, b1), (W2, b2), (W3, b3)], [-0.5, 2.0], [0.25, 4.0], [-3.0], [0.5])
    a = (4.0, 0.5)
    h1 = [_gelu_by_hand(0.3 * a[0] - 0.2 * a[1] + 0.0), _gelu_by_hand(0.1 * a[0] + 0.4 * a[1] - 1.0)]
    h2 = [_gelu_by_hand(1.5 * h1[0] - 0.5 * h1[1] + 0.1), _gelu_by_hand(-2.0 * h1[0] + 1.0 * h1[1] + 0.2)]
    expect = -3.0 + 0.5 * (0.75 * h2[0] - 1.25 * h2[1] - 0.05)
    Y = ws.forward(theta, (2, 2, 2, 1), np.array([[0.5, 4.0]]))
    assert abs(Y[0, 0] - expect) <= 1e-14 * abs(expect)
    # the hidden layers applied in the other order give another value
    g1 = [_gelu_by_hand(1.5 * a[0] - 0.5 * a[1] + 0.1), _gelu_by_hand(-2.0 * a[0] + 1.0 * a[1] + 0.2)]
    g2 = [_gelu_by_hand(0.3 * g1[0] - 0.2 * g1[1]), _gelu_by_hand(0.1 * g1[0] + 0.4 * g1[1] - 1.0)]
    swapped = -3.0 + 0.5 * (0.75 * g2[0] - 1.25 * g2[1] - 0.05)
    assert abs(Y[0, 0] - swapped) > 1e-3


def test_start_residual_amplifies_coefficient_error():
    """The decoded start's residual is linear in the coefficient error, HA A (C - W) with
    A = I + HA^T R^-1 HA/(N-1) (closed form from S = HA HA^T/(N-1) + R), so its size relative
    to ||d_j|| (the zero start's residual) is the coefficient error amplified by A's spectrum,
    which grows with m. On the 512^2 GRF workload shrunk 4x per side (m = 4,096, N = 64) a 5 %
    error in c_j already gives a start residual above ||d_j||: the true-residual judge of the
    learned start then prefers the zero start."""
    from synth.problems import workload
    P = workload("grf512_N64_m65536", seed=3, scale=4)
    N = P.N
    E = np.random.default_rng(1).standard_normal((P.m, N)) * np.sqrt(P.r)[:, None]
    _, info = oracle.cgd_enkf(P.Xf, P.rowptr, P.col, P.w, P.r, P.y, E, tol=1e-12)
    HA, D, Z = info["Zhat"], info["D"], info["Z"]
    W = HA.T @ Z / (N - 1)
    dn = np.linalg.norm(D, axis=0)
    # exact coefficients: the start is the solution, its residual is the CG tolerance's
    assert np.max(np.linalg.norm(ws.start_residual(HA, D, P.r, W), axis=0) / dn) < 1e-9
    Dl = np.random.default_rng(2).standard_normal(W.shape)
    Dl *= 0.05 * np.linalg.norm(W, axis=0) / np.linalg.norm(Dl, axis=0)
    res = ws.start_residual(HA, D, P.r, W + Dl)
    A = np.eye(N) + HA.T @ (HA / P.r[:, None]) / (N - 1)
    assert np.max(np.abs(res - HA @ (A @ Dl))) < 1e-8 * np.max(np.abs(res))
    rel = np.linalg.norm(res, axis=0) / dn
    assert np.median(rel) > 1.0
