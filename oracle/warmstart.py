"""FP64 oracle of the learned CG warm start (test infrastructure only).

The paper's CG starts from zero (Sec. 3.3); the learned warm start is an addition of this
library, built on one identity of the paper's own system: from S Z = D with
S = HA HA^T/(N-1) + R (Eq. matvec_decomp) follows R Z = D - HA W with W = HA^T Z/(N-1),
i.e. every solution column has the form z_j = R^{-1}(d_j - HA c_j) with c_j = W e_j (the
N-vector the final update X_a = X_f + A W uses). So a model only has to predict the N-vector
c_j; the decoder z0_j = R^{-1}(d_j - HA c_j) turns it into a start whose residual
d_j - S z0_j = HA ((I + HA^T R^{-1} HA/(N-1)) c_j - g_j) lies in span(HA), with
g_j = HA^T R^{-1} d_j/(N-1).

Model: per column j, features f_j = [d_j(sketch)/s_j, g_j/s_j] (a fixed sketch of K
observation indices, s_j the RMS of d_j over the sketch, 1 if that is 0), standardised per
feature; an MLP of L hidden layers of width H with GELU (Hendrycks & Gimpel 2016, exact erf
form x Phi(x)); output the standardised target t_j = c_j/s_j. Training minimises the mean
squared error in standardised units with Adam (Kingma & Ba 2015, Algorithm 1).

Parameter layout (one flat FP32 vector, the library's interface): for each layer l =
1..L+1 the weight W_l [out_l][in_l] (row-major) then the bias b_l [out_l]; then mu_in [in],
sd_in [in], mu_out [out], sd_out [out].
"""
import numpy as np
from scipy.special import erf


# ------------------------------------------------------------------ model layout
def layer_dims(in_dim, hidden, layers, out_dim):
    dims = [in_dim] + [hidden] * layers + [out_dim]
    return list(zip(dims[:-1], dims[1:]))


def param_count(in_dim, hidden, layers, out_dim):
    n = sum(o * i + o for i, o in layer_dims(in_dim, hidden, layers, out_dim))
    return n + 2 * in_dim + 2 * out_dim


def unpack(theta, in_dim, hidden, layers, out_dim):
    """Views of the flat parameter vector: ([(W, b), ...], mu_in, sd_in, mu_out, sd_out)."""
    theta = np.asarray(theta, dtype=np.float64)
    off, Ws = 0, []
    for i, o in layer_dims(in_dim, hidden, layers, out_dim):
        W = theta[off:off + o * i].reshape(o, i)
        off += o * i
        b = theta[off:off + o]
        off += o
        Ws.append((W, b))
    mu_in = theta[off:off + in_dim]; off += in_dim
    sd_in = theta[off:off + in_dim]; off += in_dim
    mu_out = theta[off:off + out_dim]; off += out_dim
    sd_out = theta[off:off + out_dim]; off += out_dim
    assert off == theta.size
    return Ws, mu_in, sd_in, mu_out, sd_out


# ------------------------------------------------------------------ GELU
def gelu(x):
    """x Phi(x) with Phi the standard normal CDF (Hendrycks & Gimpel 2016, exact form)."""
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


# ------------------------------------------------------------------ forward / backward
def forward(theta, shape, X, keep=False):
    """Raw prediction Y = mu_out + sd_out * MLP((X - mu_in)/sd_in) for rows X [B][in]."""
    Ws, mu_in, sd_in, mu_out, sd_out = unpack(theta, *shape)
    a = (np.asarray(X, np.float64) - mu_in) / sd_in
    acts, pre = [a], []
    for l, (W, b) in enumerate(Ws):
        z = a @ W.T + b
        pre.append(z)
        a = gelu(z) if l < len(Ws) - 1 else z
        acts.append(a)
    y_std = a
    Y = mu_out + sd_out * y_std
    if keep:
        return Y, y_std, acts, pre
    return Y


def loss_grad(theta, shape, X, T):
    """Mean squared error in standardised units, L = sum((y_std - (T - mu_out)/sd_out)^2)/(B out),
    and its gradient with respect to every trained entry of theta (the standardisation
    entries get zero), by the chain rule layer by layer."""
    Ws, mu_in, sd_in, mu_out, sd_out = unpack(theta, *shape)
    _, y_std, acts, pre = forward(theta, shape, X, keep=True)
    t_std = (np.asarray(T, np.float64) - mu_out) / sd_out
    B, out = y_std.shape
    diff = y_std - t_std
    L = float(np.sum(diff * diff) / (B * out))
    g = 2.0 * diff / (B * out)                # dL/dz of the output layer
    grads = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        W, _ = Ws[l]
        grads[l] = (g.T @ acts[l], g.sum(axis=0))   # dL/dW_l = g^T a_{l-1}, dL/db_l
        if l > 0:
            g = (g @ W) * gelu_grad(pre[l - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    flat = np.concatenate([flat, np.zeros(2 * shape[0] + 2 * shape[3])])
    return L, flat


def adam(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) at step number `step` >= 1; returns the
    new (theta, m, v). Entries with zero gradient history stay put."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def standardization(X, T):
    """Per-feature mean and standard deviation (population form; 1 where it is 0)."""
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    sx, st = X.std(axis=0), T.std(axis=0)
    return X.mean(axis=0), np.where(sx > 0, sx, 1.0), T.mean(axis=0), np.where(st > 0, st, 1.0)


# ------------------------------------------------------------------ warm-start maps
def sketch_indices(m, K):
    """The K sketch rows: i_k = floor(k m / K) (all rows, repeated, when m < K)."""
    return (np.arange(K, dtype=np.int64) * m) // K


def features(HA, D, r, K):
    """F [N][K + N]: f_j = [d_j(sketch)/s_j, g_j/s_j], g_j = HA^T R^{-1} d_j/(N-1); also s [N]."""
    m, N = D.shape
    idx = sketch_indices(m, K)
    Sk = D[idx, :]                                   # (K, N)
    s = np.sqrt(np.mean(Sk * Sk, axis=0))
    s = np.where(s > 0, s, 1.0)
    g = HA.T @ (D / r[:, None]) / (N - 1)            # (N, N): column j is g_j
    F = np.concatenate([Sk.T / s[:, None], g.T / s[:, None]], axis=1)
    return F, s


def targets(W, s):
    """T [N][N]: t_j = c_j/s_j with c_j = W e_j (the exact solve's W = HA^T Z/(N-1))."""
    return (W / s[None, :]).T


def decode(HA, D, r, C):
    """Z0 = R^{-1}(D - HA C), C [N][N] with column j the predicted c_j."""
    return (D - HA @ C) / r[:, None]


def start_residual(HA, D, r, C):
    """Residual of the decoded start, D - S z0 = HA E with
    E = C + (HA^T R^-1 HA C - HA^T R^-1 D)/(N-1) (from S = HA HA^T/(N-1) + R)."""
    N = HA.shape[1]
    Gw = HA.T @ (HA / r[:, None])
    g = HA.T @ (D / r[:, None])
    return HA @ (C + (Gw @ C - g) / (N - 1))
