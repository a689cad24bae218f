"""Seeded random initial parameters of the warm-start MLP (an input generator: no model
arithmetic). Layout: per layer W [out][in] then b [out]; then mu_in, sd_in, mu_out, sd_out."""
import numpy as np


def init_params(in_dim, hidden, layers, out_dim, seed, out_scale=0.1):
    """He-normal hidden weights (std sqrt(2 / fan_in)), output weights with std
    out_scale / sqrt(fan_in), zero biases, identity standardisation; float32."""
    rng = np.random.default_rng([seed, 0x31A7])
    dims = [in_dim] + [hidden] * layers + [out_dim]
    parts = []
    for l, (fi, fo) in enumerate(zip(dims[:-1], dims[1:])):
        std = np.sqrt(2.0 / fi) if l < layers else out_scale / np.sqrt(fi)
        parts.append(rng.standard_normal(fo * fi) * std)
        parts.append(np.zeros(fo))
    parts += [np.zeros(in_dim), np.ones(in_dim), np.zeros(out_dim), np.ones(out_dim)]
    return np.concatenate(parts).astype(np.float32)
