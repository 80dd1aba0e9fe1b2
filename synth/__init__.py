"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds none of the inference method's arithmetic: it only draws
data sets (and test inputs such as log-weight vectors) with numpy's PCG64
generator, in FP32, in the shapes of the paper's line-fitting workload
(Fig. 1, §5.1 Table 1 "linefitting") and of the state-space and batched
workloads built on it.  Both sides receive the same arrays.
"""
import numpy as np

TRUE_CUBIC = (1.0, -2.0, 0.0, 0.5)  # y = 1 - 2x + 0.5x^3


def poly_dataset(L, seed, coefs=TRUE_CUBIC, noise_sigma=0.5):
    """L points with x ~ U[-1, 1] and y = sum_k coefs[k] x^k + N(0, noise_sigma^2), FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(-1.0, 1.0, size=L)
    f = np.zeros(L)
    for k, ck in enumerate(coefs):
        f = f + ck * x ** k
    y = f + noise_sigma * rng.standard_normal(L)
    return x.astype(np.float32), y.astype(np.float32)


def lgssm_dataset(T, seed, phi=0.9, q_sigma=1.0, r_sigma=0.5):
    """Observations y_1..y_T of x_t = phi x_{t-1} + N(0, q^2), y_t = x_t + N(0, r^2), x_0 = 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = 0.0
    y = np.zeros(T)
    for t in range(T):
        x = phi * x + q_sigma * rng.standard_normal()
        y[t] = x + r_sigma * rng.standard_normal()
    return y.astype(np.float32)


def batched_instances(n_inst, seed, L_range=(16, 4096), N_range=(2 ** 10, 2 ** 16),
                      deg_range=(2, 5), noise_sigma=0.5):
    """Independent line-fitting instances of uneven size.

    Data lengths and particle counts are log-uniform in their ranges, the true
    degree is uniform, the true coefficients are N(0, 1), x ~ U[-1, 1] and the
    noise is N(0, noise_sigma^2).  Returns a dict of CSR-packed FP32 arrays:
    x, y (concatenated), data_off[n_inst + 1], part_off[n_inst + 1] and the
    generating degrees and coefficients.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = np.log(L_range[0]), np.log(L_range[1] + 1)
    L = np.clip(np.floor(np.exp(rng.uniform(lo, hi, n_inst))), L_range[0], L_range[1])
    lo, hi = np.log(N_range[0]), np.log(N_range[1] + 1)
    N = np.clip(np.floor(np.exp(rng.uniform(lo, hi, n_inst))), N_range[0], N_range[1])
    L = L.astype(np.int64)
    N = N.astype(np.int64)
    deg = rng.integers(deg_range[0], deg_range[1] + 1, n_inst)
    coefs = np.zeros((n_inst, 6))
    xs, ys = [], []
    for b in range(n_inst):
        c = rng.standard_normal(deg[b] + 1)
        coefs[b, :deg[b] + 1] = c
        x = rng.uniform(-1.0, 1.0, L[b])
        f = np.zeros(L[b])
        for k in range(deg[b] + 1):
            f = f + c[k] * x ** k
        xs.append(x)
        ys.append(f + noise_sigma * rng.standard_normal(L[b]))
    data_off = np.zeros(n_inst + 1, dtype=np.int64)
    data_off[1:] = np.cumsum(L)
    part_off = np.zeros(n_inst + 1, dtype=np.int64)
    part_off[1:] = np.cumsum(N)
    return {"x": np.concatenate(xs).astype(np.float32), "y": np.concatenate(ys).astype(np.float32),
            "data_off": data_off, "part_off": part_off, "L": L, "N": N, "deg": deg,
            "coefs": coefs}


def prior_datasets(n_sets, L, seed, deg_range=(2, 5), prior_sigma=10.0, noise_sigma=0.5):
    """Data sets drawn from the line-fitting model's own prior (held-out test sets).

    degree ~ uniform{deg_range}, degree+1 coefficients ~ N(0, prior_sigma^2),
    x ~ U[-1, 1], y = f(x) + N(0, noise_sigma^2).  Returns x, y of shape [n_sets, L].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    deg = rng.integers(deg_range[0], deg_range[1] + 1, n_sets)
    x = rng.uniform(-1.0, 1.0, (n_sets, L))
    y = np.zeros((n_sets, L))
    coefs = np.zeros((n_sets, 6))
    for b in range(n_sets):
        c = prior_sigma * rng.standard_normal(deg[b] + 1)
        coefs[b, :deg[b] + 1] = c
        f = np.zeros(L)
        for k in range(deg[b] + 1):
            f = f + c[k] * x[b] ** k
        y[b] = f + noise_sigma * rng.standard_normal(L)
    return {"x": x.astype(np.float32), "y": y.astype(np.float32), "deg": deg, "coefs": coefs}


def log_weights(N, seed, kind="normal", scale=3.0):
    """FP32 log-weight vectors with the structures resampling must handle."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "normal":
        lw = scale * rng.standard_normal(N)
    elif kind == "equal":
        lw = np.full(N, -1.25)
    elif kind == "onehot":
        lw = np.full(N, -np.inf)
        lw[rng.integers(0, N)] = 0.0
    elif kind == "sparse":
        lw = np.full(N, -np.inf)
        hot = rng.choice(N, size=max(1, N // 100), replace=False)
        lw[hot] = scale * rng.standard_normal(len(hot))
    elif kind == "wide":
        lw = rng.uniform(-200.0, 0.0, N)
    else:
        raise ValueError(kind)
    return lw.astype(np.float32)


def fixed_weights(N, seed, max_bits=40):
    """u64 fixed-point weights (zeros included) whose sum stays below 2^61."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bits = min(max_bits, 60 - int(np.ceil(np.log2(max(N, 2)))))
    q = rng.integers(0, 2 ** bits, N, dtype=np.uint64)
    q[rng.random(N) < 0.3] = 0
    return q


def mlp_weights(seed, sizes=((256, 64), (256, 256), (48, 256)), bias_scale=0.05):
    """Seeded network parameters: W uniform in +-1/sqrt(fan_in) rounded to values
    BF16 represents exactly (ties to even), biases uniform in +-bias_scale, FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for n_out, n_in in sizes:
        w = rng.uniform(-1.0, 1.0, (n_out, n_in)) / np.sqrt(n_in)
        w = w.astype(np.float32)
        bits = w.view(np.uint32).astype(np.uint64)
        bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
        out.append(bits.astype(np.uint32).view(np.float32).reshape(n_out, n_in))
        out.append(rng.uniform(-bias_scale, bias_scale, n_out).astype(np.float32))
    return out
