"""Oracle: a plain, slow FP64 CPU restatement of the particle-inference path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import
this package.  It shares no code with ``paper_2010_08454_gb300`` and does not
import it; the C sources here are compiled on their own with the host C
compiler (``oracle/build.py``).

Every function cites the passage of the paper (or the published method) it
restates in its C source.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_LIB = None

PURPOSE_POLY_TRACE = 1
PURPOSE_LGSSM_PROPAGATE = 2
PURPOSE_RESAMPLE = 3
PURPOSE_LEARNED_TRACE = 4
PURPOSE_FORWARD_SIM = 5


class Poly(ctypes.Structure):
    _fields_ = [("min_deg", ctypes.c_int), ("max_deg", ctypes.c_int),
                ("coef_offset", ctypes.c_int), ("obs_sigma", ctypes.c_double),
                ("prior_sigma", ctypes.c_double)]


class Lgssm(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_double), ("q_sigma", ctypes.c_double),
                ("r_sigma", ctypes.c_double)]


class IsResult(ctypes.Structure):
    _fields_ = [("log_z", ctypes.c_double), ("lse", ctypes.c_double), ("ess", ctypes.c_double),
                ("max_lw", ctypes.c_double), ("argmax", ctypes.c_int64),
                ("n_particles", ctypes.c_int64), ("map_deg", ctypes.c_int32),
                ("n_deg", ctypes.c_int32), ("p_n", ctypes.c_double * 4),
                ("mean_c", ctypes.c_double * 6), ("deg_mean", (ctypes.c_double * 6) * 4),
                ("deg_var", (ctypes.c_double * 6) * 4), ("deg_max_lw", ctypes.c_double * 4),
                ("deg_argmax", ctypes.c_int64 * 4), ("status", ctypes.c_int32),
                ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {
            "log_z": self.log_z, "lse": self.lse, "ess": self.ess, "max_lw": self.max_lw,
            "argmax": self.argmax, "n_particles": self.n_particles, "map_deg": self.map_deg,
            "n_deg": self.n_deg, "p_n": np.array(self.p_n[:]),
            "mean_c": np.array(self.mean_c[:]),
            "deg_mean": np.array([r[:] for r in self.deg_mean]),
            "deg_var": np.array([r[:] for r in self.deg_var]),
            "deg_max_lw": np.array(self.deg_max_lw[:]),
            "deg_argmax": np.array(self.deg_argmax[:]),
        }


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def lib():
    """Load liboracle.so, building it first if needed."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i64, u64, u32, i32, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_int32, ctypes.c_double)
        sig = {
            "orc_philox4x32_10": (None, [vp, vp, vp]),
            "orc_philox_block": (None, [u64, u32, u32, u32, u32, u32, vp]),
            "orc_u01": (dbl, [u32]),
            "orc_box_muller": (None, [u32, u32, vp, vp]),
            "orc_uniform_discrete": (ctypes.c_int, [u32, ctypes.c_int, ctypes.c_int]),
            "orc_ln32": (ctypes.c_float, [ctypes.c_float]),
            "orc_cos2pi32": (ctypes.c_float, [ctypes.c_float]),
            "orc_normal32": (ctypes.c_float, [u32, u32]),
            "orc_poly_trace": (dbl, [vp, vp, vp, i64, u64, u32, u32, vp, vp]),
            "orc_is_poly": (None, [vp, vp, vp, i64, i64, u64, u32, vp, vp, vp]),
            "orc_is_poly_indices": (None, [vp, vp, vp, i64, vp, i64, u64, u32, vp, vp, vp]),
            "orc_lse_ess": (None, [vp, i64, vp, vp, vp, vp]),
            "orc_posterior_poly": (None, [vp, vp, vp, vp, i64, vp]),
            "orc_exp32": (ctypes.c_float, [ctypes.c_float]),
            "orc_fixed_shift": (ctypes.c_int, [i64]),
            "orc_quantize_weights": (None, [vp, i64, vp]),
            "orc_resample_systematic": (ctypes.c_int, [vp, i64, i64, u64, u32, u32, vp]),
            "orc_resample_from_lw": (ctypes.c_int, [vp, i64, i64, u64, u32, u32, vp]),
            "orc_gather": (None, [vp, i64, vp, i64, vp]),
            "orc_kalman_logz": (dbl, [vp, vp, i64]),
            "orc_smc_lgssm": (dbl, [vp, vp, i64, i64, u64, ctypes.c_int, vp, vp, vp, vp]),
            "orc_blr_evidence": (dbl, [vp, vp, i64, ctypes.c_int, dbl, dbl, vp, vp]),
            "orc_poly_exact": (dbl, [vp, vp, vp, i64, vp, vp, vp]),
            "orc_enumerate": (ctypes.c_int, [ctypes.c_int, vp, i64, ctypes.c_int, vp, vp,
                                             ctypes.c_int]),
            "orc_is_discrete": (None, [ctypes.c_int, vp, i64, i64, u64, vp, vp]),
            "orc_customdist_is": (None, [vp, vp, i64, i64, u64, vp, vp]),
            "orc_customdist_exact": (None, [vp, vp, i64, vp]),
            "orc_set_threads": (None, [ctypes.c_int]),
            "orc_get_threads": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
        from . import mlp as _mlp
        _mlp._register(L)
    return _LIB


def set_threads(n):
    lib().orc_set_threads(int(n))


def get_threads():
    return lib().orc_get_threads()


# ---- random numbers -------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def philox_block(seed, particle, instance, step, purpose, block):
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox_block(seed, particle, instance, step, purpose, block, _p(out))
    return out


def u01(w):
    return lib().orc_u01(int(w))


def box_muller(wa, wb):
    z0, z1 = ctypes.c_double(), ctypes.c_double()
    lib().orc_box_muller(int(wa), int(wb), ctypes.byref(z0), ctypes.byref(z1))
    return z0.value, z1.value


def ln32(u):
    return lib().orc_ln32(float(u))


def cos2pi32(u):
    return lib().orc_cos2pi32(float(u))


def normal32(wa, wb):
    """The reproducible FP32 Box-Muller draw (cosine branch) of two words."""
    return lib().orc_normal32(int(wa), int(wb))


def uniform_discrete(w, lo, hi):
    return lib().orc_uniform_discrete(int(w), lo, hi)


# ---- polynomial model ----------------------------------------------------
def poly_model(min_deg=2, max_deg=5, coef_offset=1, obs_sigma=0.5, prior_sigma=10.0):
    return Poly(min_deg, max_deg, coef_offset, obs_sigma, prior_sigma)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def poly_trace(model, x, y, seed, instance, particle):
    x, y = _f64(x), _f64(y)
    n = ctypes.c_int()
    c = np.zeros(6)
    lw = lib().orc_poly_trace(ctypes.byref(model), _p(x), _p(y), len(x), seed, instance,
                              particle, ctypes.byref(n), _p(c))
    return lw, n.value, c


def is_poly(model, x, y, N, seed, instance=0):
    """Likelihood weighting over particles 0..N-1: (lw[N], n[N], c[N,6])."""
    x, y = _f64(x), _f64(y)
    lw = np.zeros(N)
    n = np.zeros(N, dtype=np.int32)
    c = np.zeros((N, 6))
    lib().orc_is_poly(ctypes.byref(model), _p(x), _p(y), len(x), N, seed, instance, _p(lw),
                      _p(n), _p(c))
    return lw, n, c


def is_poly_indices(model, x, y, idx, seed, instance=0):
    x, y = _f64(x), _f64(y)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    K = len(idx)
    lw = np.zeros(K)
    n = np.zeros(K, dtype=np.int32)
    c = np.zeros((K, 6))
    lib().orc_is_poly_indices(ctypes.byref(model), _p(x), _p(y), len(x), _p(idx), K, seed,
                              instance, _p(lw), _p(n), _p(c))
    return lw, n, c


def lse_ess(lw):
    lw = _f64(lw)
    lse, ess, mx = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    am = ctypes.c_int64()
    lib().orc_lse_ess(_p(lw), len(lw), ctypes.byref(lse), ctypes.byref(ess), ctypes.byref(mx),
                      ctypes.byref(am))
    return {"lse": lse.value, "ess": ess.value, "max_lw": mx.value, "argmax": am.value,
            "log_z": lse.value - math.log(len(lw))}


def posterior_poly(model, lw, n, c):
    lw = _f64(lw)
    n = np.ascontiguousarray(n, dtype=np.int32)
    c = np.ascontiguousarray(c, dtype=np.float64).reshape(-1, 6)
    res = IsResult()
    lib().orc_posterior_poly(ctypes.byref(model), _p(lw), _p(n), _p(c), len(lw),
                             ctypes.byref(res))
    return res.as_dict()


def infer_is_poly(model, x, y, N, seed, instance=0):
    """The whole likelihood-weighting pass: traces, normalisation, summary."""
    lw, n, c = is_poly(model, x, y, N, seed, instance)
    return posterior_poly(model, lw, n, c), (lw, n, c)


# ---- resampling ----------------------------------------------------------
def exp32(d):
    return lib().orc_exp32(float(d))


def fixed_shift(N):
    return lib().orc_fixed_shift(N)


def quantize_weights(lw32):
    lw32 = np.ascontiguousarray(lw32, dtype=np.float32)
    q = np.zeros(len(lw32), dtype=np.uint64)
    lib().orc_quantize_weights(_p(lw32), len(lw32), _p(q))
    return q


def resample_systematic(q, M, seed, instance=0, step=0):
    q = np.ascontiguousarray(q, dtype=np.uint64)
    anc = np.zeros(M, dtype=np.int32)
    st = lib().orc_resample_systematic(_p(q), len(q), M, seed, instance, step, _p(anc))
    return st, anc


def resample_from_lw(lw32, M, seed, instance=0, step=0):
    lw32 = np.ascontiguousarray(lw32, dtype=np.float32)
    anc = np.zeros(M, dtype=np.int32)
    st = lib().orc_resample_from_lw(_p(lw32), len(lw32), M, seed, instance, step, _p(anc))
    return st, anc


def gather(records, anc):
    records = np.ascontiguousarray(records)
    anc = np.ascontiguousarray(anc, dtype=np.int32)
    stride = records.strides[0] if records.ndim > 1 else records.itemsize
    out = np.empty((len(anc),) + records.shape[1:], dtype=records.dtype)
    lib().orc_gather(_p(records), stride, _p(anc), len(anc), _p(out))
    return out


# ---- state-space model -------------------------------------------------
def lgssm_model(phi=0.9, q_sigma=1.0, r_sigma=0.5):
    return Lgssm(phi, q_sigma, r_sigma)


def kalman_logz(model, y):
    y = _f64(y)
    return lib().orc_kalman_logz(ctypes.byref(model), _p(y), len(y))


def smc_lgssm(model, y, N, seed, state_f32=False):
    """Bootstrap filter; state_f32 holds state and log-weights in FP32 (the method's policy)."""
    y = _f64(y)
    T = len(y)
    ess = np.zeros(T)
    res = np.zeros(T, dtype=np.int32)
    x = np.zeros(N)
    lw = np.zeros(N)
    logz = lib().orc_smc_lgssm(ctypes.byref(model), _p(y), T, N, seed, int(state_f32), _p(ess),
                               _p(res), _p(x), _p(lw))
    return {"log_z": logz, "ess": ess, "resampled": res, "x": x, "lw": lw}


# ---- conjugate evidence -------------------------------------------------
def blr_evidence(x, y, ncoef, sigma, prior_sigma):
    x, y = _f64(x), _f64(y)
    mean, var = np.zeros(ncoef), np.zeros(ncoef)
    lz = lib().orc_blr_evidence(_p(x), _p(y), len(x), ncoef, sigma, prior_sigma, _p(mean),
                                _p(var))
    return lz, mean, var


def poly_exact(model, x, y):
    x, y = _f64(x), _f64(y)
    p_n = np.zeros(4)
    dm = np.zeros((4, 6))
    dv = np.zeros((4, 6))
    lz = lib().orc_poly_exact(ctypes.byref(model), _p(x), _p(y), len(x), _p(p_n), _p(dm), _p(dv))
    return {"log_z": lz, "p_n": p_n, "deg_mean": dm, "deg_var": dv}


# ---- discrete models ----------------------------------------------------
DISCRETE_MODELS = {"biasedcoin": 0, "binomial": 1, "geometric": 2}


def enumerate_model(name, data, max_depth=64, max_out=256):
    data = np.ascontiguousarray(data, dtype=np.int32)
    vals, probs = np.zeros(max_out), np.zeros(max_out)
    k = lib().orc_enumerate(DISCRETE_MODELS[name], _p(data), len(data), max_depth, _p(vals),
                            _p(probs), max_out)
    if k < 0:
        raise ValueError("enumeration failed")
    order = np.argsort(vals[:k])
    return vals[:k][order], probs[:k][order]


def is_discrete(name, data, N, seed):
    data = np.ascontiguousarray(data, dtype=np.int32)
    vals, lw = np.zeros(N), np.zeros(N)
    lib().orc_is_discrete(DISCRETE_MODELS[name], _p(data), len(data), N, seed, _p(vals), _p(lw))
    return vals, lw


# ---- customdist: a user-defined two-Gaussian density, observed --------------
def customdist_params(w1=0.3, mu1=-2.0, s1=0.5, mu2=1.5, s2=1.0, obs_sigma=1.0):
    """{w1, mu1, s1, mu2, s2, obs_sigma} as FP64 (the GPU takes the same values as FP32)."""
    return np.array([w1, mu1, s1, mu2, s2, obs_sigma], dtype=np.float32).astype(np.float64)


def customdist_is(prm, y, N, seed):
    y = np.ascontiguousarray(y, dtype=np.float32)
    x, lw = np.zeros(N), np.zeros(N)
    lib().orc_customdist_is(_p(np.ascontiguousarray(prm, dtype=np.float64)), _p(y), len(y), N,
                            seed, _p(x), _p(lw))
    return x, lw


def customdist_exact(prm, y):
    """log Z, posterior mean and variance of x (closed form)."""
    y = np.ascontiguousarray(y, dtype=np.float32)
    out = np.zeros(3)
    lib().orc_customdist_exact(_p(np.ascontiguousarray(prm, dtype=np.float64)), _p(y), len(y),
                               _p(out))
    return {"log_z": out[0], "mean": out[1], "var": out[2]}
