"""Oracle wrappers for the learned proposal (oracle/mlp.c).  Test infrastructure only."""
import ctypes

import numpy as np

IN, H, OUT, NPTS = 64, 256, 48, 32
_L = None


def _register(L):
    global _L
    vp, i64, u64, u32, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                              ctypes.c_double)
    sig = {
        "orc_bf16": (ctypes.c_float, [ctypes.c_float]),
        "orc_mlp_set_bf16": (None, [ctypes.c_int]),
        "orc_mlp_features": (None, [vp, vp, vp]),
        "orc_mlp_forward": (None, [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "orc_proposal_logq": (dbl, [vp, vp, ctypes.c_int, vp, vp]),
        "orc_learned_trace": (dbl, [vp, vp, vp, vp, i64, u64, u32, u32, vp, vp]),
        "orc_learned_is": (None, [vp, vp, vp, vp, i64, i64, u64, u32, vp, vp, vp]),
        "orc_forward_sim": (None, [vp, u64, u32, vp, vp, vp, vp]),
        "orc_mlp_loss_grad": (dbl, [vp] * 10 + [i64] + [vp] * 6),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _L = L
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def bf16(v):
    return _L.orc_bf16(float(v))


def set_bf16(on):
    _L.orc_mlp_set_bf16(int(on))


def features(x, y):
    x, y = _f32(x), _f32(y)
    out = np.zeros(IN, dtype=np.float32)
    _L.orc_mlp_features(_p(x), _p(y), _p(out))
    return out


def forward(weights, feat):
    W1, b1, W2, b2, W3, b3 = [_f32(w) for w in weights]
    feat = _f32(feat)
    h1, h2, out = np.zeros(H), np.zeros(H), np.zeros(OUT)
    _L.orc_mlp_forward(_p(W1), _p(b1), _p(W2), _p(b2), _p(W3), _p(b3), _p(feat), _p(h1), _p(h2),
                       _p(out))
    return out, h1, h2


def proposal_logq(model, out, n, c):
    out, c = _f64(out), _f64(c)
    g = np.zeros(OUT)
    lq = _L.orc_proposal_logq(ctypes.byref(model), _p(out), int(n), _p(c), _p(g))
    return lq, g


def learned_is(model, out, x, y, N, seed, instance=0):
    out, x, y = _f64(out), _f64(x), _f64(y)
    lw, n, c = np.zeros(N), np.zeros(N, dtype=np.int32), np.zeros((N, 6))
    _L.orc_learned_is(ctypes.byref(model), _p(out), _p(x), _p(y), len(x), N, seed, instance,
                      _p(lw), _p(n), _p(c))
    return lw, n, c


def forward_sim(model, seed, pair):
    x, y = np.zeros(NPTS, dtype=np.float32), np.zeros(NPTS, dtype=np.float32)
    n = ctypes.c_int()
    c = np.zeros(6)
    _L.orc_forward_sim(ctypes.byref(model), seed, pair, _p(x), _p(y), ctypes.byref(n), _p(c))
    return x, y, n.value, c


def loss_grad(model, weights, feats, n, c, with_grad=True):
    W1, b1, W2, b2, W3, b3 = [_f32(w) for w in weights]
    feats, n, c = _f32(feats), np.ascontiguousarray(n, dtype=np.int32), _f64(c)
    B = len(n)
    if with_grad:
        g = [np.zeros(w.shape) for w in (W1, b1, W2, b2, W3, b3)]
        gp = [_p(a) for a in g]
    else:
        g, gp = None, [None] * 6
    loss = _L.orc_mlp_loss_grad(ctypes.byref(model), _p(W1), _p(b1), _p(W2), _p(b2), _p(W3),
                                _p(b3), _p(feats), _p(n), _p(c), B, *gp)
    return loss, g
