"""FP64 reference of the warm-start network and its features.

Test infrastructure (see ``oracle/__init__``). The network and its loss are
defined in the library's interface (an 8 -> 64 -> 64 -> 2 ReLU MLP giving
rho - 1 with rho = t_CCSD / t_MP2, weighted squared error with weights
|t_MP2|^2 normalised to mean one); this module evaluates them in numpy FP64
with explicit backpropagation, so the GPU gradients can be checked. The
features follow the same definitions from the oracle's own integrals.
"""
from __future__ import annotations

import numpy as np

F, H, O = 8, 64, 2
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
         ("W3", (O, H)), ("b3", (O,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unflatten(p):
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def flatten(d):
    return np.concatenate([d[name].ravel() for name, _ in SIZES])


def forward(p, X):
    w = unflatten(p)
    z1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w["W3"].T + w["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_grad(p, X, Y):
    """L = mean_s w_s |y_s - t_s|^2 and dL/dp (chain rule, layer by layer)."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    w = unflatten(p)
    y, (x, z1, h1, z2, h2) = forward(p, X)
    n = X.shape[0]
    e = y - Y[:, :2]
    wt = Y[:, 2]
    loss = float(np.sum(wt[:, None] * e * e) / n)
    dy = 2.0 * wt[:, None] * e / n
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dh2 = (dy @ w["W3"]) * (z2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ w["W2"]) * (z1 > 0)
    g["W1"] = dh1.T @ x
    g["b1"] = dh1.sum(0)
    return loss, flatten(g)


def features(L, eps, n_occ, n):
    """Features of the first n unique elements (i<j, a<b, row-major pairs)."""
    from .integrals import antisym_full
    g = antisym_full(L)
    o = n_occ
    v = g.shape[0] - o
    O_, V_ = slice(0, o), slice(o, o + v)
    oovv = g[O_, O_, V_, V_]
    dij = np.array([[g[i, j, i, j].real for j in range(o)] for i in range(o)])
    dab = np.array([[g[o + a, o + b, o + a, o + b].real for b in range(v)] for a in range(v)])
    dia = np.array([[g[i, o + a, i, o + a].real for a in range(v)] for i in range(o)])
    iu = [(i, j) for i in range(o) for j in range(i + 1, o)]
    gs = np.sqrt(np.mean([dij[i, j] ** 2 for i, j in iu]))
    ds = 2.0 * (np.sum(eps[o:]) - np.sum(eps[:o])) / (o + v)
    au = [(a, b) for a in range(v) for b in range(a + 1, v)]
    out = np.empty((n, F))
    k = 0
    for i, j in iu:
        for a, b in au:
            if k == n:
                return out
            D = eps[i] + eps[j] - eps[o + a] - eps[o + b]
            t = np.conj(oovv[i, j, a, b]) / D
            s1 = dia[i, a] + dia[j, b]
            s2 = dia[i, b] + dia[j, a]
            out[k] = [np.log10(abs(t) + 1e-300), D / ds, dij[i, j] / gs, dab[a, b] / gs,
                      (s1 + s2) / gs, abs(s1 - s2) / gs, (eps[i] + eps[j]) / ds,
                      abs(oovv[i, j, a, b]) / gs]
            k += 1
    return out[:k]


def guess_features(H, g, eps, n_occ, seed, n):
    """Features of the learned Davidson start for the first n 2h1p elements
    (j<k row-major, b fastest) of a root seeded at the 1h element `seed`:
    log10|c|, Re(d_i - d_nu) / ds, |W_ibjk| / gs, [seed is j or k],
    Re(d_i) / ds, <jk||jk> / gs, (<jb||jb> + <kb||kb>) / gs and
    |<jb||jb> - <kb||kb>| / gs, with c the first-order component
    -W_ibjk / (d_i - d_nu) and d the IP diagonal (``ipeom.diagonal``); the
    scales are those of ``features``. ``H`` is ``ipeom.hbar``'s dict, ``g``
    the integral blocks."""
    from .ipeom import diagonal
    o = n_occ
    v = len(eps) - o
    d = diagonal(H, o, v)
    iu = [(i, j) for i in range(o) for j in range(i + 1, o)]
    gs = np.sqrt(np.mean([g.oooo[i, j, i, j].real ** 2 for i, j in iu]))
    ds = 2.0 * (np.sum(eps[o:]) - np.sum(eps[:o])) / (o + v)
    dia = np.array([[g.ovov[i, a, i, a].real for a in range(v)] for i in range(o)])
    i = seed
    out = np.empty((n, F))
    k = 0
    for p, (j, kk) in enumerate(iu):
        for b in range(v):
            if k == n:
                return out
            nu = o + p * v + b
            w = -H["ovoo"][i, b, j, kk]
            c = w / (d[i] - d[nu])
            out[k] = [np.log10(abs(c) + 1e-30), (d[i] - d[nu]).real / ds, abs(w) / gs,
                      1.0 if i in (j, kk) else 0.0, d[i].real / ds,
                      g.oooo[j, kk, j, kk].real / gs, (dia[j, b] + dia[kk, b]) / gs,
                      abs(dia[j, b] - dia[kk, b]) / gs]
            k += 1
    return out[:k]
