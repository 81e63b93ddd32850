"""Plain FP64 CPU reference of the learned interpolation weights (test infrastructure only).

A small network maps each finest-level coarse edge's local problem to the values of its column of
P on the patch (the interior part of Eq. sparseP), in place of the exact local solve.  Only the
test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it.

Definitions (the library implements the same ones independently):
  * slog(v) = sign(v) log(1 + |v|).
  * For coarse edge c with exterior pair (d1, s1), (d2, s2) and sorted patch p (at most M_IN DoFs),
    with a = A[d1, d1]:  for slot q < |p|, g = p[q]:
        feat[3q]     = slog(A[g, g] / a)
        feat[3q + 1] = slog(-(A[g, d1] s1 + A[g, d2] s2) / a)      (the local right-hand side)
        feat[3q + 2] = slog(sum_{h in p, h != g} |A[g, h]| / a)     (coupling inside the patch)
    unused slots are 0; feat[3 M_IN] = |p| / M_IN, feat[3 M_IN + 1] = slog(A[d2, d2] / a).
  * Target: the exact local solution x_c of Eq. sparseP on the patch (slot q), mask 1 on used slots.
  * Network: h1 = relu(X W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3 (width 64).
  * Loss: sum over the batch of sum_q mask (y - t)^2, divided by the number of used slots.
  * Adam (Kingma and Ba, 2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected.
  * BF16 storage (precision="bf16"): the network's inputs, the weight matrices W1, W2, W3 and the
    hidden activations h1, h2 are held as bfloat16 (each the float32 value rounded to the nearest
    bfloat16, ties to even); biases, pre-activations, outputs, gradients and the Adam state stay at
    full precision, and the gradients are taken with the stored (rounded) operands.  The FP32
    master weights are what Adam updates.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

M_IN = 64
D_IN = 3 * M_IN + 2
WIDTH = 64


def slog(v):
    return np.sign(v) * np.log1p(np.abs(v))


def patch_features(A, edge, patch, m_in=M_IN):
    """Feature vector (3 m_in + 2) and slot mask (m_in) of one coarse edge."""
    A = sp.csr_matrix(A)
    d1, s1, d2, s2 = edge[0], edge[1], edge[2], edge[3]
    a = A[d1, d1]
    f = np.zeros(3 * m_in + 2)
    mask = np.zeros(m_in)
    pset = set(int(g) for g in patch)
    for q, g in enumerate(patch[:m_in]):
        row = A.getrow(g)
        cols, vals = row.indices, row.data
        f[3 * q] = slog(A[g, g] / a)
        f[3 * q + 1] = slog(-(A[g, d1] * s1 + A[g, d2] * s2) / a)
        f[3 * q + 2] = slog(sum(abs(v) for c, v in zip(cols, vals) if c in pset and c != g) / a)
        mask[q] = 1.0
    f[3 * m_in] = len(patch) / m_in
    f[3 * m_in + 1] = slog(A[d2, d2] / a)
    return f, mask


def patch_target(A, edge, patch, m_in=M_IN):
    """Exact local solution of Eq. sparseP on the patch, padded to m_in slots."""
    A = sp.csr_matrix(A)
    d1, s1, d2, s2 = edge[0], edge[1], edge[2], edge[3]
    t = np.zeros(m_in)
    if len(patch):
        App = A[patch][:, patch].toarray()
        rhs = A[patch][:, [d1]].toarray().ravel() * s1 + A[patch][:, [d2]].toarray().ravel() * s2
        t[:len(patch)] = -sla.cho_solve(sla.cho_factor(App, lower=True), rhs)
    return t


def init_params(u01, d_in=D_IN, width=WIDTH, d_out=M_IN):
    """Glorot-uniform weights from a stream of U(0,1) draws (consumed in the order W1, W2, W3);
    zero biases.  u01(count, offset) -> array."""
    shapes = [(d_in, width), (width, width), (width, d_out)]
    params, off = [], 0
    for (fi, fo) in shapes:
        lim = np.sqrt(6.0 / (fi + fo))
        w = (2.0 * u01(fi * fo, off) - 1.0) * lim
        off += fi * fo
        params += [w.reshape(fi, fo), np.zeros(fo)]
    return params


def to_bf16(x):
    """The nearest bfloat16 (ties to even) of x's float32 rounding, as a float64 array: a bfloat16
    is the upper 16 bits of a float32, so the float32 bit pattern is rounded at bit 16."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _storage(precision):
    if precision == "fp32":
        return lambda v: v
    if precision == "bf16":
        return to_bf16
    raise ValueError("precision must be 'fp32' or 'bf16'")


def forward(params, X, precision="fp32"):
    """y and the stored intermediates (X, z1, h1, z2, h2, W1, W2, W3 as the products used them)."""
    q = _storage(precision)
    W1, b1, W2, b2, W3, b3 = params
    X, W1, W2, W3 = q(X), q(W1), q(W2), q(W3)
    z1 = X @ W1 + b1
    h1 = q(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + b2
    h2 = q(np.maximum(z2, 0.0))
    y = h2 @ W3 + b3
    return y, (X, z1, h1, z2, h2, W1, W2, W3)


def loss(params, X, T, M, precision="fp32"):
    y, _ = forward(params, X, precision)
    return float(((y - T) ** 2 * M).sum() / max(M.sum(), 1.0))


def backward(params, X, T, M, precision="fp32"):
    """Loss and the gradients of every parameter (the chain rule written out by hand), taken with
    the operands as stored."""
    y, (X, z1, h1, z2, h2, W1, W2, W3) = forward(params, X, precision)
    nrm = max(M.sum(), 1.0)
    L = float(((y - T) ** 2 * M).sum() / nrm)
    dy = 2.0 * (y - T) * M / nrm
    gW3 = h2.T @ dy
    gb3 = dy.sum(axis=0)
    dh2 = dy @ W3.T
    dz2 = dh2 * (z2 > 0)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * (z1 > 0)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(axis=0)
    return L, [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(params, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of every parameter (t = 1, 2, ...); state holds the moment estimates."""
    if not state:
        state.extend([[np.zeros_like(p), np.zeros_like(p)] for p in params])
    out = []
    for p, g, st in zip(params, grads, state):
        st[0] = b1 * st[0] + (1 - b1) * g
        st[1] = b2 * st[1] + (1 - b2) * g * g
        mh = st[0] / (1 - b1 ** t)
        vh = st[1] / (1 - b2 ** t)
        out.append(p - lr * mh / (np.sqrt(vh) + eps))
    return out


def learned_interpolation(A, edges, patches, ndof, params):
    """Eq. sparseP's pattern with the interior values predicted by the network: column c is s1 at
    DoF1, s2 at DoF2 and forward(features of c)[q] at the patch's q-th DoF."""
    rows, cols, vals = [], [], []
    for c, (e, p) in enumerate(zip(edges, patches)):
        rows += [e[0], e[2]]
        cols += [c, c]
        vals += [e[1], e[3]]
        if len(p):
            f, _ = patch_features(A, e, p)
            y, _ = forward(params, f[None, :])
            rows += list(p)
            cols += [c] * len(p)
            vals += y[0, :len(p)].tolist()
    P = sp.csr_matrix((vals, (rows, cols)), shape=(ndof, len(edges)))
    P.sort_indices()
    return P


def setup_learned(A, G, params, **kw):
    """Hierarchy whose finest P comes from the network (the coarser levels use the exact local
    solves), built with the oracle's own coarsening and Galerkin product."""
    from . import amg as O
    A = sp.csr_matrix(A)
    A.sort_indices()
    H0 = O.smoother_level(A, G)
    H0["G"] = sp.csr_matrix(G)
    cz = O.coarsen(A, G, **{k: v for k, v in kw.items() if k in ("p_max", "ring", "strength", "theta")})
    P = learned_interpolation(A, cz["edges"], cz["patches"], A.shape[0], params)
    H0["coarsening"] = cz
    H0["P"] = P
    return [H0] + O.setup(O.galerkin(A, P), cz["Gc"], **kw)
