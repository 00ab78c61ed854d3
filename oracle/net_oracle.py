"""FP64 NumPy oracle of the learned SOR warm-start network.

TEST INFRASTRUCTURE ONLY: the reference the GPU network's forward pass and
gradients are checked against.  Only tests/ (and smoke / bench CPU legs) use it.

The network (the paper has no learned part; this is the warm start the library
adds): bias-free 3x3x3 convolutions with zero padding on NDHWC arrays,
  e0 = relu(c0(x)), e1 = relu(c1(pool e0)), e2 = relu(c2(pool e1)),
  e3 = relu(c3(pool e2)), d2 = relu(c4(up e3)) + e2, d1 = relu(c5(up d2)) + e1,
  d0 = relu(c6(up d1)) + e0, y = mask * (d0 . w_head)
with pool the 2x2x2 mean (children outside the grid count as zero) and up the
nearest-neighbour copy.  Input x: channel 0 = mask * r / rms_mask(r), channel 1
= mask, channels 2..15 zero.  Loss: mean over the batch of
mean_mask (y - t / rms_mask(t))^2.

With an input stride s the sample is first pooled s times per axis (block
means, cells outside the grid counting as zero), the network runs on the coarse
grid, and its output is prolongated to the fine cells by trilinear
interpolation between coarse cell centres and masked.

Pins (tests/test_oracle_net.py): the convolution equals scipy.signal's
correlation channel by channel, pool/up are adjoint to their backward
maps, the full gradient matches central finite differences, strided pooling
reduces to the 2x2x2 pool and preserves block means, and the prolongation
reproduces constants everywhere and linear functions away from the clamped
boundary cells.
"""

from __future__ import annotations

import numpy as np

CIN = [16, 16, 32, 64, 128, 64, 32]
COUT = [16, 32, 64, 128, 64, 32, 16]
HEAD = 16


def unflatten(theta):
    """Flat parameter vector -> list of conv weights [27][Cout][Cin] and head [16]."""
    ws, o = [], 0
    for ci, co in zip(CIN, COUT):
        n = 27 * co * ci
        ws.append(np.asarray(theta[o:o + n], np.float64).reshape(27, co, ci))
        o += n
    head = np.asarray(theta[o:o + HEAD], np.float64)
    return ws, head


def flatten(ws, head):
    return np.concatenate([w.ravel() for w in ws] + [head.ravel()])


# ---------------------------------------------------------------------------
# primitives (arrays are [Z, Y, X, C])

def conv3(x, w):
    """y[z,y,x,o] = sum_tap sum_c w[tap,o,c] x[z+dz-1, y+dy-1, x+dx-1, c], zero padded."""
    Z, Y, X, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((Z, Y, X, w.shape[1]))
    for tap in range(27):
        dx, dy, dz = tap % 3, (tap // 3) % 3, tap // 9
        y += xp[dz:dz + Z, dy:dy + Y, dx:dx + X, :] @ w[tap].T
    return y


def conv3_bwd(x, w, gy):
    """Gradients of conv3 w.r.t. its input and weights."""
    Z, Y, X, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for tap in range(27):
        dx, dy, dz = tap % 3, (tap // 3) % 3, tap // 9
        sl = (slice(dz, dz + Z), slice(dy, dy + Y), slice(dx, dx + X))
        gxp[sl] += gy @ w[tap]
        gw[tap] = np.einsum("zyxo,zyxc->oc", gy, xp[sl])
    return gxp[1:-1, 1:-1, 1:-1], gw


def pool(a):
    Z, Y, X, C = a.shape
    ap = np.pad(a, ((0, Z % 2), (0, Y % 2), (0, X % 2), (0, 0)))
    Zc, Yc, Xc = ap.shape[0] // 2, ap.shape[1] // 2, ap.shape[2] // 2
    return ap.reshape(Zc, 2, Yc, 2, Xc, 2, C).sum(axis=(1, 3, 5)) / 8.0


def pool_bwd(g, shape):
    Z, Y, X, C = shape
    up_ = np.repeat(np.repeat(np.repeat(g, 2, 0), 2, 1), 2, 2) / 8.0
    return up_[:Z, :Y, :X]


def up(b, shape):
    Z, Y, X, _ = shape
    return np.repeat(np.repeat(np.repeat(b, 2, 0), 2, 1), 2, 2)[:Z, :Y, :X]


def up_bwd(g, cshape):
    Zc, Yc, Xc, C = cshape
    Z, Y, X, _ = g.shape
    gp = np.pad(g, ((0, 2 * Zc - Z), (0, 2 * Yc - Y), (0, 2 * Xc - X), (0, 0)))
    return gp.reshape(Zc, 2, Yc, 2, Xc, 2, C).sum(axis=(1, 3, 5))


def relu(a):
    return np.maximum(a, 0.0)


def rms(a, mask):
    m = mask.sum()
    return np.sqrt((mask * a * a).sum() / m) if m > 0 else 0.0


def pack(r, mask):
    s = rms(r, mask)
    x = np.zeros(r.shape + (16,))
    x[..., 0] = mask * r / s if s > 0 else 0.0
    x[..., 1] = mask
    return x


# ---------------------------------------------------------------------------

def forward(theta, r, mask):
    """One sample r, mask [Z, Y, X] -> y [Z, Y, X] and the activations."""
    ws, head = unflatten(theta)
    x = pack(r, mask)
    A = {"x": x}
    A["e0"] = relu(conv3(x, ws[0]))
    A["p0"] = pool(A["e0"])
    A["e1"] = relu(conv3(A["p0"], ws[1]))
    A["p1"] = pool(A["e1"])
    A["e2"] = relu(conv3(A["p1"], ws[2]))
    A["p2"] = pool(A["e2"])
    A["e3"] = relu(conv3(A["p2"], ws[3]))
    A["u2"] = up(A["e3"], A["e2"].shape[:3] + (128,))
    A["r2"] = relu(conv3(A["u2"], ws[4]))
    A["d2"] = A["r2"] + A["e2"]
    A["u1"] = up(A["d2"], A["e1"].shape[:3] + (64,))
    A["r1"] = relu(conv3(A["u1"], ws[5]))
    A["d1"] = A["r1"] + A["e1"]
    A["u0"] = up(A["d1"], A["e0"].shape[:3] + (32,))
    A["r0"] = relu(conv3(A["u0"], ws[6]))
    A["d0"] = A["r0"] + A["e0"]
    y = mask * (A["d0"] @ head)
    return y, A


def loss_and_grad(theta, rs, masks, ts):
    """Batch loss and its gradient (flat, same layout as theta)."""
    ws, head = unflatten(theta)
    gws = [np.zeros_like(w) for w in ws]
    ghead = np.zeros_like(head)
    B = len(rs)
    L = 0.0
    for r, mask, t in zip(rs, masks, ts):
        y, A = forward(theta, r, mask)
        st = rms(t, mask)
        tn = t / st if st > 0 else np.zeros_like(t)
        n = mask.sum()
        e = mask * (y - tn)
        L += (e * e).sum() / (n * B)
        gy = 2.0 * e / (n * B)
        gym = gy * mask
        ghead += np.einsum("zyx,zyxc->c", gym, A["d0"])
        gd0 = gym[..., None] * head[None, None, None, :]
        # d0 = relu(c6(u0)) + e0
        g = gd0 * (A["r0"] > 0)
        gu0, gw6 = conv3_bwd(A["u0"], ws[6], g)
        gws[6] += gw6
        gd1 = up_bwd(gu0, A["d1"].shape)
        g = gd1 * (A["r1"] > 0)
        gu1, gw5 = conv3_bwd(A["u1"], ws[5], g)
        gws[5] += gw5
        gd2 = up_bwd(gu1, A["d2"].shape)
        g = gd2 * (A["r2"] > 0)
        gu2, gw4 = conv3_bwd(A["u2"], ws[4], g)
        gws[4] += gw4
        ge3 = up_bwd(gu2, A["e3"].shape)
        g = ge3 * (A["e3"] > 0)
        gp2, gw3 = conv3_bwd(A["p2"], ws[3], g)
        gws[3] += gw3
        ge2 = gd2 + pool_bwd(gp2, A["e2"].shape)
        g = ge2 * (A["e2"] > 0)
        gp1, gw2 = conv3_bwd(A["p1"], ws[2], g)
        gws[2] += gw2
        ge1 = gd1 + pool_bwd(gp1, A["e1"].shape)
        g = ge1 * (A["e1"] > 0)
        gp0, gw1 = conv3_bwd(A["p0"], ws[1], g)
        gws[1] += gw1
        ge0 = gd0 + pool_bwd(gp0, A["e0"].shape)
        g = ge0 * (A["e0"] > 0)
        _, gw0 = conv3_bwd(A["x"], ws[0], g)
        gws[0] += gw0
    return L, flatten(gws, ghead)


def loss(theta, rs, masks, ts):
    B = len(rs)
    L = 0.0
    for r, mask, t in zip(rs, masks, ts):
        y, _ = forward(theta, r, mask)
        st = rms(t, mask)
        tn = t / st if st > 0 else np.zeros_like(t)
        e = mask * (y - tn)
        L += (e * e).sum() / (mask.sum() * B)
    return L


# ---------------------------------------------------------------------------
# input stride: the network runs on the grid coarsened s times per axis

def pool_s(a, s):
    """Block sums over s x s x s fine cells / s^3 (cells outside the grid count as zero)."""
    Z, Y, X = a.shape
    ap = np.pad(a, ((0, -Z % s), (0, -Y % s), (0, -X % s)))
    Zc, Yc, Xc = ap.shape[0] // s, ap.shape[1] // s, ap.shape[2] // s
    return ap.reshape(Zc, s, Yc, s, Xc, s).sum(axis=(1, 3, 5)) / float(s ** 3)


def interp_matrix(n_fine, s):
    """1-D linear interpolation from coarse cell centres to fine cell centres:
    fine centre f is at coarse coordinate (f + 1/2)/s - 1/2, clamped to the
    first / last coarse centre."""
    C = -(-n_fine // s)
    P = np.zeros((n_fine, C))
    for f in range(n_fine):
        x = (f + 0.5) / s - 0.5
        c0 = int(np.floor(x))
        w = x - c0
        if c0 < 0:
            c0, w = 0, 0.0
        if c0 >= C - 1:
            c0, w = C - 1, 0.0
        P[f, c0] += 1.0 - w
        if w > 0.0:
            P[f, c0 + 1] += w
    return P


def prolong(yc, shape, s):
    """Trilinear prolongation of a coarse [Zc, Yc, Xc] field to the fine shape."""
    Pz, Py, Px = (interp_matrix(n, s) for n in shape)
    return np.einsum("zc,yb,xa,cba->zyx", Pz, Py, Px, yc)


def forward_strided(theta, r, mask, s):
    """The network on the pooled sample, prolongated and masked on the fine grid."""
    yc, _ = forward(theta, pool_s(r, s), pool_s(mask, s))
    return mask * prolong(yc, r.shape, s)


def loss_and_grad_strided(theta, rs, masks, ts, s):
    """Training at the coarse level against the pooled targets."""
    return loss_and_grad(theta, [pool_s(r, s) for r in rs], [pool_s(m, s) for m in masks],
                         [pool_s(t, s) for t in ts])


def init_params(seed):
    """He-normal parameters (for tests that do not start from the GPU net)."""
    rng = np.random.default_rng(seed)
    ws = [rng.standard_normal((27, co, ci)) * np.sqrt(2.0 / (27.0 * (2 if k == 0 else ci)))
          for k, (ci, co) in enumerate(zip(CIN, COUT))]
    head = rng.standard_normal(HEAD) * np.sqrt(1.0 / HEAD)
    return flatten(ws, head)
