"""3-level U-Net preconditioner, FP64 numpy forward and backward (TEST
INFRASTRUCTURE).  The network is not in the paper; it is the learned
preconditioner for the implicit (I + dt A) solve.

Architecture (channels c1, c2, c3 = 16, 32, 64 by default, input Cin):
    enc1: conv3x3(Cin->c1) ReLU, conv3x3(c1->c1) ReLU           -> s1  (H x W)
    avgpool 2x2
    enc2: conv3x3(c1->c2) ReLU, conv3x3(c2->c2) ReLU            -> s2  (H/2)
    avgpool 2x2
    mid : conv3x3(c2->c3) ReLU, conv3x3(c3->c3) ReLU                   (H/4)
    nearest upsample x2, concat [up, s2]
    dec2: conv3x3(c3+c2->c2) ReLU, conv3x3(c2->c2) ReLU                (H/2)
    nearest upsample x2, concat [up, s1]
    dec1: conv3x3(c2+c1->c1) ReLU, conv3x3(c1->c1) ReLU                (H)
    out : conv1x1(c1->1)
3x3 convolutions are cross-correlations with zero padding ("same").  The
parameters live in one flat vector: for each layer in the order above, the
weights [co][ci][ky][kx] followed by the bias [co].
"""
import numpy as np

LAYERS = ["enc1a", "enc1b", "enc2a", "enc2b", "mid_a", "mid_b", "dec2a", "dec2b", "dec1a",
          "dec1b", "out"]


def layer_shapes(cin, c1=16, c2=32, c3=64):
    """(name, co, ci, k) for each layer, in parameter order."""
    return [("enc1a", c1, cin, 3), ("enc1b", c1, c1, 3),
            ("enc2a", c2, c1, 3), ("enc2b", c2, c2, 3),
            ("mid_a", c3, c2, 3), ("mid_b", c3, c3, 3),
            ("dec2a", c2, c3 + c2, 3), ("dec2b", c2, c2, 3),
            ("dec1a", c1, c2 + c1, 3), ("dec1b", c1, c1, 3),
            ("out", 1, c1, 1)]


def n_params(cin, **kw):
    return sum(co * ci * k * k + co for _, co, ci, k in layer_shapes(cin, **kw))


def unpack(theta, cin, **kw):
    """Flat vector -> {name: (W[co,ci,k,k], b[co])} (views)."""
    out, o = {}, 0
    for name, co, ci, k in layer_shapes(cin, **kw):
        nw = co * ci * k * k
        W = theta[o:o + nw].reshape(co, ci, k, k)
        o += nw
        b = theta[o:o + co]
        o += co
        out[name] = (W, b)
    assert o == theta.size
    return out


def init_params(cin, seed, **kw):
    """He-normal weights (std sqrt(2 / (ci k^2))), zero biases."""
    g = np.random.default_rng(seed)
    parts = []
    for _, co, ci, k in layer_shapes(cin, **kw):
        parts.append(g.normal(0.0, np.sqrt(2.0 / (ci * k * k)), co * ci * k * k))
        parts.append(np.zeros(co))
    return np.concatenate(parts)


# ---------------------------------------------------------------- primitives
def conv(x, W, b):
    """y[o,i,j] = b[o] + sum_c sum_{dy,dx} W[o,c,dy,dx] x[c, i+dy-r, j+dx-r]."""
    co, ci, k, _ = W.shape
    r = k // 2
    C, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (r, r), (r, r)))
    y = np.zeros((co, H, Wd)) + b[:, None, None]
    for dy in range(k):
        for dx in range(k):
            patch = xp[:, dy:dy + H, dx:dx + Wd]                  # (ci, H, W)
            y += np.tensordot(W[:, :, dy, dx], patch, axes=([1], [0]))
    return y


def conv_backward(x, W, gy):
    """Gradients of conv: returns (gx, gW, gb)."""
    co, ci, k, _ = W.shape
    r = k // 2
    C, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (r, r), (r, r)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for dy in range(k):
        for dx in range(k):
            patch = xp[:, dy:dy + H, dx:dx + Wd]
            gW[:, :, dy, dx] = np.tensordot(gy, patch, axes=([1, 2], [1, 2]))
            gxp[:, dy:dy + H, dx:dx + Wd] += np.tensordot(W[:, :, dy, dx], gy, axes=([0], [0]))
    gb = gy.sum(axis=(1, 2))
    return gxp[:, r:r + H, r:r + Wd], gW, gb


def pool(x):
    C, H, W = x.shape
    return x.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def pool_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) * 0.25


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(gy):
    C, H, W = gy.shape
    return gy.reshape(C, H // 2, 2, W // 2, 2).sum(axis=(2, 4))


# ---------------------------------------------------------------- network
def forward(theta, x, cin=None, **kw):
    """x: (Cin, H, W), H and W divisible by 4.  Returns (y (H, W), cache)."""
    cin = x.shape[0] if cin is None else cin
    P = unpack(theta, cin, **kw)
    cache = {"x": x}

    def cr(name, inp):
        pre = conv(inp, *P[name])
        cache[name] = (inp, pre)
        return np.maximum(pre, 0.0)

    a = cr("enc1b", cr("enc1a", x))
    s1 = a
    a = cr("enc2b", cr("enc2a", pool(s1)))
    s2 = a
    a = cr("mid_b", cr("mid_a", pool(s2)))
    a = np.concatenate([up(a), s2], axis=0)
    a = cr("dec2b", cr("dec2a", a))
    a = np.concatenate([up(a), s1], axis=0)
    a = cr("dec1b", cr("dec1a", a))
    y = conv(a, *P["out"])
    cache["out"] = (a, y)
    return y[0], cache


def backward(theta, cache, gy, cin=None, **kw):
    """Gradient of <gy, forward(theta, x)> w.r.t. theta (flat) and x."""
    x = cache["x"]
    cin = x.shape[0] if cin is None else cin
    P = unpack(theta, cin, **kw)
    grads = {}
    shapes = {n: (co, ci) for n, co, ci, _ in layer_shapes(cin, **kw)}

    a_in, _ = cache["out"]
    g, gW, gb = conv_backward(a_in, P["out"][0], gy[None])
    grads["out"] = (gW, gb)

    def br(name, g):
        inp, pre = cache[name]
        g = g * (pre > 0)
        gi, gW, gb = conv_backward(inp, P[name][0], g)
        grads[name] = (gW, gb)
        return gi

    g = br("dec1a", br("dec1b", g))
    c1 = shapes["enc1a"][0]
    g_up, g_s1 = g[:-c1], g[-c1:]
    g = up_backward(g_up)
    g = br("dec2a", br("dec2b", g))
    c2 = shapes["enc2a"][0]
    g_up, g_s2 = g[:-c2], g[-c2:]
    g = up_backward(g_up)
    g = br("mid_a", br("mid_b", g))
    g = pool_backward(g) + g_s2
    g = br("enc2a", br("enc2b", g))
    g = pool_backward(g) + g_s1
    gx = br("enc1a", br("enc1b", g))

    flat = []
    for name, co, ci, k in layer_shapes(cin, **kw):
        gW, gb = grads[name]
        flat.append(gW.ravel())
        flat.append(gb)
    return np.concatenate(flat), gx


# ---------------------------------------------------------------- preconditioner
# The network is used as the coarse part of a preconditioner M for
# (I + dt A) x = b:  M(r) = r / d + s * P(N(F(r))), where d = 1 + dt A_zz
# (Jacobi part), s = rms(r), P repeats a coarse value over its RF x RF block,
# and F(r) are the coarse input channels: the RF^2 values of r / s in each
# block (space to depth, channel dy * RF + dx) followed by the block means of
# log(1 + dt w_k) for the three canonical half-stencil weights and of the
# three canonical offsets / 8.
RF = 4
N_STATIC = 9
N_FEATURES = RF * RF + N_STATIC


def restrict(f, rf=RF):
    C, H, W = f.shape
    return f.reshape(C, H // rf, rf, W // rf, rf).mean(axis=(2, 4))


def space_to_depth(a, rf=RF):
    H, W = a.shape
    return a.reshape(H // rf, rf, W // rf, rf).transpose(1, 3, 0, 2).reshape(rf * rf, H // rf, W // rf)


def prolong(y, rf=RF):
    return np.repeat(np.repeat(y, rf, axis=-2), rf, axis=-1)


def coarse_features(offs, w, dt, r):
    """F(r) [N_FEATURES, H/RF, W/RF] and s = rms(r)."""
    shape = r.shape
    s = float(np.sqrt(np.mean(np.asarray(r, np.float64) ** 2)))
    st = np.zeros((N_STATIC,) + shape)
    for k in range(3):
        st[k] = np.log1p(dt * w[:, k]).reshape(shape)
        st[3 + 2 * k] = (offs[:, k, 0] / 8.0).reshape(shape)
        st[4 + 2 * k] = (offs[:, k, 1] / 8.0).reshape(shape)
    rs = r / s if s > 0 else np.zeros(shape)
    return np.concatenate([space_to_depth(rs), restrict(st)]), s


def precondition(theta, offs, w, dt, diag, r, **kw):
    """z = M(r) (see above); diag = A_zz."""
    f, s = coarse_features(offs, w, dt, r)
    if s == 0.0:
        return np.zeros_like(r)
    y, _ = forward(theta, f, **kw)
    return r / (1.0 + dt * diag) + s * prolong(y)


def training_target(offs, w, dt, diag, r, e):
    """What the network should output for residual r with error e:
    R((e - r / d) / s)."""
    s = float(np.sqrt(np.mean(np.asarray(r, np.float64) ** 2)))
    return restrict(((e - r / (1.0 + dt * diag)) / s)[None])[0]
