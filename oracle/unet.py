"""FP64 3D-conv U-Net for the learned pressure preconditioner (forward, backward).

Test infrastructure (see ``oracle/__init__``).

The paper (arXiv:1404.0959) solves a pressure-correction equation in every
PISO corrector (Sec. 2 par. 1) but says nothing about learning; the network
is this project's extension: a 3-level U-Net on the periodic grid whose output
is used as a search direction inside flexible CG.  Layers (3x3x3 kernels,
periodic padding, ReLU after every layer but the last):

  e1a: Cin->16, e1b: 16->16                       (N^3)       -> skip s1
  d1 : 16->32, stride 2; e2: 32->32               ((N/2)^3)   -> skip s2
  d2 : 32->64, stride 2; e3: 64->64               ((N/4)^3)
  u2 : [up2(e3), s2] 96->32                       ((N/2)^3)
  u1 : [up2(u2), s1] 48->16                       (N^3)
  out: 16->1 (linear)                             (N^3)

up2 = nearest-neighbour upsampling by 2 per axis; [a, b] = channel concat.
A stride-2 convolution is the stride-1 convolution sampled at even cells.
Convolution (definition): y[co](v) = b[co] + sum_{t in {-1,0,1}^3} sum_ci
W[t, ci, co] x[ci](v + t), periodic.  Arrays: (C, N, N, N), [z, y, x].

Preconditioner (residual form).  The pressure-correction operator of the
PISO corrector (Sec. 2 par. 1) is M = diag(psi/dt) - dt/2 D(G2 .), whose
Jacobi diagonal is d = psi/dt + 3 dt/h^2.  For a residual r the network
corrects the Jacobi direction r/d instead of replacing it:

  rho   = rms(r) = sqrt(mean(r^2));  d0 = 1 / (1/dt + 3 dt/h^2)  (d at psi = 1)
  input = [ (r/d) / (rho d0),  (3 dt/h^2) / d ]   (second channel in (0, 1):
          the share of the diagonal that comes from the Laplacian, i.e. six
          times the Jacobi neighbour weight; it carries dt and psi)
  z     = r/d + rho d0 net(input)

so that a network whose last layer is zero is exactly Jacobi, and z scales
with r.  A training pair (r, e) with M e = r has the target
t = (e - r/d) / (rho d0): the part of M^{-1} r that Jacobi misses, in the
same units as the network output; loss ||y - t||^2 / ||t||^2.

Parity pins (tests/test_oracle_unet.py): the convolution against a brute
force loop on a tiny grid; every parameter and input gradient against
centred finite differences; translation equivariance; a zero last layer
gives the Jacobi direction; the direction of the exact correction target
solves M z = r; direction and input scale with r.
"""
import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]

# (name, cin, cout, stride) in forward order; cin of u2/u1 are concat widths
LAYERS = [("e1a", None, 16, 1), ("e1b", 16, 16, 1), ("d1", 16, 32, 2), ("e2", 32, 32, 1),
          ("d2", 32, 64, 2), ("e3", 64, 64, 1), ("u2", 96, 32, 1), ("u1", 48, 16, 1), ("out", 16, 1, 1)]


def shift(x, t):
    """x(v + t) for every v (periodic); x has shape (C, N, N, N) or (N, N, N)."""
    dz, dy, dx = t
    return np.roll(x, (-dz, -dy, -dx), axis=(-3, -2, -1))


def conv(x, W, b, stride=1):
    """W: (27, Cin, Cout) indexed by TAPS order; b: (Cout,)."""
    cout = W.shape[2]
    y = np.zeros((cout,) + x.shape[1:])
    for ti, t in enumerate(TAPS):
        xs = shift(x, t)
        y += np.einsum("ic,i...->c...", W[ti], xs)
    y += b[:, None, None, None]
    if stride == 2:
        y = y[:, ::2, ::2, ::2]
    return y


def conv_backward(x, W, dy, stride=1):
    """Gradients of conv w.r.t. x, W, b given dy (shape of the conv output)."""
    if stride == 2:
        full = np.zeros((dy.shape[0],) + x.shape[1:])
        full[:, ::2, ::2, ::2] = dy
        dy = full
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for ti, t in enumerate(TAPS):
        xs = shift(x, t)
        dW[ti] = np.einsum("izyx,czyx->ic", xs, dy)
        # y(v) gets W x(v + t): x(w) contributes to y(w - t)
        dx += np.einsum("ic,c...->i...", W[ti], shift(dy, (-t[0], -t[1], -t[2])))
    db = dy.sum(axis=(1, 2, 3))
    return dx, dW, db


def up2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def up2_backward(dy):
    C, N = dy.shape[0], dy.shape[1] // 2
    return dy.reshape(C, N, 2, N, 2, N, 2).sum(axis=(2, 4, 6))


def relu(x):
    return np.maximum(x, 0.0)


def init_params(cin, seed=0):
    """He-style random weights (input generator for tests; training sets its own)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co, _s in LAYERS:
        ci = cin if ci is None else ci
        std = np.sqrt(2.0 / (27 * ci))
        P[name + ".W"] = rng.standard_normal((27, ci, co)) * std
        P[name + ".b"] = rng.standard_normal(co) * 0.01
    return P


def forward(P, x):
    """x: (Cin, N, N, N).  Returns (output (1, N, N, N), cache)."""
    c = {"x": x}
    c["e1a"] = relu(conv(x, P["e1a.W"], P["e1a.b"]))
    c["e1b"] = relu(conv(c["e1a"], P["e1b.W"], P["e1b.b"]))
    c["d1"] = relu(conv(c["e1b"], P["d1.W"], P["d1.b"], 2))
    c["e2"] = relu(conv(c["d1"], P["e2.W"], P["e2.b"]))
    c["d2"] = relu(conv(c["e2"], P["d2.W"], P["d2.b"], 2))
    c["e3"] = relu(conv(c["d2"], P["e3.W"], P["e3.b"]))
    c["u2in"] = np.concatenate([up2(c["e3"]), c["e2"]], axis=0)
    c["u2"] = relu(conv(c["u2in"], P["u2.W"], P["u2.b"]))
    c["u1in"] = np.concatenate([up2(c["u2"]), c["e1b"]], axis=0)
    c["u1"] = relu(conv(c["u1in"], P["u1.W"], P["u1.b"]))
    y = conv(c["u1"], P["out.W"], P["out.b"])
    return y, c


def backward(P, c, dy):
    """Gradients of a scalar loss given dy = dL/d(output).  Returns (grads, dx)."""
    G = {}
    d, G["out.W"], G["out.b"] = conv_backward(c["u1"], P["out.W"], dy)
    d = d * (c["u1"] > 0)
    d, G["u1.W"], G["u1.b"] = conv_backward(c["u1in"], P["u1.W"], d)
    d_u2 = up2_backward(d[:32])
    d_e1b_skip = d[32:]
    d = d_u2 * (c["u2"] > 0)
    d, G["u2.W"], G["u2.b"] = conv_backward(c["u2in"], P["u2.W"], d)
    d_e3 = up2_backward(d[:64])
    d_e2_skip = d[64:]
    d = d_e3 * (c["e3"] > 0)
    d, G["e3.W"], G["e3.b"] = conv_backward(c["d2"], P["e3.W"], d)
    d = d * (c["d2"] > 0)
    d, G["d2.W"], G["d2.b"] = conv_backward(c["e2"], P["d2.W"], d, 2)
    d = (d + d_e2_skip) * (c["e2"] > 0)
    d, G["e2.W"], G["e2.b"] = conv_backward(c["d1"], P["e2.W"], d)
    d = d * (c["d1"] > 0)
    d, G["d1.W"], G["d1.b"] = conv_backward(c["e1b"], P["d1.W"], d, 2)
    d = (d + d_e1b_skip) * (c["e1b"] > 0)
    d, G["e1b.W"], G["e1b.b"] = conv_backward(c["e1a"], P["e1b.W"], d)
    d = d * (c["e1a"] > 0)
    dx, G["e1a.W"], G["e1a.b"] = conv_backward(c["x"], P["e1a.W"], d)
    return G, dx


def loss_rel_mse(y, target):
    """||y - t||^2 / ||t||^2 and its gradient w.r.t. y."""
    tt = float(np.sum(target * target))
    diff = y - target
    return float(np.sum(diff * diff)) / tt, 2.0 * diff / tt


def adam_update(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma and Ba 2015) with bias correction; returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def jacobi_diag(psi, dt, h):
    """Diagonal of M = diag(psi/dt) - dt/2 D(G2 .): psi/dt + 3 dt/h^2."""
    return psi / dt + 3.0 * dt / (h * h)


def precond_scales(r, dt, h):
    """(rho, d0): r.m.s. of r and the Jacobi inverse of the uniform state psi = 1."""
    rho = float(np.sqrt(np.mean(r * r)))
    d0 = 1.0 / (1.0 / dt + 3.0 * dt / (h * h))
    return rho, d0


def network_input(r, psi, dt, h):
    """The two input channels: Jacobi direction r/d over rho d0, and (3 dt/h^2)/d."""
    d = jacobi_diag(psi, dt, h)
    rho, d0 = precond_scales(r, dt, h)
    s = (r / d) / (rho * d0) if rho > 0.0 else np.zeros_like(r)
    w = (3.0 * dt / (h * h)) / d
    return np.stack([s, w])


def direction(P, r, psi, dt, h):
    """Preconditioned direction z = r/d + rho d0 net(input) for residual r."""
    d = jacobi_diag(psi, dt, h)
    rho, d0 = precond_scales(r, dt, h)
    if rho == 0.0:
        return np.zeros_like(r)
    y, _ = forward(P, network_input(r, psi, dt, h))
    return r / d + rho * d0 * y[0]


def training_target(r, e, psi, dt, h):
    """Target of the network output for a pair (r, e) with M e = r."""
    d = jacobi_diag(psi, dt, h)
    rho, d0 = precond_scales(r, dt, h)
    return ((e - r / d) / (rho * d0))[None]
