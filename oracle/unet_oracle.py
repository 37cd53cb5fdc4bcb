"""FP64 reference of the learned warm start's network.  TEST INFRASTRUCTURE ONLY:
only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may use it.

The warm start maps three input channels on the (n+1) x (n+1) grid -- the
interior n x n sites padded with one zero row and column -- to an estimate of
the posterior mean mu = A~^-1 f (Sec. 2.2; the chain's law does not depend on
its starting state, so the estimate only shortens burn-in):
  channel 0: log(kappa^2 / 10) at each site,
  channel 1: sum over observations k of the row weight B_{k,i} (the bilinear
             weights of point observation k at site i),
  channel 2: sum over k of B_{k,i} y_k.
Network (a U-Net): channels-last arrays [batch][H][W][C]; c_s = c0 * 2^s.
  encoder level s = 0, 1, 2: conv3x3 + ReLU twice (-> skip_s), 2x2 average pool;
  bottom (level 3): conv3x3 + ReLU twice;
  decoder level s = 2, 1, 0: nearest 2x upsampling, concatenation [upsampled,
  skip_s] along channels, conv3x3 + ReLU twice;
  output: 1x1 convolution to one channel (no activation); the first n rows and
  columns are the estimate.
Convolutions: zero padding, stride 1, y[o] = b[o] + sum_{ky,kx,c} W[o,ky,kx,c]
x[y+ky-1, x+kx-1, c].  Loss: mean squared error over the n x n interior.
Parameters as one flat vector: per convolution W [cout][3][3][cin] then b
[cout], in the layer order of layer_table(), then the output layer w [c0], b [1].

With bf16=True the values the device stores in BF16 (inputs, weights,
activations, activation gradients) are rounded to BF16 at the same points;
the sums stay FP64.
"""
import numpy as np


def bf16_round(a):
    """Round FP64 values to the nearest BF16 value (ties to even), returned as FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_table(c0):
    """(name, level, cin, cout) of the 14 convolutions in evaluation order."""
    c = [c0, 2 * c0, 4 * c0, 8 * c0]
    return [("e0a", 0, 3, c[0]), ("e0b", 0, c[0], c[0]), ("e1a", 1, c[0], c[1]), ("e1b", 1, c[1], c[1]),
            ("e2a", 2, c[1], c[2]), ("e2b", 2, c[2], c[2]), ("ba", 3, c[2], c[3]), ("bb", 3, c[3], c[3]),
            ("d2a", 2, c[3] + c[2], c[2]), ("d2b", 2, c[2], c[2]), ("d1a", 1, c[2] + c[1], c[1]),
            ("d1b", 1, c[1], c[1]), ("d0a", 0, c[1] + c[0], c[0]), ("d0b", 0, c[0], c[0])]


def n_params(c0):
    return sum(co * 9 * ci + co for _, _, ci, co in layer_table(c0)) + c0 + 1


def unpack(theta, c0):
    """Flat parameter vector -> list of (W [cout,3,3,cin], b [cout]) and (w_out [c0], b_out)."""
    theta = np.asarray(theta, dtype=np.float64)
    layers, o = [], 0
    for _, _, ci, co in layer_table(c0):
        W = theta[o:o + co * 9 * ci].reshape(co, 3, 3, ci)
        o += co * 9 * ci
        b = theta[o:o + co]
        o += co
        layers.append((W, b))
    w_out = theta[o:o + c0]
    b_out = theta[o + c0]
    return layers, (w_out, b_out)


def conv3(x, W, b):
    """3x3 convolution, zero padding: y[b,i,j,o] = b[o] + sum_{ky,kx,c} W[o,ky,kx,c] x[b,i+ky-1,j+kx-1,c]."""
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, Wd, W.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("bhwc,oc->bhwo", xp[:, ky:ky + H, kx:kx + Wd, :], W[:, ky, kx, :])
    return y


def conv3_backward(x, W, dy):
    """Gradients of sum(dy * conv3(x, W, b)) with respect to x, W and b."""
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            dW[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dy, xp[:, ky:ky + H, kx:kx + Wd, :])
            dxp[:, ky:ky + H, kx:kx + Wd, :] += np.einsum("bhwo,oc->bhwc", dy, W[:, ky, kx, :])
    return dxp[:, 1:-1, 1:-1, :], dW, dy.sum(axis=(0, 1, 2))


def pool2(x):
    """2x2 average pooling."""
    return 0.25 * (x[:, 0::2, 0::2] + x[:, 1::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 1::2])


def pool2_backward(dy):
    dx = np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2)
    return 0.25 * dx


def up2(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(dy):
    return dy[:, 0::2, 0::2] + dy[:, 1::2, 0::2] + dy[:, 0::2, 1::2] + dy[:, 1::2, 1::2]


def forward(theta, x_in, c0, bf16=False):
    """Network output [B,H,W] and the saved activations (for backward)."""
    rnd = bf16_round if bf16 else (lambda a: a)
    layers, (w_out, b_out) = unpack(theta, c0)
    layers = [(rnd(W), b) for W, b in layers]
    w_out = rnd(w_out)
    x = rnd(np.asarray(x_in, dtype=np.float64))
    ins, acts = [], []

    def conv(i, inp):
        ins.append(inp)
        y = rnd(np.maximum(conv3(inp, *layers[i]), 0.0))
        acts.append(y)
        return y

    s0 = conv(1, conv(0, x))
    s1 = conv(3, conv(2, rnd(pool2(s0))))
    s2 = conv(5, conv(4, rnd(pool2(s1))))
    bt = conv(7, conv(6, rnd(pool2(s2))))
    d2 = conv(9, conv(8, np.concatenate([up2(bt), s2], axis=3)))
    d1 = conv(11, conv(10, np.concatenate([up2(d2), s1], axis=3)))
    d0 = conv(13, conv(12, np.concatenate([up2(d1), s0], axis=3)))
    out = np.einsum("bhwc,c->bhw", d0, w_out) + b_out
    return out, (ins, acts, layers, w_out)


def loss_and_grad(theta, x_in, target, c0, bf16=False):
    """Mean squared error over the n x n interior and its gradient (flat, like theta)."""
    out, (ins, acts, layers, w_out) = forward(theta, x_in, c0, bf16)
    rnd = bf16_round if bf16 else (lambda a: a)
    B, H, _ = out.shape
    n = target.shape[1]
    diff = out[:, :n, :n] - target
    loss = float(np.mean(diff ** 2))
    dout = np.zeros_like(out)
    dout[:, :n, :n] = 2.0 * diff / diff.size
    d0 = acts[13]
    dw_out = np.einsum("bhw,bhwc->c", dout, d0)
    db_out = float(dout.sum())
    grads = [None] * 14
    dact = [None] * 14
    dact[13] = np.einsum("bhw,c->bhwc", dout, w_out)

    def back(i):
        dz = rnd(dact[i] * (acts[i] > 0))
        dx, dW, db = conv3_backward(ins[i], layers[i][0], dz)
        grads[i] = (dW, db)
        return dx

    def split(dx, cup):
        return dx[..., :cup], dx[..., cup:]

    c = [c0, 2 * c0, 4 * c0, 8 * c0]
    dact[12] = back(13)
    du, dskip0 = split(back(12), c[1])
    dact[11] = up2_backward(du)
    dact[10] = back(11)
    du, dskip1 = split(back(10), c[2])
    dact[9] = up2_backward(du)
    dact[8] = back(9)
    du, dskip2 = split(back(8), c[3])
    dact[7] = up2_backward(du)
    dact[6] = back(7)
    dact[5] = dskip2 + pool2_backward(back(6))
    dact[4] = back(5)
    dact[3] = dskip1 + pool2_backward(back(4))
    dact[2] = back(3)
    dact[1] = dskip0 + pool2_backward(back(2))
    dact[0] = back(1)
    back(0)
    flat = []
    for dW, db in grads:
        flat += [dW.ravel(), db.ravel()]
    flat += [dw_out.ravel(), np.array([db_out])]
    return loss, np.concatenate(flat)


def adam_step(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) at step t >= 1."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def make_inputs(n, kappa2, obs_site, obs_w, y):
    """The three input channels [n+1][n+1][3] of one problem (dense site ids i + n j)."""
    H = n + 1
    x = np.zeros((H, H, 3))
    k2 = np.broadcast_to(np.asarray(kappa2, dtype=np.float64), (n * n,)).reshape(n, n)
    x[:n, :n, 0] = np.log(k2 / 10.0)
    if obs_site is not None:
        for k in range(obs_site.shape[0]):
            for t in range(obs_site.shape[1]):
                s = int(obs_site[k, t])
                if s < 0:
                    continue
                i, j = s % n, s // n
                x[j, i, 1] += obs_w[k, t]
                x[j, i, 2] += obs_w[k, t] * y[k]
    return x


class SplitMix64:
    """splitmix64 (Steele, Lea & Flood, OOPSLA 2014): state += 0x9E3779B97F4A7C15, then
    two xor-shift-multiply rounds and a final xor-shift.  uniform() = (top 53 bits + 1/2)
    2^-53; normal() = Box-Muller cosine branch, one pair of uniforms per draw."""
    MASK = (1 << 64) - 1

    def __init__(self, seed):
        self.s = seed & self.MASK

    def next(self):
        self.s = (self.s + 0x9E3779B97F4A7C15) & self.MASK
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self):
        return ((self.next() >> 11) + 0.5) * 2.0 ** -53

    def normal(self):
        r = np.sqrt(-2.0 * np.log(self.uniform()))
        return r * np.cos(2.0 * np.pi * self.uniform())


def init_params(c0, seed):
    """He-normal initial weights (std sqrt(2 / (9 cin)), drawn in the flat order, stored
    as FP32), zero biases, output weights of std sqrt(1 / c0) and zero output bias."""
    r = SplitMix64(seed)
    parts = []
    for _, _, ci, co in layer_table(c0):
        sd = np.sqrt(2.0 / (9 * ci))
        parts += [np.array([sd * r.normal() for _ in range(co * 9 * ci)], dtype=np.float32), np.zeros(co)]
    parts += [np.array([np.sqrt(1.0 / c0) * r.normal() for _ in range(c0)], dtype=np.float32), np.zeros(1)]
    return np.concatenate(parts).astype(np.float64)


def epoch_permutation(n_samples, r):
    """Fisher-Yates from the last position: swap i with next() mod (i + 1), i = n-1 .. 1."""
    perm = list(range(n_samples))
    for i in range(n_samples - 1, 0, -1):
        j = r.next() % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def train(theta, x, t, c0, epochs, batch, lr, shuffle_seed, bf16=False):
    """Adam over shuffled mini-batches (n_samples // batch steps per epoch); returns the
    final parameters and the mean training loss of each epoch."""
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    r = SplitMix64(shuffle_seed)
    step, losses = 0, []
    for _ in range(epochs):
        perm = epoch_permutation(x.shape[0], r)
        acc, nb = 0.0, x.shape[0] // batch
        for b in range(nb):
            idx = perm[b * batch:(b + 1) * batch]
            loss, g = loss_and_grad(theta, x[idx], t[idx], c0, bf16)
            step += 1
            theta, m, v = adam_step(theta, m, v, g, step, lr)
            acc += loss
        losses.append(acc / nb)
    return theta, np.array(losses)
