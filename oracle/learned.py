"""Plain FP64 restatement of the learned proposal: its input features and its MLP.

TEST INFRASTRUCTURE ONLY: the test suite is the only caller; the GPU scheduler never
imports this module, and this module never imports the scheduler.

The paper's method has no learned part; the proposal network is this project's addition
(a policy trained on the paper's FastMDP action choices, Alg. 1 / Sec. III). This module
states what the GPU computes, in plain numpy and double precision:

features(...)   the 128 inputs at one state: 8 own/goal terms, then 20 sectors around the
                aircraft (10 azimuth sectors of 36 degrees in its heading frame x above /
                below), each holding the nearest plan sample of the next step within
                R_F metres: relative position and velocity relative to the aircraft's own
                (speed along its heading), both scaled by (1 - distance / R_F), so an empty
                or distant sector reads zero;
mlp_forward     128 -> 256 -> 256 -> 256 -> 256 -> 25, ReLU between layers;
loss_and_grad   mean softmax cross-entropy over a batch and its exact gradient; with
                round_fn (bf16 below) the same computation with the bf16 network's rounding
                points stated: hidden activations after ReLU, and the output gradients of a
                layer where they enter a matrix product (its bias gradient uses them unrounded).
bf16            round to the nearest bfloat16 (ties to even), as a float64 array.

Parameter vector: for each layer l, W_l (in x out, row-major) then b_l (out).
"""
import numpy as np

DIMS = (128, 256, 256, 256, 256, 25)
R_F = 1000.0          # metres: intruder sectors reach this far
N_SECTORS = 20        # 10 azimuth sectors x (above, below)
N_OWN = 8


def n_params(dims=DIMS):
    return sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(len(dims) - 1))


def unpack(params, dims=DIMS):
    out, o = [], 0
    for i in range(len(dims) - 1):
        a, b = dims[i], dims[i + 1]
        W = np.asarray(params[o:o + a * b], dtype=np.float64).reshape(a, b)
        o += a * b
        bias = np.asarray(params[o:o + b], dtype=np.float64)
        o += b
        out.append((W, bias))
    return out


def bf16(x):
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    a = (a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000
    return a.astype(np.uint32).view(np.float32).astype(np.float64)


def _identity(x):
    return x


def mlp_forward(params, X, dims=DIMS, round_fn=_identity):
    """Logits for the rows of X; also the hidden activations (post-ReLU) per layer."""
    layers = unpack(params, dims)
    h = np.asarray(X, dtype=np.float64)
    acts = [h]
    for i, (W, b) in enumerate(layers):
        z = h @ W + b
        h = z if i == len(layers) - 1 else round_fn(np.maximum(z, 0.0))
        acts.append(h)
    return h, acts


def loss_and_grad(params, X, y, dims=DIMS, n_valid=None, round_fn=_identity):
    """Mean cross-entropy of softmax(logits) against labels y, and d loss / d params.
    Logits at or beyond n_valid (an action set smaller than the output) are masked."""
    logits, acts = mlp_forward(params, X, dims, round_fn)
    B = logits.shape[0]
    if n_valid is not None and n_valid < logits.shape[1]:
        logits = logits.copy()
        logits[:, n_valid:] = -np.inf
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    p = e / e.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(p[np.arange(B), y])))
    g = p.copy()
    g[np.arange(B), y] -= 1.0
    g /= B
    layers = unpack(params, dims)
    grads = []
    for i in range(len(layers) - 1, -1, -1):
        W, _ = layers[i]
        h_in = acts[i]
        gr = round_fn(g)
        gW = h_in.T @ gr
        gb = g.sum(axis=0)
        grads.append((gW, gb))
        if i > 0:
            g = (gr @ W.T) * (acts[i] > 0.0)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def _heading_frame(hc, hs, v):
    """Components of v along the heading (forward) and to its left."""
    return v[0] * hc + v[1] * hs, -v[0] * hs + v[1] * hc


def features(s, hc, hs, speed, goal, box, p1, p2, dt=1.0, terrain=None):
    """The 128 inputs at state s (x, y, z) with heading (cos, sin) = (hc, hs) and speed.

    goal: (x, y, z); box: (x0, y0, z0, x1, y1, z1); p1, p2: every plan sample at the next
    step and the same plan's sample one step later (NaN rows: none), arrays of shape
    (n, 3); terrain: callable h(x, y) or None."""
    s = np.asarray(s, dtype=np.float64)
    f = np.zeros(N_OWN + 6 * N_SECTORS)
    z0, z1 = box[2], box[5]
    f[0] = (s[2] - z0) / (z1 - z0)
    clr = (s[2] - terrain(s[0], s[1])) if terrain is not None else (s[2] - z0)
    f[1] = min(max(clr / 200.0, -1.0), 4.0)
    g = np.asarray(goal, dtype=np.float64) - s
    gf, gl = _heading_frame(hc, hs, g)
    gh = np.hypot(gf, gl)
    f[2] = min(max(gf / 5000.0, -4.0), 4.0)
    f[3] = min(max(gl / 5000.0, -4.0), 4.0)
    f[4] = min(max(g[2] / 200.0, -4.0), 4.0)
    f[5] = min(gh / 20000.0, 4.0)
    f[6] = gf / gh if gh > 0 else 1.0
    f[7] = gl / gh if gh > 0 else 0.0
    best = {}
    for i in range(len(p1)):
        q = np.asarray(p1[i], dtype=np.float64)
        if not np.isfinite(q[0]):
            continue
        rel = q - s
        d = np.sqrt(rel @ rel)
        if not d < R_F:
            continue
        rf, rl = _heading_frame(hc, hs, rel)
        az = np.arctan2(rl, rf)  # (-pi, pi]
        sector = min(int(np.floor((az + np.pi) / (2.0 * np.pi) * 10.0)), 9) + (10 if rel[2] >= 0.0 else 0)
        if sector not in best or d < best[sector][0]:
            best[sector] = (d, i)
    for sector, (d, i) in best.items():
        rel = np.asarray(p1[i], dtype=np.float64) - s
        q2 = np.asarray(p2[i], dtype=np.float64)
        vel = (q2 - p1[i]) / dt if np.isfinite(q2[0]) else np.zeros(3)
        w = 1.0 - d / R_F
        rf, rl = _heading_frame(hc, hs, rel)
        vf, vl = _heading_frame(hc, hs, vel)
        o = N_OWN + 6 * sector
        f[o:o + 6] = np.array([rf / 500.0, rl / 500.0, rel[2] / 500.0, (vf - speed) / 50.0, vl / 50.0,
                               vel[2] / 50.0]) * w
    return f
