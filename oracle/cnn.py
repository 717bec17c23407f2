"""FP64 reference of the learned initial guess (TEST INFRASTRUCTURE ONLY).

A plain numpy restatement of the small convolutional network that maps the log-amplitude
of a measured diffraction pattern to the complex object patch under the probe, its loss,
gradients and Adam update.  The CUDA library (paper_2106_07575_gb300/csrc/cnn.cu) is checked
against it; it shares no code with the library.

Network (the workload's description; the paper has no learned component):
    a_0 = log(1 + sqrt(d)), zero frequency centred  input, 1 channel, P x P
    z_l = conv3x3(a_{l-1}; W_l, b_l), zero padding  l = 1..L
    a_l = GELU(z_l) = z_l Phi(z_l)                  l = 1..L-1 (Phi: standard normal CDF)
    amplitude = 0.8 + 0.2 sigmoid(z_L[0]),  phase = (pi/2) sigmoid(z_L[1])
    o = amplitude * exp(i phase)                    predicted object patch
    loss = sum_b sum_px w(px) |o - t|^2 / (B sum_px w(px)),  w = |probe|^2
Convolution is cross-correlation: z[co, y, x] = b[co] + sum_ci sum_{dy,dx in -1..1}
W[co, ci, dy+1, dx+1] a[ci, y+dy, x+dx].
"""
from __future__ import annotations

import math

import numpy as np


def conv3x3(a, W, b):
    """a [B][Cin][P][P], W [Cout][Cin][3][3], b [Cout] -> [B][Cout][P][P] (zero padding)."""
    B, Cin, P, _ = a.shape
    Cout = W.shape[0]
    ap = np.zeros((B, Cin, P + 2, P + 2), np.float64)
    ap[:, :, 1:-1, 1:-1] = a
    z = np.zeros((B, Cout, P, P), np.float64) + b[None, :, None, None]
    for dy in range(3):
        for dx in range(3):
            patch = ap[:, :, dy:dy + P, dx:dx + P]  # [B][Cin][P][P]
            z += np.einsum("oc,bcyx->boyx", W[:, :, dy, dx], patch)
    return z


def conv3x3_backward(a, W, dz):
    """Gradients of conv3x3 w.r.t. its input, weights and bias given dz = dL/dz."""
    B, Cin, P, _ = a.shape
    ap = np.zeros((B, Cin, P + 2, P + 2), np.float64)
    ap[:, :, 1:-1, 1:-1] = a
    dap = np.zeros_like(ap)
    dW = np.zeros_like(W)
    for dy in range(3):
        for dx in range(3):
            patch = ap[:, :, dy:dy + P, dx:dx + P]
            dW[:, :, dy, dx] = np.einsum("boyx,bcyx->oc", dz, patch)
            dap[:, :, dy:dy + P, dx:dx + P] += np.einsum("oc,boyx->bcyx", W[:, :, dy, dx], dz)
    db = dz.sum(axis=(0, 2, 3))
    return dap[:, :, 1:-1, 1:-1], dW, db


def features(d):
    """Network input from counts: log(1 + sqrt(d)), spectrum centred (zero frequency moved
    from [0, 0] to [P/2, P/2]).  d [B][P][P] -> [B][P][P]."""
    P = d.shape[-1]
    return np.roll(np.log1p(np.sqrt(np.maximum(d, 0.0))), (P // 2, P // 2), axis=(-2, -1))


def _phi(x):
    return np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def _Phi(x):
    from scipy.special import erf

    return 0.5 * (1.0 + erf(x / math.sqrt(2.0)))


def gelu(z):
    return z * _Phi(z)


def gelu_grad(z):
    return _Phi(z) + z * _phi(z)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def init_params(channels=32, layers=6, seed=0):
    """He-normal weights (std sqrt(2 / (9 Cin))), zero biases: [(W, b)] per layer."""
    rng = np.random.default_rng(seed)
    params = []
    cin = 1
    for l in range(layers):
        cout = 2 if l == layers - 1 else channels
        W = rng.standard_normal((cout, cin, 3, 3)) * math.sqrt(2.0 / (9 * cin))
        params.append((W, np.zeros(cout)))
        cin = cout
    return params


def forward(params, x):
    """x [B][P][P] -> (o [B][P][P] complex, cache)."""
    a = x[:, None].astype(np.float64)
    zs, acts = [], [a]
    for l, (W, b) in enumerate(params):
        z = conv3x3(a, W, b)
        zs.append(z)
        if l < len(params) - 1:
            a = gelu(z)
            acts.append(a)
    zL = zs[-1]
    s0, s1 = sigmoid(zL[:, 0]), sigmoid(zL[:, 1])
    amp = 0.8 + 0.2 * s0
    ph = (math.pi / 2) * s1
    o = amp * np.exp(1j * ph)
    return o, (acts, zs, s0, s1, amp, ph)


def loss_and_grads(params, x, t, w):
    """Weighted squared error of the predicted patch and the gradients of every parameter."""
    B = x.shape[0]
    o, (acts, zs, s0, s1, amp, ph) = forward(params, x)
    norm = B * w.sum()
    r = o - t
    loss = float(np.sum(w[None] * np.abs(r) ** 2) / norm)
    # dL/do* = w r / norm; dL/damp = 2 Re(conj(r) e^{i ph}) w / norm; dL/dph = 2 Re(conj(r) i o) w / norm
    e = np.exp(1j * ph)
    damp = 2.0 * np.real(np.conj(r) * e) * w[None] / norm
    dph = 2.0 * np.real(np.conj(r) * 1j * o) * w[None] / norm
    dz = np.stack([damp * 0.2 * s0 * (1 - s0), dph * (math.pi / 2) * s1 * (1 - s1)], axis=1)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        da, dW, db = conv3x3_backward(acts[l], W, dz)
        grads[l] = (dW, db)
        if l > 0:
            dz = da * gelu_grad(zs[l - 1])
    return loss, grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update (Kingma & Ba, Algorithm 1); state = {"t", "m", "v"},
    filled with zero moments on the first call.  Returns the new parameter list."""
    flat_p = [x for Wb in params for x in Wb]
    flat_g = [x for Wb in grads for x in Wb]
    if not state:
        state.update({"t": 0, "m": [np.zeros_like(x) for x in flat_p], "v": [np.zeros_like(x) for x in flat_p]})
    state["t"] += 1
    t = state["t"]
    new = []
    for j, (p, g) in enumerate(zip(flat_p, flat_g)):
        state["m"][j] = b1 * state["m"][j] + (1 - b1) * g
        state["v"][j] = b2 * state["v"][j] + (1 - b2) * g * g
        mh = state["m"][j] / (1 - b1**t)
        vh = state["v"][j] / (1 - b2**t)
        new.append(p - lr * mh / (np.sqrt(vh) + eps))
    return [(new[2 * l], new[2 * l + 1]) for l in range(len(params))]


def stitch(patches, probe, pos, shape, floor=1e-3):
    """Probe-weighted average of patch estimates: sum |p|^2 o_k / (sum |p|^2 + floor max),
    pixels no position covers set to 1."""
    H, W = shape
    P = probe.shape[0]
    num = np.zeros((H, W), np.complex128)
    den = np.zeros((H, W), np.float64)
    w = np.abs(probe.astype(np.complex128)) ** 2
    for k, (r, c) in enumerate(pos):
        num[r:r + P, c:c + P] += w * patches[k]
        den[r:r + P, c:c + P] += w
    out = np.ones((H, W), np.complex128)
    m = den > 0
    out[m] = num[m] / (den[m] + floor * den.max())
    return out
