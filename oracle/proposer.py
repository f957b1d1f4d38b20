"""Learned proposer of sketch sizes K_n and TR ranks R_n (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper fixes K_n and R_n by hand for each experiment (Section 4).  The
proposer replaces that choice with a small multilayer perceptron that reads
the singular-value spectrum of every sketched unfolding Y_n = X_(n) Omega_n
(Algorithm 1, step 5) and outputs (K_n, R_n) per mode.  Everything below is
this build's own definition (the paper has no learned component); the CUDA
library implements the same definition in its own kernels:

* features: for mode n < 5, the singular values s_0 >= s_1 >= ... of Y_n
  (at most 64), mapped to f[64 n + i] = max(0, 1 + log10(s_i / s_0) / 6);
  entries past min(I_n, K_n) and modes n >= N are 0.
* network: 320 -> 128 -> 128 -> 128 -> 10, GELU (erf form) after the three
  hidden layers, none after the last.  Every matrix product rounds both
  operands to bfloat16 and accumulates the products exactly (here in
  float64, on the GPU in float32); biases, activations and the master
  weights stay in full precision.
* parameter vector theta = [W1 (128 x 320, row-major), b1, W2 (128 x 128),
  b2, W3 (128 x 128), b3, W4 (10 x 128), b4].
* loss: 0.5 * sum(M * (out - T)^2) / sum(M) over a batch with targets T and
  a 0/1 mask M (unused modes masked out).
* Adam (Kingma and Ba, 2015): beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias
  correction at step t (t = 1, 2, ...).
* outputs: out[2 n] * 64 -> K_n, out[2 n + 1] * 16 -> R_n (rounded, clamped).
"""
import numpy as np
from scipy.special import erf

from .omega import to_bf16

N_IN, N_HID, N_OUT = 320, 128, 10
MODES, SPEC = 5, 64
K_SCALE, R_SCALE = 64.0, 16.0
LAYERS = ((N_HID, N_IN), (N_HID, N_HID), (N_HID, N_HID), (N_OUT, N_HID))
BETA1, BETA2, ADAM_EPS = 0.9, 0.999, 1e-8
FLOOR_DECADES = 6.0


def param_count():
    return sum(o * i + o for o, i in LAYERS)


def unpack(theta):
    """theta -> [(W, b)] per layer (views)."""
    out, off = [], 0
    for o, i in LAYERS:
        W = theta[off:off + o * i].reshape(o, i)
        off += o * i
        b = theta[off:off + o]
        off += o
        out.append((W, b))
    return out


def gelu(x):
    """GELU(x) = x * Phi(x), Phi the standard normal CDF (Hendrycks and Gimpel)."""
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    """d/dx GELU(x) = Phi(x) + x * phi(x)."""
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def spectrum_features(Ys):
    """Features of the sketches Y_n (list of I_n x K_n arrays, N <= 5)."""
    f = np.zeros(N_IN)
    for n, Y in enumerate(Ys):
        s = np.linalg.svd(np.asarray(Y, dtype=np.float64), compute_uv=False)[:SPEC]
        if s.size == 0 or s[0] <= 0:
            continue
        with np.errstate(divide="ignore"):
            v = 1.0 + np.log10(s / s[0]) / FLOOR_DECADES
        f[SPEC * n:SPEC * n + s.size] = np.maximum(v, 0.0)
    return f


def _mm(A, B, rnd):
    """A @ B.T with both operands rounded to bfloat16 (if rnd)."""
    if rnd:
        A, B = to_bf16(A), to_bf16(B)
    return A @ B.T


def forward(theta, F, rnd=True):
    """Returns (out, cache) for inputs F (batch x 320)."""
    layers = unpack(theta)
    H = np.asarray(F, dtype=np.float64)
    Hs, Zs = [H], []
    for l, (W, b) in enumerate(layers):
        Z = _mm(H, W, rnd) + b
        Zs.append(Z)
        H = gelu(Z) if l < 3 else Z
        Hs.append(H)
    return H, (Hs, Zs)


def loss_and_grad(theta, F, T, M, rnd=True):
    """Loss and its gradient with respect to theta (same layout)."""
    out, (Hs, Zs) = forward(theta, F, rnd)
    cnt = float(np.sum(M))
    r = M * (out - T)
    loss = 0.5 * float(np.sum(r * (out - T))) / cnt
    dZ = r / cnt
    layers = unpack(theta)
    grads = [None] * 4
    for l in range(3, -1, -1):
        W, _ = layers[l]
        dW = _mm(dZ.T, Hs[l].T, rnd)          # sum_b dZ[b, o] H[b, i]
        db = dZ.sum(axis=0)
        grads[l] = (dW, db)
        if l > 0:
            dH = _mm(dZ, W.T, rnd)            # sum_o dZ[b, o] W[o, i]
            dZ = dH * gelu_grad(Zs[l - 1])
    return loss, np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])


def adam_step(theta, grad, m, v, t, lr):
    """One Adam step at step number t >= 1; returns new (theta, m, v)."""
    m = BETA1 * m + (1.0 - BETA1) * grad
    v = BETA2 * v + (1.0 - BETA2) * grad * grad
    mh = m / (1.0 - BETA1 ** t)
    vh = v / (1.0 - BETA2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def decode(out, dims, r_max=16):
    """Network output -> (K_n, R_n) for a tensor of shape dims."""
    K, R = [], []
    for n, I in enumerate(dims):
        K.append(int(min(max(np.rint(out[2 * n] * K_SCALE), 1), min(I, SPEC))))
        R.append(int(min(max(np.rint(out[2 * n + 1] * R_SCALE), 1), r_max)))
    return K, R


def targets(K, R):
    """Training target and mask rows for per-mode labels (K_n, R_n)."""
    T, M = np.zeros(N_OUT), np.zeros(N_OUT)
    for n, (k, r) in enumerate(zip(K, R)):
        T[2 * n], T[2 * n + 1] = k / K_SCALE, r / R_SCALE
        M[2 * n] = M[2 * n + 1] = 1.0
    return T, M
