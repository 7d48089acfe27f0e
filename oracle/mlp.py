"""FP64 reference of the surrogate MLP (numpy).  TEST INFRASTRUCTURE ONLY.

in -> hidden -> hidden -> hidden -> 1 with GELU(z) = z Phi(z) = 0.5 z (1 +
erf(z / sqrt 2)) after each hidden layer; mean-squared-error loss; the
gradient by the chain rule written out layer by layer; Adam.  Parameters use
the library's flat layout (W^T matrices [out][in]).
"""
import math

import numpy as np

_erf = np.vectorize(math.erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def unpack(p, n_in, hidden):
    out, o = [], 0
    for shape in [(hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (hidden, hidden), (hidden,), (hidden,), (1,)]:
        n = int(np.prod(shape))
        out.append(np.asarray(p[o:o + n], dtype=np.float64).reshape(shape))
        o += n
    return out


def forward(p, x, n_in, hidden):
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p, n_in, hidden)
    a = np.asarray(x, np.float64)
    Zs, As = [], [a]
    for W, b in ((W1, b1), (W2, b2), (W3, b3)):
        z = a @ W.T + b
        a = gelu(z)
        Zs.append(z)
        As.append(a)
    y = a @ w4 + b4[0]
    return y, Zs, As


def loss_and_grad(p, x, t, n_in, hidden):
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p, n_in, hidden)
    y, Zs, As = forward(p, x, n_in, hidden)
    B = len(t)
    d = y - t
    loss = float((d * d).mean())
    dy = 2.0 * d / B
    gw4 = As[3].T @ dy
    gb4 = np.array([dy.sum()])
    dz = np.outer(dy, w4) * gelu_grad(Zs[2])
    grads = {}
    for l, W in ((2, W3), (1, W2), (0, W1)):
        grads[l] = (dz.T @ As[l], dz.sum(axis=0))
        if l > 0:
            dz = (dz @ W) * gelu_grad(Zs[l - 1])
    flat = np.concatenate([grads[0][0].ravel(), grads[0][1], grads[1][0].ravel(), grads[1][1],
                           grads[2][0].ravel(), grads[2][1], gw4, gb4])
    return loss, flat
