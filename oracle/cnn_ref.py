"""CPU reference of the learned window proposal's network (float64 numpy).

TEST INFRASTRUCTURE ONLY, like the rest of this package.  The network is not
part of the paper; this module writes its operations out from their
definitions so that the CUDA kernels can be checked against them:

  conv3x3(x, w, b, dil)    y[n,y,x,co] = b[co] + sum_{ky,kx,ci}
                           x[n, y+dil(ky-1), x+dil(kx-1), ci] w[3ky+kx, ci, co]
                           (zero outside the image)
  conv3x3_dgrad(dz, w, dil)  gradient of the input
  conv3x3_wgrad(x, dz, dil)  gradient of w and b
  band_head(logits, bands, labels)  log-sum-exp pooling over each band's
                           rows and columns, softmax cross-entropy (mean over
                           images and bands), its gradient, the argmax bin
Weights are [taps][cin][cout] (taps 9..15 of a single-channel layer unused).
"""
import numpy as np


def _shift(x, dy, dx):
    """x[n, y+dy, x+dx, c], zero outside."""
    N, H, W, C = x.shape
    out = np.zeros_like(x)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    if ys < ye and xs < xe:
        out[:, ys:ye, xs:xe] = x[:, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv3x3(x, w, b, dil):
    N, H, W, cin = x.shape
    y = np.zeros((N, H, W, w.shape[-1]))
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        xs = _shift(x, dil * (ky - 1), dil * (kx - 1))
        y += xs @ w[tap, :cin] if cin > 1 else xs[..., :1] * w[tap, 0][None, None, None, :]
    if b is not None:
        y += b
    return y


def conv3x3_dgrad(dz, w, dil):
    """d(input) of conv3x3 from d(output): the transposed convolution."""
    N, H, W, cout = dz.shape
    cin = w.shape[1]
    dx = np.zeros((N, H, W, cin))
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        # input pixel p + off contributes to output pixel p
        dx += _shift(dz @ w[tap].T, -dil * (ky - 1), -dil * (kx - 1))
    return dx


def conv3x3_wgrad(x, dz, dil, taps=9):
    N, H, W, cin = x.shape
    dw = np.zeros((taps, cin, dz.shape[-1]))
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        xs = _shift(x, dil * (ky - 1), dil * (kx - 1))
        dw[tap] = xs.reshape(-1, cin).T @ dz.reshape(-1, dz.shape[-1])
    return dw, dz.reshape(-1, dz.shape[-1]).sum(0)


def band_head(logits, bands, labels=None):
    N, H, W, C = logits.shape
    rpb = H // bands
    z = logits.reshape(N, bands, rpb * W, C)
    m = z.max(axis=2, keepdims=True)
    pooled = (m + np.log(np.exp(z - m).sum(axis=2, keepdims=True)))[:, :, 0, :]   # [N, b, C]
    pred = pooled.argmax(-1)
    if labels is None:
        return pooled, None, None, pred
    pm = pooled.max(-1, keepdims=True)
    lse = pm[..., 0] + np.log(np.exp(pooled - pm).sum(-1))
    lab = np.asarray(labels).reshape(N, bands)
    nll = lse - np.take_along_axis(pooled, lab[..., None], -1)[..., 0]
    loss = nll.mean()
    soft = np.exp(pooled - lse[..., None])
    dpool = soft.copy()
    np.put_along_axis(dpool, lab[..., None], np.take_along_axis(soft, lab[..., None], -1) - 1, -1)
    dpool /= N * bands
    dz = dpool[:, :, None, :] * np.exp(z - pooled[:, :, None, :])
    return pooled, loss, dz.reshape(N, H, W, C), pred
