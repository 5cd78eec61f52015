"""The learned encoder aid: a network that predicts each level-0 block's
(shift, mode) from 48 statistics of its residuals, trained on the GPU on the
exhaustive search's choices, with the search kept as arbiter and fallback.

Every step runs in librlfc's kernels (rlfc_encode_ex, rlfc_ks_*, rlfc_mlp_*);
torch holds the device buffers and draws the seeded shuffles.  Decoding is
unchanged: an aided stream is an ordinary format-v1 stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import rlfc

P = 14576
NCLASSES = 112


def _p(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s(stream=None):
    return (torch.cuda.current_stream() if stream is None else stream).cuda_stream


def leaf_dataset(rgb: torch.Tensor, U: int, V: int, L: int, c, tau_p: int, tau_b: int, q: int = 0,
                 tau_err: int = 4, lam_q8: int = 256):
    """Encode with the (shift, mode) search and collect the level-0 blocks the
    energy test keeps: (stream bytes, residuals [nblk, 16] int16, labels
    [nblk] uint8 (0xFF = not kept), index [n] int32 of the kept blocks, n)."""
    H, W = rgb.shape[1], rgb.shape[2]
    nblk = U * V * 3 * ((W + 3) // 4) * ((H + 3) // 4)
    resid = torch.empty((nblk, 16), dtype=torch.int16, device="cuda")
    label = torch.empty(nblk, dtype=torch.uint8, device="cuda")
    data = rlfc.encode(rgb, U, V, L, c, tau_p=tau_p, tau_b=tau_b, q=q, mode_space=1, tau_err=tau_err,
                       lam_q8=lam_q8, leaf_resid=resid, leaf_label=label)
    index, n = compact(label)
    return data, resid, label, index, n


def compact(label: torch.Tensor):
    """(index [n] int32 of the entries != 0xFF, ascending; n)."""
    index = torch.empty(label.numel(), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    rlfc._check(rlfc.lib().rlfc_ks_compact(_p(label), label.numel(), _p(index), _p(count), _s()))
    n = int(count.item())
    return index[:n], n


def features(resid: torch.Tensor, label: torch.Tensor | None, index: torch.Tensor | None, n: int):
    """(X [n, 48] bfloat16, Y [n] uint8 labels or None) of blocks resid[index]."""
    x = torch.empty((n, 48), dtype=torch.bfloat16, device="cuda")
    y = torch.empty(n, dtype=torch.uint8, device="cuda") if label is not None else None
    rlfc._check(rlfc.lib().rlfc_ks_features(_p(resid), _p(label), _p(index), n, _p(x), _p(y), _s()))
    return x, y


def search(resid: torch.Tensor, q: int = 0, tau_err: int = 4, lam_q8: int = 256) -> torch.Tensor:
    """The exhaustive search's label of every block of resid [n, 16]."""
    out = torch.empty(resid.shape[0], dtype=torch.uint8, device="cuda")
    rlfc._check(rlfc.lib().rlfc_ks_search(_p(resid), resid.shape[0], q, tau_err, lam_q8, _p(out), _s()))
    return out


class Aid:
    """The 48 -> 64 -> 64 -> 112 network: FP32 master parameters, their BF16
    copy used by the kernels, Adam state."""

    def __init__(self, seed: int = 0):
        rng = np.random.default_rng(seed)
        w = np.zeros(P, dtype=np.float32)
        o = 0
        for fan_in, fan_out in ((48, 64), (64, 64), (64, 112)):
            w[o:o + fan_in * fan_out] = rng.normal(0, np.sqrt(2.0 / fan_in), fan_in * fan_out)
            o += fan_in * fan_out + fan_out          # biases stay zero
        self.master = torch.from_numpy(w).cuda()
        self.w = self.master.to(torch.bfloat16)
        self.m = torch.zeros(P, dtype=torch.float32, device="cuda")
        self.v = torch.zeros(P, dtype=torch.float32, device="cuda")
        self.grad = torch.zeros(P, dtype=torch.float32, device="cuda")
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.step = 0

    def loss_grad(self, x: torch.Tensor, y: torch.Tensor, order: torch.Tensor | None = None, n: int | None = None):
        """Add the summed loss / gradient of samples order[:n] (or x[:n])."""
        n = x.shape[0] if n is None else n
        rlfc._check(rlfc.lib().rlfc_mlp_loss_grad(_p(self.w), _p(x), _p(y), _p(order), n, _p(self.grad),
                                                  _p(self.loss), _s()))

    def adam(self, lr: float, scale: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.step += 1
        rlfc._check(rlfc.lib().rlfc_mlp_adam(_p(self.master), _p(self.w), _p(self.grad), _p(self.m), _p(self.v),
                                             lr, beta1, beta2, eps, scale, self.step, _s()))

    def train(self, x: torch.Tensor, y: torch.Tensor, epochs: int = 8, batch: int = 4096, lr: float = 2e-3,
              seed: int = 0) -> list:
        """Mini-batch Adam over seeded shuffles; returns the mean loss of each
        epoch."""
        n = x.shape[0]
        g = torch.Generator(device="cpu")
        g.manual_seed(seed)
        hist = []
        for ep in range(epochs):
            order = torch.randperm(n, generator=g).to(torch.int32).cuda()
            self.loss.zero_()
            for b0 in range(0, n, batch):
                nb = min(batch, n - b0)
                self.loss_grad(x, y, order[b0:], nb)
                self.adam(lr * (0.5 ** (ep // 3)), 1.0 / nb)
            hist.append(float(self.loss.item()) / n)
        return hist

    def predict(self, x: torch.Tensor, index: torch.Tensor | None = None, out: torch.Tensor | None = None):
        """Predicted labels: out[index[i]] (or out[i]) for each row of x."""
        if out is None:
            out = torch.empty(x.shape[0], dtype=torch.uint8, device="cuda")
        rlfc._check(rlfc.lib().rlfc_mlp_predict(_p(self.w), _p(x), x.shape[0], _p(index), _p(out), _s()))
        return out


def encode_aided(rgb: torch.Tensor, U: int, V: int, L: int, c, tau_p: int, tau_b: int, aid: Aid,
                 x: torch.Tensor, index: torch.Tensor, nblk: int, q: int = 0, tau_err: int = 4,
                 lam_q8: int = 256) -> bytes:
    """Encode with the network's (shift, mode) for the level-0 blocks of
    `index` (features x) and the search everywhere else or where a
    prediction is not a candidate."""
    modes = torch.full((nblk,), 0xFF, dtype=torch.uint8, device="cuda")
    aid.predict(x, index, modes)
    return rlfc.encode(rgb, U, V, L, c, tau_p=tau_p, tau_b=tau_b, q=q, mode_space=1, tau_err=tau_err,
                       lam_q8=lam_q8, leaf_modes=modes)


def psnr_ycocg(orig: np.ndarray, dec: np.ndarray, cap: float = 99.0) -> float:
    """Eq. 4-5: per image (6 PSNR_Y + PSNR_Co + PSNR_Cg) / 8 with peak 255 on
    the YCoCg-R planes, averaged over the images; a lossless plane counts as
    `cap` dB.  orig and dec are uint8 RGB [n, H, W, 3]."""
    def ycc(a):
        a = a.astype(np.int32)
        r, g, b = a[..., 0], a[..., 1], a[..., 2]
        co = r - b
        t = b + (co >> 1)
        cg = g - t
        return np.stack([t + (cg >> 1), co, cg], axis=-1).reshape(a.shape[0], -1, 3)
    mse = ((ycc(orig) - ycc(dec)).astype(np.float64) ** 2).mean(axis=1)
    with np.errstate(divide="ignore"):
        p = np.where(mse > 0, 10.0 * np.log10(255.0 ** 2 / np.maximum(mse, 1e-300)), cap)
    p = np.minimum(p, cap)
    return float(((6.0 * p[:, 0] + p[:, 1] + p[:, 2]) / 8.0).mean())
