"""Learned initial guess: network training on stamps rendered on the fly, and
the start of a batch of single-Sersic + sky fits.

Every step runs in libgf.so's kernels (through :mod:`gf`): drawing training
parameters and PSFs, rendering (model + convolution), noise, input scaling,
forward and backward passes, Adam, the default guess, decoding, the chi^2 of
both starts, and the choice between them.  This module only sequences the calls
and holds the state (weights, Adam moments) in device tensors.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

from . import gf

SIDE = gf.CNN_SIDE
PSF_SIZE = 33
OS_FACTOR, OS_BOX = 5, 8
SIGMA_READ, GAIN = 0.01, 1.0


def stamp_desc(psf_size: int = PSF_SIZE, conv_method: int = gf.CONV_FFT) -> gf.Desc:
    """Single Sersic + sky on 64x64 stamps, 5x5 oversampling in the central 8x8.

    The convolution defaults to the FFT: a 64x64 stamp with a 33x33 PSF has a
    96x96 extended grid, which one CTA transforms in shared memory at about a
    third of the direct sum's time per LM iteration (measured on 65,536 stamps;
    the direct sum stays ahead below P = 15)."""
    return gf.make_desc(SIDE, SIDE, psf_size, [gf.SERSIC, gf.SKY], OS_FACTOR, OS_BOX,
                        conv_method=conv_method)


def uniform_batch(count: int, psf_size: int = PSF_SIZE) -> gf.Batch:
    return gf.make_batch([SIDE] * count, [SIDE] * count, psf_size=psf_size)


def _mix(seed: int, step: int, stream: int) -> int:
    return (seed * 1_000_003 + step) * 4 + stream


def render(params_dev, psf_dev, noise_seed: int, desc=None, batch=None, ws=None):
    """Noisy stamps (image, sigma), each [count, 64, 64], of device parameters."""
    count = params_dev.shape[0]
    desc = desc or stamp_desc(psf_dev.shape[-1])
    batch = batch or uniform_batch(count, psf_dev.shape[-1])
    _, m = gf.evaluate_batch_dev(desc, batch, params_dev, None, None, psf_dev.reshape(-1), ws=ws)
    img, sig = gf.noise(m, noise_seed, SIGMA_READ, GAIN)
    return img.view(count, SIDE, SIDE), sig.view(count, SIDE, SIDE)


@dataclass
class Trainer:
    """Network weights, Adam moments and the step counter (device tensors)."""
    seed: int = 40
    batch: int = 512
    lr: float = 2e-4
    w: object = None
    m: object = None
    v: object = None
    step: int = 0
    losses: list = field(default_factory=list)

    def __post_init__(self):
        import torch
        if self.w is None:
            self.w = gf.cnn_init(self.seed)
        self.m = torch.zeros_like(self.w) if self.m is None else self.m
        self.v = torch.zeros_like(self.w) if self.v is None else self.v
        self._desc = stamp_desc()
        self._b = uniform_batch(self.batch)
        self._ws_r = gf.Workspace()
        self._ws_n = gf.Workspace()
        self._grad = torch.empty_like(self.w)
        self._loss = torch.empty(256, dtype=torch.float32, device=self.w.device)  # ring

    def lr_at(self, step: int, total: int) -> float:
        """Constant, then a cosine fall to 1 % over the last half."""
        import math
        if total <= 0 or step < total // 2:
            return self.lr
        u = (step - total // 2) / max(1, total - total // 2)
        return self.lr * (0.01 + 0.99 * 0.5 * (1.0 + math.cos(math.pi * u)))

    def train_step(self, total: int = 0):
        """One Adam step on a fresh batch of rendered stamps; the loss stays on the device."""
        k = self.step
        p, psf = gf.train_sample(_mix(self.seed, k, 0), self.batch, PSF_SIZE)
        img, sig = render(p, psf, _mix(self.seed, k, 1), self._desc, self._b, self._ws_r)
        x = gf.cnn_input(img, sig)
        t = gf.cnn_encode(p)
        loss = self._loss[k % self._loss.numel():k % self._loss.numel() + 1]
        gf.cnn_loss_grad(self.w, x, t, ws=self._ws_n, grad=self._grad, loss=loss)
        self.step += 1
        gf.cnn_adam(self.w, self.m, self.v, self._grad, self.step, self.lr_at(k, total))
        if self.step % self._loss.numel() == 0 or self.step == total:
            n = (self.step - 1) % self._loss.numel() + 1
            self.losses += self._loss[:n].cpu().tolist()

    def train(self, steps: int):
        for _ in range(steps):
            self.train_step(total=steps)
        return self

    def save(self, path: str):
        """Weights and Adam moments as raw float32, plus a JSON manifest."""
        os.makedirs(path, exist_ok=True)
        for name in ("w", "m", "v"):
            getattr(self, name).cpu().numpy().tofile(os.path.join(path, f"{name}.f32"))
        with open(os.path.join(path, "manifest.json"), "w") as fh:
            json.dump({"nparams": gf.cnn_nparams(), "step": self.step, "seed": self.seed,
                       "batch": self.batch, "lr": self.lr, "files": ["w.f32", "m.f32", "v.f32"]},
                      fh)

    @classmethod
    def load(cls, path: str):
        import torch
        with open(os.path.join(path, "manifest.json")) as fh:
            man = json.load(fh)
        t = {name: torch.as_tensor(np.fromfile(os.path.join(path, f"{name}.f32"), np.float32)).cuda()
             for name in ("w", "m", "v")}
        tr = cls(seed=man["seed"], batch=man["batch"], lr=man["lr"], **t)
        tr.step = man["step"]
        return tr


def starts(w, batch: gf.Batch, img, sig, psf, desc=None, lo=None, hi=None, ws=None,
           moment_centre=False):
    """Starts of single-Sersic + sky fits of 64x64 stamps packed in img / sig.

    Returns (starts [count, 9] device float64, choice [count] int32 with 1 where
    the network's start was kept, default starts [count, 9])."""
    desc = desc or stamp_desc(int(round(psf.numel() / batch.count) ** 0.5))
    dflt = gf.default_guess(batch, img, ws=ws)
    x = gf.cnn_input(img, sig)
    y = gf.cnn_forward(w, x, ws=ws)
    cand = gf.cnn_decode(y, dflt, moment_centre=moment_centre)
    x2c, _ = gf.evaluate_batch_dev(desc, batch, cand, img, sig, psf, ws=ws)
    x2d, _ = gf.evaluate_batch_dev(desc, batch, dflt, img, sig, psf, ws=ws)
    out, choice = gf.guess_select(cand, x2c, dflt, x2d, lo, hi, ws=ws)
    return out, choice, dflt
