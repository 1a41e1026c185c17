"""Optimiser and learning-rate schedulers (oracle; test infrastructure).

Sec. 5.3 selects Adam with ReduceLROnPlateau (Table 2) and, for the first step
of a time series, StepLR (Table 3); SGD and RMSprop, the other optimisers of
its search, are provided as well.  The paper ran them through torch.optim in
PyTorch 2.6 (Sec. 5.2), so their defaults apply where the tables are silent:
epsilon 1e-8, bias correction on, no weight decay, no amsgrad; plateau mode
'min' with a relative threshold, min_lr 0, and a reduction applied only when it
changes the rate by more than 1e-8.

Adam (Kingma & Ba), at step t = 1, 2, ...:
    m <- beta1 m + (1 - beta1) g
    v <- beta2 v + (1 - beta2) g^2
    x <- x - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)
"""
from __future__ import annotations

import math

import numpy as np


class Adam:
    def __init__(self, n, lr, betas=(0.9, 0.999), eps=1e-8):
        self.lr = float(lr)
        self.beta1, self.beta2 = float(betas[0]), float(betas[1])
        self.eps = float(eps)
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0

    def step(self, x, g, lr_scale=None):
        """Return the updated parameter vector (x is not modified).

        lr_scale (optional, per entry) multiplies the learning rate.
        """
        self.t += 1
        b1, b2 = self.beta1, self.beta2
        self.m = b1 * self.m + (1.0 - b1) * g
        self.v = b2 * self.v + (1.0 - b2) * g * g
        m_hat = self.m / (1.0 - b1 ** self.t)
        v_hat = self.v / (1.0 - b2 ** self.t)
        lr = self.lr if lr_scale is None else self.lr * lr_scale
        return x - lr * m_hat / (np.sqrt(v_hat) + self.eps)


class SGD:
    """Sec. 5.3's SGD (PyTorch semantics, dampening 0, no Nesterov):
    buf <- momentum * buf + g;  x <- x - lr * buf  (buf = g without momentum)."""

    def __init__(self, n, lr, momentum=0.0):
        self.lr = float(lr)
        self.momentum = float(momentum)
        self.buf = np.zeros(n)
        self.t = 0

    def step(self, x, g, lr_scale=None):
        self.t += 1
        self.buf = self.momentum * self.buf + g if self.momentum != 0.0 else np.asarray(g, np.float64)
        lr = self.lr if lr_scale is None else self.lr * lr_scale
        return x - lr * self.buf


class RMSprop:
    """Sec. 5.3's RMSprop (Hinton; PyTorch semantics, not centred, no momentum):
    v <- alpha v + (1 - alpha) g^2;  x <- x - lr * g / (sqrt(v) + eps)."""

    def __init__(self, n, lr, alpha=0.99, eps=1e-8):
        self.lr = float(lr)
        self.alpha, self.eps = float(alpha), float(eps)
        self.v = np.zeros(n)
        self.t = 0

    def step(self, x, g, lr_scale=None):
        self.t += 1
        self.v = self.alpha * self.v + (1.0 - self.alpha) * g * g
        lr = self.lr if lr_scale is None else self.lr * lr_scale
        return x - lr * g / (np.sqrt(self.v) + self.eps)


class ReduceLROnPlateau:
    """Plateau rule: after more than `patience` non-improving steps, lr *= factor.

    A step improves when metric < best * (1 - threshold).  After a reduction,
    `cooldown` steps pass during which non-improving steps are not counted.
    """

    def __init__(self, opt, factor=0.1, patience=10, threshold=1e-4, cooldown=0,
                 min_lr=0.0, eps=1e-8):
        self.opt = opt
        self.factor, self.patience = float(factor), int(patience)
        self.threshold, self.cooldown = float(threshold), int(cooldown)
        self.min_lr, self.eps = float(min_lr), float(eps)
        self.best = math.inf
        self.num_bad = 0
        self.cooldown_counter = 0

    def step(self, metric):
        metric = float(metric)
        if metric < self.best * (1.0 - self.threshold):
            self.best = metric
            self.num_bad = 0
        else:
            self.num_bad += 1
        if self.cooldown_counter > 0:
            self.cooldown_counter -= 1
            self.num_bad = 0
        if self.num_bad > self.patience:
            old = self.opt.lr
            new = max(old * self.factor, self.min_lr)
            if old - new > self.eps:
                self.opt.lr = new
            self.cooldown_counter = self.cooldown
            self.num_bad = 0


class StepLR:
    """lr = lr0 * gamma^floor(steps / step_size)."""

    def __init__(self, opt, step_size, gamma):
        self.opt = opt
        self.lr0 = opt.lr
        self.step_size, self.gamma = int(step_size), float(gamma)
        self.count = 0

    def step(self, metric=None):
        self.count += 1
        self.opt.lr = self.lr0 * self.gamma ** (self.count // self.step_size)


class ConstantLR:
    def __init__(self, opt):
        self.opt = opt

    def step(self, metric=None):
        pass
