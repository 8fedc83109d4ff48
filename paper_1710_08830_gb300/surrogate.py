"""Learned surrogate of the loop k-sums for the Rashba-Hubbard family (not part of the paper).

The network maps 20 features of (transfer momentum q, temperature, model parameters alpha, t', mu)
to the compact P and C loops of the 24x24 / 8x8-per-cell, 9-bond discretisation (2 x 25 x 16 complex
values), learning T dF/dT (the flow variable), centred per output and scaled by one global factor.
Training data are loops that the library's own direct k-sum computes; training runs entirely in the
library's BF16 kernels (forward, backward, Adam).  Inside a flow the library checks the surrogate
against the direct k-sum at a few transfer momenta and falls back to the direct k-sum, for the rest of
the flow, at the first check whose residual exceeds the tolerance.
"""
from __future__ import annotations

import ctypes as C
import math
import time
from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import torch

from . import _lib
from .api import CH_C, CH_P, PRODUCTS_SIMT, SPLIT32, Model
from .inputs import rashba_hubbard

N_FEAT = 20
LOGT_C, LOGT_S = -0.8, 3.1       # (log T - centre) / scale; the library uses the same constants
T_MIN, T_MAX = 0.02, 10.0


class Net:
    """A tufrg_mlp network (BF16 weights, FP32 accumulation) owned from Python."""

    def __init__(self, n_in: int = N_FEAT, width: int = 256, depth: int = 4, n_out: int = 1600, seed: int = 0,
                 stream: Optional[torch.cuda.Stream] = None):
        self._L = _lib.lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        st = self._L.tufrg_mlp_create(n_in, width, depth, n_out, C.c_ulonglong(seed), C.c_void_p(self.stream.cuda_stream),
                                      C.byref(h))
        self._h = h
        if st != 0:
            msg = self._L.tufrg_mlp_last_error(h).decode() if h.value else ""
            raise _lib.TufrgError(st, msg)
        self.n_in, self.width, self.depth, self.n_out = n_in, width, depth, n_out
        self.n_params = int(self._L.tufrg_mlp_num_params(self._h))

    def _check(self, st):
        if st != 0:
            raise _lib.TufrgError(st, self._L.tufrg_mlp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.tufrg_mlp_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params, np.float32)
        self._check(self._L.tufrg_mlp_get_params(self._h, p.ctypes.data))
        return p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.n_params
        self._check(self._L.tufrg_mlp_set_params(self._h, p.ctypes.data))

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        X = X.contiguous().float()
        Y = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=X.device)
        self._check(self._L.tufrg_mlp_forward(self._h, C.c_void_p(X.data_ptr()), X.shape[0], C.c_void_p(Y.data_ptr())))
        return Y

    def gradients(self, X: torch.Tensor, T: torch.Tensor):
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        loss = C.c_float()
        self._check(self._L.tufrg_mlp_gradients(self._h, C.c_void_p(X.contiguous().data_ptr()),
                                                C.c_void_p(T.contiguous().data_ptr()), X.shape[0],
                                                C.c_void_p(g.data_ptr()), C.byref(loss)))
        return loss.value, g

    def train_step(self, X: torch.Tensor, T: torch.Tensor, lr: float, want_loss: bool = False):
        loss = C.c_float()
        self._check(self._L.tufrg_mlp_train_step(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                                 X.shape[0], C.c_float(lr), C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None


def features(Lq: int, T: float, alpha: float, tp: float, mu: float) -> np.ndarray:
    """The 20 input features of every transfer momentum (same formula as the library's kernel)."""
    q = np.arange(Lq * Lq)
    qx = 2.0 * math.pi * (q // Lq) / Lq
    qy = 2.0 * math.pi * (q % Lq) / Lq
    X = np.zeros((Lq * Lq, N_FEAT), np.float64)
    for n in range(1, 5):
        X[:, 4 * (n - 1) + 0] = np.sin(n * qx)
        X[:, 4 * (n - 1) + 1] = np.cos(n * qx)
        X[:, 4 * (n - 1) + 2] = np.sin(n * qy)
        X[:, 4 * (n - 1) + 3] = np.cos(n * qy)
    X[:, 16] = (math.log(T) - LOGT_C) / LOGT_S
    X[:, 17] = (alpha - 0.2) / 0.2
    X[:, 18] = (tp + 0.15) / 0.15
    X[:, 19] = (mu + 0.9) / 0.3
    return X.astype(np.float32)


def family_draw(rng: np.random.Generator):
    """(t', alpha, mu) of the Rashba-Hubbard family, drawn in that order."""
    tp = float(rng.uniform(-0.3, 0.0))
    alpha = float(rng.uniform(0.0, 0.4))
    mu = float(rng.uniform(-1.2, -0.6))
    return tp, alpha, mu


@dataclass
class Dataset:
    X: torch.Tensor          # [n][20]
    Y: torch.Tensor          # [n][n_out]  T dF/dT (unstandardised)
    draws: list              # (tp, alpha, mu, T) per block
    q_per_block: int         # samples per (model, temperature) block


def generate(n_samples: int, seed: int, Lq: int = 24, nc: int = 8, n_ff: int = 9, q_per_block: int = 64,
             temps_per_model: int = 8, U: float = 2.5, T_range=(T_MIN, T_MAX)) -> Dataset:
    """Loops from the library's direct k-sum for random family members and log-uniform temperatures.

    Each (model, temperature) block contributes q_per_block distinct transfer momenta drawn at random
    (all Nq, in order, when q_per_block >= Nq), so a fixed sample budget covers many more points of the
    (T, alpha, t', mu) space than whole blocks would."""
    rng = np.random.default_rng(seed)
    Nq = Lq * Lq
    per = min(q_per_block, Nq)
    n_blocks = int(math.ceil(n_samples / per))
    Xs, Ys, draws = [], [], []
    m = None
    for i in range(n_blocks):
        if i % temps_per_model == 0:
            tp, alpha, mu = family_draw(rng)
            if m is not None:
                m.close()
            m = Model(rashba_hubbard(1.0, tp, alpha, U, mu, Lq=Lq, nc=nc, n_ff=n_ff), SPLIT32, products=PRODUCTS_SIMT)
        T = float(math.exp(rng.uniform(math.log(T_range[0]), math.log(T_range[1]))))
        L = m.loops(T, CH_P | CH_C)                            # [2][Nq][nd][4][4] complex128
        y = (T * L).permute(1, 0, 2, 3, 4).reshape(Nq, -1)     # [Nq][2 * nd * 16] complex
        qs = np.arange(Nq) if per == Nq else np.sort(rng.choice(Nq, per, replace=False))
        qi = torch.from_numpy(qs).cuda()
        Ys.append(torch.view_as_real(y).reshape(Nq, -1).float()[qi])
        Xs.append(torch.from_numpy(features(Lq, T, alpha, tp, mu)[qs]).cuda())
        draws.append((tp, alpha, mu, T))
    if m is not None:
        m.close()
    return Dataset(torch.cat(Xs)[:n_samples].contiguous(), torch.cat(Ys)[:n_samples].contiguous(), draws, per)


@dataclass
class Trained:
    net: Net
    mean: np.ndarray
    std: np.ndarray
    history: list
    seconds: float


def train(data: Dataset, epochs: int = 40, batch: int = 1024, lr: float = 2e-3, lr_end: float = 2e-5, seed: int = 0,
          width: int = 256, depth: int = 4) -> Trained:
    """Adam with a geometric learning-rate decay, all in the library's kernels.

    Targets are centred per output and scaled by one global standard deviation: per-output scaling
    would blow up outputs that vanish by symmetry (pure rounding noise) to unit variance."""
    mean = data.Y.mean(0)
    std = torch.full_like(mean, float((data.Y - mean).pow(2).mean().sqrt().clamp_min(1e-30)))
    Yn = ((data.Y - mean) / std).contiguous()
    net = Net(N_FEAT, width, depth, data.Y.shape[1], seed=seed)
    n = data.X.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    steps = epochs * (n // batch)
    decay = (lr_end / lr) ** (1.0 / max(1, steps))
    hist = []
    t0 = time.perf_counter()
    k = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        losses = []
        for b in range(n // batch):
            idx = perm[b * batch:(b + 1) * batch]
            X = data.X[idx].contiguous()
            Y = Yn[idx].contiguous()
            last = b == n // batch - 1
            l = net.train_step(X, Y, lr * decay ** k, want_loss=last)
            k += 1
            if last:
                losses.append(l)
        hist.append(float(np.mean(losses)))
    torch.cuda.synchronize()
    return Trained(net, mean.cpu().numpy().astype(np.float32), std.cpu().numpy().astype(np.float32), hist,
                   time.perf_counter() - t0)


def relative_errors(tr: Trained, data: Dataset) -> np.ndarray:
    """Relative Frobenius error of the predicted T dF/dT per (model, temperature) block (whole blocks)."""
    Nq = data.q_per_block
    Y = tr.net.forward(data.X)
    pred = Y * torch.from_numpy(tr.std).cuda() + torch.from_numpy(tr.mean).cuda()
    out = []
    for i in range(data.X.shape[0] // Nq):
        p = pred[i * Nq:(i + 1) * Nq]
        t = data.Y[i * Nq:(i + 1) * Nq]
        out.append(float(torch.linalg.norm(p - t) / torch.linalg.norm(t)))
    return np.asarray(out)


def check_momenta(Lq: int, n_check: int = 8, seed: int = 3) -> List[int]:
    """q = 0, q = (pi, pi) and seeded random transfer momenta for the residual check."""
    rng = np.random.default_rng(seed)
    qs = [0, (Lq // 2) * Lq + Lq // 2]
    while len(qs) < n_check:
        q = int(rng.integers(0, Lq * Lq))
        if q not in qs:
            qs.append(q)
    return qs


def attach(model: Model, tr: Trained, alpha: float, tp: float, mu: float, tol: float = 1e-3, n_check: int = 8):
    """Use the trained network as the model's loop surrogate (tufrg_set_surrogate)."""
    qs = np.asarray(check_momenta(model.spec.Lq, n_check), np.int32)
    par = np.asarray([alpha, tp, mu], np.float64)
    st = model._L.tufrg_set_surrogate(model._h, tr.net._h, tr.mean.ctypes.data, tr.std.ctypes.data, par.ctypes.data,
                                      C.c_double(tol), len(qs), qs.ctypes.data)
    model._check(st)
    model._surrogate = tr   # keep the network alive while the model uses it


def detach(model: Model):
    model._check(model._L.tufrg_set_surrogate(model._h, None, None, None, None, C.c_double(0.0), 0, None))


def stats(model: Model):
    """(accepted, rejected, skipped) evaluations since the surrogate was attached."""
    a, r, k = C.c_longlong(), C.c_longlong(), C.c_longlong()
    model._check(model._L.tufrg_surrogate_stats(model._h, C.byref(a), C.byref(r), C.byref(k)))
    return a.value, r.value, k.value
