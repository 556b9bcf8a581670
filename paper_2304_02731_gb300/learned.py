"""Learned importance-sampling proposal: orchestration of the C-ABI calls.

Steps (all arithmetic in the library's kernels; this module only sequences
calls):

1. Training data: lanes of one Ca-H system drawn like the mixed study
   (E ~ U[0.05, 0.30] hartree, b^2 ~ U[0, 100] bohr^2, v in 0..10, j in
   0..20), integrated in FP64 or, for speed, with the FP32 integrator (its
   outcome classes agree with FP64 on >= 99.9 % of lanes; the labels only
   shape the proposal, so the estimator stays unbiased either way); inputs
   x = (E, b, v, j, theta, phi, chi, eta) from qcams_mlp_features, targets
   the outcome classes.
2. Training: minibatch Adam steps (qcams_mlp_train: minibatch indices drawn
   on the device, gradient over the gathered rows, Adam).
3. Proposal at one (E, v, j): qcams_build_proposal.
4. Estimation: lanes drawn from the proposal (qcams_sample_proposal), their
   initial states built from the drawn uniforms (qcams_init_states with
   u_in), integrated exactly, and reduced with likelihood-ratio weights:
   sigma_R = pi b_max^2 mean(w 1_R) with its sample standard error.  The
   uniform baseline draws b^2 uniformly and the angles from the usual
   generator, weight 1.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import qcams as Q

B2_MAX = 100.0


def draw_training_lanes(n: int, seed: int):
    """Seeded lane inputs of the mixed study for one system."""
    rng = np.random.default_rng(seed)
    E = rng.uniform(0.05, 0.30, n)
    b = np.sqrt(rng.uniform(0.0, B2_MAX, n))
    v = rng.integers(0, 11, n).astype(np.int32)
    j = rng.integers(0, 21, n).astype(np.int32)
    return E, b, v, j


def generate(system_spec, n: int, seed: int, device="cuda", integ=None, precision: int = 64):
    """Integrate n training lanes (FP64, or the FP32 integrator at its
    tolerances rtol 1e-6 / atol 1e-8 with precision=32); returns (x [n, 8]
    float32 device, cls uint8 device, host dict with E, b, v, j and the
    outcome classes)."""
    dev = torch.device(device)
    E, b, v, j = draw_training_lanes(n, seed)
    batch = Q.Batch.empty(n, dev)
    if integ is None:
        integ = (Q.make_integ(rtol=1e-6, atol=1e-8, persistent=True, precision=32)
                 if precision == 32 else Q.make_integ(persistent=True))
    Q.init_states([system_spec], batch, E, b, v, j, 30.0, seed, 0)
    Q.run_batch([system_spec], batch, integ)
    x = Q.mlp_features(batch, E, b, v, j)
    torch.cuda.synchronize()
    cls = batch.cls.clone()
    host = dict(E=E, b=b, v=v, j=j, cls=cls.cpu().numpy())
    return x, cls, host


def train(mlp: "Q.MLP", x: torch.Tensor, cls: torch.Tensor, epochs: int = 8,
          batch: int = 4096, lr: float = 2e-3, seed: int = 0, log=None):
    """Minibatch Adam (qcams_mlp_train: indices drawn on the device) for
    epochs x n / batch steps; returns the per-epoch mean minibatch losses."""
    mlp.fit_standardizer(x)
    n = x.shape[0]
    per_epoch = max(1, n // batch)
    losses, _ = mlp.train(x, cls, epochs * per_epoch, min(batch, n), lr, seed)
    per = losses.view(epochs, per_epoch).mean(1).cpu().numpy()
    if log:
        for ep, l in enumerate(per):
            log(f"epoch {ep}: loss {l:.4f}")
    return [float(v) for v in per]


def best_state(host, min_count: int | None = None):
    """(v, j) with the largest reactive fraction in the training data, among
    the states holding at least min_count lanes (default: 200, or half the
    mean count per state when the data are smaller)."""
    v, j, cls = host["v"], host["j"], host["cls"]
    if min_count is None:
        min_count = min(200, max(1, len(cls) // (2 * 11 * 21)))
    key = v * 21 + j
    n = np.bincount(key, minlength=11 * 21)
    r = np.bincount(key, weights=((cls == 1) | (cls == 2)).astype(float), minlength=11 * 21)
    frac = np.where(n >= min_count, r / np.maximum(n, 1), -1.0)
    k = int(np.argmax(frac))
    return k // 21, k % 21, float(frac[k])


@dataclass
class Estimate:
    sigma: float
    se: float
    seconds: float
    n: int
    n_reactive: int

    @property
    def fom(self) -> float:
        """1 / (SE^2 T): standard error per GPU-second."""
        return 1.0 / (self.se ** 2 * self.seconds) if self.se > 0 else float("inf")


def estimate_is(system_spec, mlp: "Q.MLP", spec: "Q.ProposalSpec", n: int, seed: int,
                integ=None, device="cuda") -> Estimate:
    """sigma_R (= sigma(AC+B) + sigma(BC+A)) at spec's (E, v, j) from n lanes
    drawn from the learned proposal, with likelihood-ratio weights."""
    dev = torch.device(device)
    if integ is None:
        integ = Q.make_integ(persistent=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    q, qfix, cdf = mlp.build_proposal(spec)
    b, u, w, cell = Q.sample_proposal(spec, qfix, cdf, n, seed)
    batch = Q.Batch.empty(n, dev, isw=w)
    E = torch.full((n,), spec.E_col, dtype=torch.float64, device=dev)
    v = torch.full((n,), spec.v, dtype=torch.int32, device=dev)
    j = torch.full((n,), spec.j, dtype=torch.int32, device=dev)
    Q.init_states([system_spec], batch, E, b, v, j, 30.0, seed, 0, u_in=u)
    Q.run_batch([system_spec], batch, integ)
    hist, cells, groups = Q.reduce_xsec(batch, 1, [1.0], [B2_MAX / 2.0], [0], 1, weighted=True)
    dt = time.perf_counter() - t0
    h = hist.cpu().numpy()[0]
    return Estimate(groups[0, 6, 0], groups[0, 6, 1], dt, n,
                    int(h[Q.H_COUNT + 1] + h[Q.H_COUNT + 2]))


def estimate_uniform(system_spec, spec: "Q.ProposalSpec", n: int, seed: int, integ=None,
                     device="cuda") -> Estimate:
    """The same sigma_R from n lanes drawn uniformly (b^2 ~ U[0, b_max^2],
    angles and phase from the library's generator), weight 1."""
    dev = torch.device(device)
    if integ is None:
        integ = Q.make_integ(persistent=True)
    rng = np.random.default_rng(seed)
    b = np.sqrt(rng.uniform(0.0, B2_MAX, n))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch = Q.Batch.empty(n, dev)
    Q.init_states([system_spec], batch, np.full(n, spec.E_col), b, np.full(n, spec.v, np.int32),
                  np.full(n, spec.j, np.int32), 30.0, seed, 0)
    Q.run_batch([system_spec], batch, integ)
    hist, cells, groups = Q.reduce_xsec(batch, 1, [1.0], [B2_MAX / 2.0], [0], 1)
    dt = time.perf_counter() - t0
    h = hist.cpu().numpy()[0]
    return Estimate(groups[0, 6, 0], groups[0, 6, 1], dt, n,
                    int(h[Q.H_COUNT + 1] + h[Q.H_COUNT + 2]))
