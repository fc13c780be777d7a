"""Seeded synthetic HDLSS two-class inputs for the generalized DWD solver.

This module only draws random data; it holds none of the solver's arithmetic.
It feeds both the CUDA path (through the C-ABI) and the CPU oracle in the tests
and the benchmark.  Every draw comes from numpy's Philox4x32-10 bit generator
keyed by the instance seed; the held-out set of an instance reuses its class
structure (mean direction, spike directions) and draws fresh samples from an
advanced Philox stream.

Shapes and distributions follow the workloads the solver is measured on
(the paper's UCI/LIBSVM sets are not available; these stand in for them):

* ``plain_fp64``     d=500, n=100, classes N(+-0.5 e1, I), q=1, C=1, sigma0=1, tol 1e-9
* ``spiked_fp32``    d=20000, n=1000, x = +-2 v + N(0, I + 49 S S^T), S: 5 orthonormal spikes,
                     q=1, C=10, tol 1e-6
* ``gaussian``       x = +-shift v + N(0, I) (C-grid, uneven batches, served requests)
* ``heavy_tailed``   Student-t (nu=3) entries, columns normalised to unit length, 1:3 classes
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Instance:
    """One gDWD problem: Z = X diag(y) (d x n, column i = y_i x_i) plus its parameters."""
    X: np.ndarray
    y: np.ndarray
    q: float
    C: float
    tol: float
    sigma0: float = 0.0          # <= 0: the paper's rule min(10C, n)^q
    mu: float = 1.0
    name: str = ""
    seed: int = 0
    Xtest: np.ndarray | None = None
    ytest: np.ndarray | None = None

    @property
    def Z(self) -> np.ndarray:
        return self.X * self.y[None, :].astype(self.X.dtype)

    @property
    def d(self) -> int:
        return self.X.shape[0]

    @property
    def n(self) -> int:
        return self.X.shape[1]


def _gen(seed: int, stream: int = 0) -> np.random.Generator:
    bg = np.random.Philox(key=int(seed))
    if stream:
        bg = bg.jumped(stream)
    return np.random.Generator(bg)


def _labels(n: int, n_pos: int) -> np.ndarray:
    return np.where(np.arange(n) < n_pos, 1.0, -1.0)


def plain_fp64(seed: int = 1001, d: int = 500, n: int = 100, m_test: int = 1000) -> Instance:
    """Two classes N(+-0.5 e1, I_d), 50 + 50 samples, FP64."""
    g = _gen(seed)
    y = _labels(n, n // 2)
    X = g.standard_normal((d, n))
    X[0] += 0.5 * y
    gt = _gen(seed, 1)
    yt = _labels(m_test, m_test // 2)
    Xt = gt.standard_normal((d, m_test))
    Xt[0] += 0.5 * yt
    return Instance(X, y, q=1.0, C=1.0, tol=1e-9, sigma0=1.0, name="plain_fp64", seed=seed, Xtest=Xt, ytest=yt)


def spiked_fp32(seed: int = 2001, d: int = 20000, n: int = 1000, m_test: int = 1000, shift: float = 2.0,
                spikes: int = 5, spike_var: float = 50.0) -> Instance:
    """x = y*shift*v + g + sqrt(spike_var - 1) * sum_k z_k s_k, FP32 (spiked covariance)."""
    g = _gen(seed)
    v = g.standard_normal(d)
    v /= np.linalg.norm(v)
    S = np.linalg.qr(g.standard_normal((d, spikes)))[0]
    amp = np.sqrt(spike_var - 1.0)

    def draw(gen, m, ylab):
        Xm = gen.standard_normal((d, m), dtype=np.float32).astype(np.float64)
        Xm += shift * np.outer(v, ylab) + amp * (S @ gen.standard_normal((spikes, m)))
        return Xm.astype(np.float32)

    y = _labels(n, n // 2)
    X = draw(g, n, y)
    yt = _labels(m_test, m_test // 2)
    Xt = draw(_gen(seed, 1), m_test, yt)
    return Instance(X, y, q=1.0, C=10.0, tol=1e-6, name="spiked_fp32", seed=seed, Xtest=Xt, ytest=yt)


def gaussian(seed: int, d: int, n: int, shift: float = 1.5, n_pos: int | None = None, q: float = 1.0,
             C: float = 10.0, tol: float = 1e-6, m_test: int = 0, dtype=np.float32) -> Instance:
    """x = y*shift*v + N(0, I_d), v a random unit vector."""
    g = _gen(seed)
    v = g.standard_normal(d)
    v /= np.linalg.norm(v)
    n_pos = n // 2 if n_pos is None else n_pos

    def draw(gen, m, ylab):
        Xm = gen.standard_normal((d, m), dtype=np.float32)
        Xm += (shift * v.astype(np.float32))[:, None] * ylab[None, :].astype(np.float32)
        return Xm.astype(dtype)

    y = _labels(n, n_pos)
    X = draw(g, n, y)
    Xt = yt = None
    if m_test:
        yt = _labels(m_test, m_test // 2)
        Xt = draw(_gen(seed, 1), m_test, yt)
    return Instance(X, y, q=q, C=C, tol=tol, name="gaussian", seed=seed, Xtest=Xt, ytest=yt)


def heavy_tailed(seed: int, d: int, n: int, n_pos: int, q: float = 1.0, C: float = 1.0, tol: float = 1e-6,
                 nu: float = 3.0) -> Instance:
    """Entries iid Student-t(nu) = N / sqrt(chi2_nu / nu), each column normalised to unit length."""
    g = _gen(seed)
    y = _labels(n, n_pos)
    X = g.standard_normal((d, n), dtype=np.float32)
    X /= np.sqrt(g.chisquare(nu, size=(d, n)).astype(np.float32) / np.float32(nu))
    X /= np.linalg.norm(X, axis=0, keepdims=True)
    return Instance(X, y, q=q, C=C, tol=tol, name="heavy_tailed", seed=seed)


def uneven_batch(seed: int, count: int = 64, d_range=(5000, 50000), n_range=(200, 2000),
                 qs=(0.5, 1.0, 2.0, 4.0), ratio_range=(1.0, 4.0), shift: float = 1.5, C: float = 10.0):
    """Shapes of an uneven batch: d, n log-uniform, q uniform over qs, class ratio 1:1..1:4."""
    g = _gen(seed)
    out = []
    for k in range(count):
        d = int(round(np.exp(g.uniform(np.log(d_range[0]), np.log(d_range[1])))))
        n = int(round(np.exp(g.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        q = float(qs[g.integers(len(qs))])
        ratio = g.uniform(*ratio_range)
        n_pos = max(1, min(n - 1, int(round(n / (1.0 + ratio)))))
        out.append(dict(seed=seed * 1000 + k, d=d, n=n, q=q, n_pos=n_pos, C=C, shift=shift))
    return out
