"""Linear cost model of a hashing launch, fitted to measured launches.

The paper models GPU time as work over throughput plus fixed costs
(Eq. 2; its per-item form P_gpu / N_thread + T_alloc + T_memcpy).  Here the
work of a batch is counted per algorithm as padded blocks x ops per block
(RFC 1321 Sec. 3.1-3.2, FIPS 180-4 Sec. 5.1.1, GB/T 32905 Sec. 5.2 for the
padding), and the model is

    T = a_md5 * W_md5 + a_sha1 * W_sha1 + a_sm3 * W_sm3 + T0

with one rate per algorithm (seconds per op) and a fixed launch cost T0,
fitted by least squares.  A fitted model predicts the time of a batch from
its lengths and algorithms alone, e.g. to bound how much work a scheduler
may queue for a latency target.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import shard


def work_by_alg(lengths, algs=None, alg: int | None = None) -> np.ndarray:
    """Ops of each algorithm in a batch: [W_md5, W_sha1, W_sm3]."""
    costs = shard.message_costs(lengths, algs, alg)
    out = np.zeros(3, dtype=np.float64)
    if algs is None:
        out[int(alg)] = float(costs.sum())
    else:
        codes = np.asarray(algs)
        for a in range(3):
            out[a] = float(costs[codes == a].sum())
    return out


@dataclasses.dataclass
class CostModel:
    rate: np.ndarray      # seconds per op, per algorithm
    overhead: float       # seconds per launch
    r2: float             # coefficient of determination on the fitting set

    def predict(self, work: np.ndarray) -> float:
        return float(np.dot(self.rate, work) + self.overhead)

    def predict_batch(self, lengths, algs=None, alg: int | None = None) -> float:
        return self.predict(work_by_alg(lengths, algs, alg))


def fit(samples) -> CostModel:
    """samples: iterable of (work vector [3], seconds).  Algorithms absent
    from every sample keep a zero rate."""
    W = np.array([np.asarray(w, dtype=np.float64) for w, _ in samples])
    t = np.array([float(s) for _, s in samples])
    if W.shape[0] < 2:
        raise ValueError("need at least two samples")
    used = W.sum(axis=0) > 0
    X = np.concatenate([W[:, used], np.ones((W.shape[0], 1))], axis=1)
    coef, *_ = np.linalg.lstsq(X, t, rcond=None)
    rate = np.zeros(3)
    rate[used] = coef[:-1]
    pred = X @ coef
    ss_res = float(((t - pred) ** 2).sum())
    ss_tot = float(((t - t.mean()) ** 2).sum())
    r2 = 1.0 - ss_res / ss_tot if ss_tot > 0 else 1.0
    return CostModel(rate, float(coef[-1]), r2)
