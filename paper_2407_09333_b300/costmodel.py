"""Linear cost model of hashing work, fitted to measured launches.

The paper models GPU time as work over throughput plus fixed costs (Eq. 2;
its per-item form P_gpu / N_thread + T_alloc + T_memcpy).  Here the work of a
batch is counted per algorithm as padded blocks x ops per block (RFC 1321
Sec. 3.1-3.2, FIPS 180-4 Sec. 5.1.1, GB/T 32905 Sec. 5.2 for the padding),
and the time of a launch is

    T = sum_a ( rate_a * W_a + msg_a * N_a ) + T0

with W_a the ops and N_a the messages of algorithm a: a throughput term per
op, a per-message term (metadata, staging set-up, digest store, the lanes a
chunk's shorter messages leave idle) and a fixed launch cost T0, fitted by
non-negative least squares.

A message is also a serial chain of compressions (the Merkle-Damgard
iteration: block j needs the chaining value of block j - 1), so however much
of the GPU is free, a message of W ops takes at least W / chain_a seconds,
chain_a being the op rate one chain reaches on a loaded SM.  A request's
latency is bounded below by its longest message's chain; `chain_time`
gives that bound once `chain` is calibrated (`fit_chain`).
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


def msgs_by_alg(n_or_algs, alg: int | None = None) -> np.ndarray:
    """Messages of each algorithm: [N_md5, N_sha1, N_sm3]."""
    out = np.zeros(3, dtype=np.float64)
    if alg is not None:
        out[int(alg)] = float(n_or_algs)
    else:
        codes = np.asarray(n_or_algs)
        for a in range(3):
            out[a] = float((codes == a).sum())
    return out


@dataclasses.dataclass
class CostModel:
    rate: np.ndarray      # seconds per op, per algorithm
    overhead: float       # seconds per launch (T0)
    r2: float             # coefficient of determination on the fitting set
    per_msg: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))
    chain: np.ndarray | None = None   # ops per second of one serial chain, per algorithm
    latency_t0: float = 0.0           # fixed latency of a served request (fit_chain)

    def predict(self, work: np.ndarray, msgs: np.ndarray | None = None) -> float:
        t = float(np.dot(self.rate, work) + self.overhead)
        if msgs is not None:
            t += float(np.dot(self.per_msg, msgs))
        return t

    def predict_batch(self, lengths, algs=None, alg: int | None = None) -> float:
        lengths = np.asarray(lengths)
        msgs = msgs_by_alg(algs) if alg is None else msgs_by_alg(lengths.shape[0], alg)
        return self.predict(work_by_alg(lengths, algs, alg), msgs)

    def work_seconds(self, lengths, alg: int) -> float:
        """Throughput part of one algorithm's messages (no launch cost): the
        GPU-seconds they occupy when the GPU is saturated."""
        lengths = np.asarray(lengths)
        w = work_by_alg(lengths, alg=alg)
        return float(self.rate[alg] * w[alg] + self.per_msg[alg] * lengths.shape[0])

    def request_costs(self, lengths, alg: int) -> tuple[float, float]:
        """(work_seconds, chain_time) of one algorithm's messages in a single
        pass over their lengths: what a server computes for every arriving
        request, so it is kept to one array operation and two reductions."""
        lengths = np.asarray(lengths)
        n = lengths.shape[0]
        if n == 0:
            return 0.0, 0.0
        nb = shard.padded_blocks(lengths)
        ops = int(shard.OPS_PER_BLOCK[alg])
        work = float(self.rate[alg]) * float(nb.sum()) * ops + float(self.per_msg[alg]) * n
        if self.chain is None or self.chain[alg] <= 0:
            return work, 0.0
        return work, float(nb.max()) * ops / float(self.chain[alg])

    def chain_time(self, lengths, alg: int) -> float:
        """Time of the longest message's serial chain among `lengths` (one
        algorithm): the least time the set can take however many SMs are free
        (0 when `chain` is not calibrated)."""
        if self.chain is None or self.chain[alg] <= 0:
            return 0.0
        lengths = np.asarray(lengths)
        if lengths.shape[0] == 0:
            return 0.0
        return float(shard.message_costs(lengths.max(initial=0)[None], alg=alg)[0] / self.chain[alg])


def _nnls(X: np.ndarray, t: np.ndarray) -> np.ndarray:
    try:
        from scipy.optimize import nnls
        return nnls(X, t)[0]
    except ImportError:  # plain least squares, negative coefficients clipped
        return np.maximum(np.linalg.lstsq(X, t, rcond=None)[0], 0.0)


def fit(samples) -> CostModel:
    """samples: iterable of (work [3], seconds) or (work [3], msgs [3],
    seconds).  Columns that are zero in every sample (an algorithm never
    used, or no message counts given) keep a zero coefficient; the others
    are fitted non-negative, with the launch cost T0."""
    rows = [tuple(s) for s in samples]
    if len(rows) < 2:
        raise ValueError("need at least two samples")
    W = np.array([np.asarray(r[0], dtype=np.float64) for r in rows])
    M = np.array([np.asarray(r[1], dtype=np.float64) if len(r) == 3 else np.zeros(3) for r in rows])
    t = np.array([float(r[-1]) for r in rows])
    F = np.concatenate([W, M], axis=1)
    used = F.sum(axis=0) > 0
    # scale columns to comparable magnitudes for a well-conditioned solve
    scale = np.where(used, np.abs(F).max(axis=0), 1.0)
    X = np.concatenate([F[:, used] / scale[used], np.ones((F.shape[0], 1))], axis=1)
    coef = _nnls(X, t)
    full = np.zeros(6)
    full[used] = coef[:-1] / scale[used]
    pred = X @ coef
    ss_res = float(((t - pred) ** 2).sum())
    ss_tot = float(((t - t.mean()) ** 2).sum())
    r2 = 1.0 - ss_res / ss_tot if ss_tot > 0 else 1.0
    return CostModel(full[:3].copy(), float(coef[-1]), r2, per_msg=full[3:].copy())


def fit_chain(model: CostModel, observations) -> CostModel:
    """Calibrates the per-algorithm chain rate from served requests:
    observations are (alg, longest message length, latency seconds), e.g.
    every request of a moderately loaded run, whose latency is mostly its
    longest message's chain.  Fits latency = t0 + ops / chain_a by
    non-negative least squares (one fixed cost t0 for all requests, stored
    as `latency_t0`); algorithms without observations keep no chain term."""
    obs = [(int(a), float(shard.message_costs(np.array([L]), alg=int(a))[0]), float(lat))
           for a, L, lat in observations if lat > 0]
    chain = np.zeros(3)
    t0 = 0.0
    if obs:
        algs_seen = sorted({a for a, _, _ in obs})
        X = np.zeros((len(obs), len(algs_seen) + 1))
        y = np.zeros(len(obs))
        for i, (a, ops, lat) in enumerate(obs):
            X[i, algs_seen.index(a)] = ops
            X[i, -1] = 1.0
            y[i] = lat
        scale = np.maximum(np.abs(X).max(axis=0), 1e-30)
        coef = _nnls(X / scale, y) / scale
        for j, a in enumerate(algs_seen):
            chain[a] = 1.0 / coef[j] if coef[j] > 0 else 0.0
        t0 = float(coef[-1])
    return dataclasses.replace(model, chain=chain, latency_t0=t0)
