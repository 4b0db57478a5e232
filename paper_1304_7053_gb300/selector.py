"""Autotuner and learned variant selector.

The autotuner times every kernel variant of a problem class with the
library's native timing core (``sbgemm_time_variant``: CUDA events, L2
evicted before every call, the mean of the calls within 2 us of their
median) and appends the times to a JSONL timing database keyed by device, shape and variant; a resumed run skips rows it
already has.  The exhaustive choice per class is the fastest measured
variant.

The launch shapes of the batched paths are tuned the same way, exhaustively
on the batch at hand: the bucketing window of a variable-size plan
(``tune_vbatch``) and the grouped call's threads x stage bytes x depth
(``tune_grouped``).

The learned selector is a 3-layer perceptron (``sbgemm_mlp_*`` kernels,
fp32) that maps problem features to one predicted log-time per variant,
relative to the class's mean variant.  It is trained on the database with
the library's own forward, backward and Adam kernels.  At selection time
the valid variant with the smallest prediction wins if it is predicted to
beat the library's built-in rule by more than a trust margin; the margin is
picked per storage type on out-of-fold predictions (networks that did not
see the classes they are judged on), so the network is switched off for a
type where it does not beat the rule.  The choices go to the library as a
selection table or as the network itself (the MODEL selector mode).
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import numpy as np

from . import inputs, sbgemm

DTYPES = ["s", "d", "c", "z", "h", "b"]
NFEAT = 16
NVAR = 9          # variants of specialised shapes; generic shapes have fewer
HIDDEN = 64
# L2 penalty on the network's parameters.  Without it the network fits the
# few hundred training classes almost exactly and generalises worse than the
# library's built-in rule (held-out mean regret 3.0% against 2.5%, with
# absolute log-time targets); with 5e-3 it reached 1.9% on the held-out
# classes and 1.6% against 2.05% with the training and held-out sets swapped.
L2_PENALTY = 5e-3
TORCH_DT = {"s": "float32", "d": "float64", "c": "float32", "z": "float64",
            "h": "float16", "b": "bfloat16"}


def features(dtype, m, n, k, ta, tb, conj, beta0, N) -> np.ndarray:
    f = np.zeros(NFEAT, dtype=np.float32)
    f[0], f[1], f[2] = m / 16.0, n / 16.0, k / 16.0
    f[3] = (math.log10(max(1, N)) - 4.5) / 1.5
    f[4 + DTYPES.index(dtype)] = 1.0
    f[10], f[11], f[12], f[13] = float(ta), float(tb), float(conj), float(beta0)
    f[14] = 1.0 if sbgemm.num_variants(dtype, m, n, k) > 3 else 0.0
    f[15] = (m * n * k) ** (1.0 / 3.0) / 16.0
    return f


def size_class(N: int) -> int:
    c = 0
    while N >= 10 and c < 7:
        N //= 10
        c += 1
    return c


# ---------------------------------------------------------------- timing DB

class TimingDB:
    """Append-only JSONL file of measured variant times."""

    def __init__(self, path: str | None):
        self.path = path
        self.rows: list[dict] = []
        if path and os.path.exists(path):
            with open(path) as f:
                self.rows = [json.loads(l) for l in f if l.strip()]
        self._keys = {self.key(r) for r in self.rows}

    @staticmethod
    def key(r):
        return (r["device"], r["dtype"], r["m"], r["n"], r["k"], r["ta"], r["tb"], r["conj"],
                r["beta0"], r["N"], r["variant"])

    def has(self, r) -> bool:
        return self.key(r) in self._keys

    def add(self, r: dict) -> None:
        self.rows.append(r)
        self._keys.add(self.key(r))
        if self.path:
            with open(self.path, "a") as f:
                f.write(json.dumps(r) + "\n")


def device_name() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}/{p.multi_processor_count}sm"


class Tuner:
    """Times every variant of a problem class on the current GPU."""

    def __init__(self, db: TimingDB, reps: int = 5, flush_bytes: int = 256 << 20,
                 max_bytes: int = 16 * 256 * 1_000_000):
        import torch
        self.torch = torch
        self.db = db
        self.reps = reps
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.flush = torch.empty(flush_bytes, dtype=torch.uint8, device=self.dev)
        self.stream = torch.cuda.current_stream(self.dev)
        self.name = device_name()
        # one set of operand buffers for every class, refilled with
        # uniform[-1, 1) values of the element width the class reads
        # (``TORCH_DT``).  The values matter: the fp64 tensor-core kernel
        # recomputes with fp64 FMAs every entry whose accuracy its digit
        # split cannot guarantee, which fp32 bit patterns read as doubles
        # (wildly spread exponents) trigger often.
        n = (max_bytes + 7) // 8 * 8
        self.pool = [torch.empty(n, dtype=torch.uint8, device=self.dev) for _ in range(3)]
        self._fill = None
        self.max_bytes = max_bytes

    def _buffers(self, dtype, m, n, k, ta, tb, N):
        ar, ac = inputs.stored_shape("T" if ta else "N", m, k)
        br, bc = inputs.stored_shape("T" if tb else "N", k, n)
        es = inputs.ELEM_BYTES[dtype]
        need = es * N * max(ar * ac, br * bc, m * n)
        if need > self.max_bytes:
            raise ValueError("problem class larger than the tuner's buffers")
        fam = TORCH_DT[dtype]
        if self._fill != fam:
            torch = self.torch
            g = torch.Generator(device=self.dev)
            g.manual_seed(3 + sorted(set(TORCH_DT.values())).index(fam))
            for t in self.pool:
                t.view(getattr(torch, fam)).uniform_(-1.0, 1.0, generator=g)
            self._fill = fam
        return tuple(self.pool), (max(1, ar), ar * ac, max(1, br), br * bc, max(1, m), m * n)

    def time_class(self, dtype, m, n, k, ta, tb, conj, beta0, N) -> list[float]:
        """Median ms of every variant; cached in (and read from) the DB."""
        nv = sbgemm.num_variants(dtype, m, n, k)
        out = [None] * nv
        base = dict(device=self.name, dtype=dtype, m=m, n=n, k=k, ta=int(ta), tb=int(tb),
                    conj=int(conj), beta0=int(beta0), N=int(N))
        todo = []
        for v in range(nv):
            r = dict(base, variant=v)
            hit = [x for x in self.db.rows if TimingDB.key(x) == TimingDB.key(dict(r, ms=0))] \
                if self.db.has(r) else []
            if hit:
                out[v] = hit[-1]["ms"]
            else:
                todo.append(v)
        if not todo:
            return out
        (A, B, C), (lda, lda2, ldb, ldb2, ldc, ldc2) = self._buffers(dtype, m, n, k, ta, tb, N)
        opa = ("C" if conj else "T") if ta else "N"
        opb = ("C" if conj else "T") if tb else "N"
        ab = sbgemm._scalar_buf(dtype, 1.5)
        bb = sbgemm._scalar_buf(dtype, 0.0 if beta0 else -0.5)
        L = sbgemm.lib()
        ms = ctypes.c_float()
        for v in todo:
            st = L.sbgemm_time_variant(sbgemm.TYPE_CODES[dtype], opa.encode(), opb.encode(), m, n, k,
                                       ctypes.addressof(ab), A.data_ptr(), lda, lda2, B.data_ptr(),
                                       ldb, ldb2, ctypes.addressof(bb), C.data_ptr(), ldc, ldc2,
                                       N, v, self.reps, self.flush.data_ptr(), self.flush.numel(),
                                       self.stream.cuda_stream, ctypes.byref(ms))
            if st != 0:
                raise sbgemm.SbgemmError(st, "time_variant")
            out[v] = float(ms.value)
            self.db.add(dict(base, variant=v, ms=out[v]))
        return out


# ---------------------------------------------------------------- launch-shape tuning

def _time_calls(fn, reps: int, stream) -> float:
    """Median CUDA-event time (ms) of fn() on `stream` after one warm call."""
    import torch
    ts = []
    with torch.cuda.stream(stream):
        fn()
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


WHOLE_BATCH = 1 << 30     # a bucketing window that holds any batch


def tune_vbatch(dtype: str, problems, A, B, C, alpha=1.0, beta=1.0,
                windows=(WHOLE_BATCH, 262144, 65536, 16384), reps=5, stream=None):
    """Exhaustive tuning of a variable-size batch's bucketing window: one
    plan per window, `reps` timed runs each; the fastest window is installed
    process-wide (``sbgemm_vbatch_config``) for the plans created after this
    call.  Returns (best window, {window: ms}); ``WHOLE_BATCH`` buckets the
    whole batch at once.  C is overwritten by the trial runs."""
    import torch
    stream = stream or torch.cuda.current_stream()
    L = sbgemm.lib()
    times = {}
    try:
        for w in windows:
            L.sbgemm_vbatch_config(w)
            plan = sbgemm.VPlan(dtype, problems)
            try:
                times[w] = _time_calls(lambda: plan.run(alpha, A, B, beta, C, stream=stream),
                                       reps, stream)
            finally:
                plan.close()
    finally:
        L.sbgemm_vbatch_config(0)
    best = min(times, key=times.get)
    L.sbgemm_vbatch_config(best)
    return best, times


def tune_grouped(dtype: str, call, configs=None, reps=20, stream=None):
    """Exhaustive tuning of the grouped launch configuration for one set of
    batches: `call()` issues the grouped call on `stream`; every (threads,
    stage bytes, stages) candidate is timed and the fastest is installed
    (``sbgemm_grouped_config``).  Returns (best config, {config: ms})."""
    import torch
    stream = stream or torch.cuda.current_stream()
    if configs is None:
        configs = [(t, sb, st) for t in (128, 256) for sb in (16384, 20480, 24576, 28672, 32768, 40960)
                   for st in (2, 3) if st * sb + sb // 2 <= 220 * 1024]
    times = {}
    for cfg in configs:
        sbgemm.grouped_config(dtype, *cfg)
        times[cfg] = _time_calls(call, reps, stream)
    best = min(times, key=times.get)
    sbgemm.grouped_config(dtype, *best)
    return best, times


def random_classes(count: int, seed: int, dtypes=("s", "d", "c", "z", "h", "b"),
                   square_frac: float = 0.5):
    """Random problem classes: m, n, k in 1..16 (half of them square or one of
    the specialised rectangular shapes), N log-uniform in 1e3..1e6, random
    dtype, ops and beta == 0."""
    rect = [(3, 9, 3), (4, 16, 4), (16, 16, 1), (9, 16, 9), (16, 8, 16)]
    r = inputs.splitmix64(seed, 10 * count).reshape(count, 10)
    u = (r >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    out = []
    for i in range(count):
        if u[i, 0] < square_frac:
            if u[i, 1] < 0.8:
                s = 1 + int(u[i, 2] * 16)
                m = n = k = s
            else:
                m, n, k = rect[int(u[i, 2] * len(rect))]
        else:
            m, n, k = (1 + int(u[i, j] * 16) for j in (3, 4, 5))
        N = int(round(10 ** (3 + 3 * u[i, 6])))
        dtype = dtypes[int(u[i, 7] * len(dtypes))]
        ta, tb = int(u[i, 8] * 2), int(u[i, 9] * 2)
        conj = int(dtype in "cz" and (int(r[i, 0]) & 1) == 1)
        beta0 = int((int(r[i, 1]) >> 3) & 1)
        out.append((dtype, m, n, k, ta, tb, conj, beta0, N))
    return out


# ---------------------------------------------------------------- the network

class CostModel:
    """The MLP, trained and evaluated with the library's CUDA kernels."""

    def __init__(self, F=NFEAT, H=HIDDEN, V=NVAR, seed=0):
        import torch
        self.torch = torch
        self.F, self.H, self.V = F, H, V
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.n = int(sbgemm.lib().sbgemm_mlp_param_count(F, H, V))
        p = np.zeros(self.n, dtype=np.float32)
        d = inputs.uniform(seed, H * F + H * H + V * H)
        # weights uniform with variance 1/fan_in, biases 0
        p[:H * F] = d[:H * F] * math.sqrt(3.0 / F)
        o = H * F + H
        p[o:o + H * H] = d[H * F:H * F + H * H] * math.sqrt(3.0 / H)
        o += H * H + H
        p[o:o + V * H] = d[H * F + H * H:] * math.sqrt(3.0 / H)
        self.params = torch.from_numpy(p).to(self.dev)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self.mu = None
        self.sd = None

    def _check(self, st, where):
        if st != 0:
            raise sbgemm.SbgemmError(st, where)

    def forward(self, X):
        torch = self.torch
        X = X.contiguous()
        B = X.shape[0]
        Y = torch.empty(B, self.V, device=self.dev)
        work = torch.empty(4 * B * self.H, device=self.dev)
        s = torch.cuda.current_stream().cuda_stream
        self._check(sbgemm.lib().sbgemm_mlp_forward(self.F, self.H, self.V, self.params.data_ptr(),
                                                    X.data_ptr(), B, Y.data_ptr(), work.data_ptr(), s),
                    "mlp_forward")
        return Y, work

    def step(self, X, T, mask, lr=3e-3, l2=0.0):
        """One full-batch training step (Adam with an L2 penalty l2 on every
        parameter); returns the loss (device tensor)."""
        torch = self.torch
        B = X.shape[0]
        Y, work = self.forward(X)
        work2 = torch.empty(B * (self.V + 2 * self.H), device=self.dev)
        loss = torch.empty(2, device=self.dev)
        s = torch.cuda.current_stream().cuda_stream
        L = sbgemm.lib()
        self._check(L.sbgemm_mlp_backward(self.F, self.H, self.V, self.params.data_ptr(),
                                          X.data_ptr(), B, Y.data_ptr(), T.data_ptr(),
                                          mask.data_ptr(), work.data_ptr(), self.grads.data_ptr(),
                                          work2.data_ptr(), loss.data_ptr(), s), "mlp_backward")
        self.t += 1
        self._check(L.sbgemm_mlp_adam(self.n, self.params.data_ptr(), self.grads.data_ptr(),
                                      self.m.data_ptr(), self.v.data_ptr(), self.t, lr, 0.9, 0.999,
                                      1e-8, l2, s), "mlp_adam")
        return loss

    # -------- training on timing data
    def fit(self, feats: np.ndarray, times: np.ndarray, steps=2000, lr=3e-3, l2=L2_PENALTY):
        """feats: (B, F); times: (B, V) ms with NaN where a variant was not
        timed.  The targets are each class's log-times relative to the mean
        over its own timed variants, scaled by their root mean square: a
        choice compares the variants of one class only, and the class's
        overall time (which spans orders of magnitude with N and the shape)
        would otherwise take the network's capacity.  Classes with a single
        variant carry no choice and are left out.  ``l2`` penalises the
        parameters (see ``L2_PENALTY``)."""
        torch = self.torch
        ok = np.isfinite(times)
        lt = np.log(np.where(ok, times, 1.0))
        mask = (ok & (ok.sum(axis=1, keepdims=True) > 1)).astype(np.float64)
        cnt = np.maximum(mask.sum(axis=1, keepdims=True), 1.0)
        rel = (lt - (lt * mask).sum(axis=1, keepdims=True) / cnt) * mask
        self.mu = 0.0
        self.sd = float(np.sqrt((rel ** 2).sum() / mask.sum())) if mask.sum() > 0 else 1.0
        self.sd = self.sd or 1.0
        T = torch.from_numpy((rel / self.sd).astype(np.float32)).to(self.dev)
        X = torch.from_numpy(feats.astype(np.float32)).to(self.dev)
        Mk = torch.from_numpy(mask.astype(np.float32)).to(self.dev)
        hist = []
        for i in range(steps):
            loss = self.step(X, T, Mk, lr, l2)
            if i % 100 == 0 or i == steps - 1:
                hist.append(float(loss[0].item()))
        return hist

    def predict_rel(self, feats: np.ndarray) -> np.ndarray:
        """Predicted time of every variant relative to the class's mean
        variant (only ratios within a row are meaningful)."""
        X = self.torch.from_numpy(feats.astype(np.float32)).to(self.dev)
        Y, _ = self.forward(X)
        return np.exp(Y.cpu().numpy().astype(np.float64) * self.sd + self.mu)

    def host_params(self) -> np.ndarray:
        return self.params.cpu().numpy().astype(np.float32)

    def install(self, margins=0.0) -> None:
        """Hand the trained network to the library as its cost model (the
        library then evaluates it per class with its own forward kernel and
        consults it under the MODEL selector mode); ``margins``: one trust
        margin, or one per storage type (``sbgemm.margin_array``)."""
        if self.mu is None:
            raise RuntimeError("the network has not been fitted")
        sbgemm.set_cost_model(self.F, self.H, self.V, self.host_params(), self.mu, self.sd, margins)

    def save(self, path: str, margins=0.0) -> None:
        """Install the network and write it to a versioned cost-model file
        that any process can load (``sbgemm_load_cost_model`` or the
        SBGEMM_COST_MODEL environment setting)."""
        self.install(margins)
        sbgemm.save_cost_model(path)

    def choose(self, feats: np.ndarray, nvalid: np.ndarray, margins=0.0,
               defaults: np.ndarray | None = None, dtypes=None) -> np.ndarray:
        """The library's rule on this network's predictions (``rule_choice``);
        ``margins`` a number or a mapping from dtype letter to margin (then
        ``dtypes`` gives each class's dtype)."""
        dflt = np.zeros(len(feats), dtype=np.int64) if defaults is None else defaults
        return rule_choice(self.predict_rel(feats), nvalid, row_margins(margins, dtypes, len(feats)),
                           dflt)


def row_margins(margins, dtypes, count: int) -> np.ndarray:
    """One trust margin per class from a number or a dtype -> margin map."""
    if isinstance(margins, dict):
        return np.array([margins.get(d, 0.0) for d in dtypes], dtype=np.float64)
    return np.full(count, float(margins))


def rule_choice(pred: np.ndarray, nvalid: np.ndarray, margin: np.ndarray,
                dflt: np.ndarray) -> np.ndarray:
    """The selection rule the library applies to the cost model's outputs:
    the valid variant (index < nvalid) with the smallest predicted time,
    unless it is not predicted to beat the class's default variant by more
    than the class's margin (a fraction; 1 never overrides): then the
    default."""
    idx = np.arange(pred.shape[1])[None, :]
    pred = np.where(idx < nvalid[:, None], pred, np.inf)
    best = np.argmin(pred, axis=1)
    rows = np.arange(len(best))
    gain = pred[rows, best] < pred[rows, dflt] * (1.0 - margin)
    return np.where(gain, best, dflt)


def default_choices(classes) -> np.ndarray:
    """The library's built-in choice for each class (``sbgemm_default_variant``:
    the tensor-core variant of the 16-bit types at m = n = k = 8, 16 and of
    fp64 at large shapes; variant 2 for complex64 and for fp32 below 1e6
    pairs; variant 0 otherwise)."""
    return np.array([sbgemm.default_variant(c[0], c[1], c[2], c[3], c[7], size_class(c[8]))
                     for c in classes], dtype=np.int64)


def table_from_db(rows):
    """Group DB rows into (class, times[NVAR]) with NaN for missing variants."""
    by = {}
    for r in rows:
        key = (r["dtype"], r["m"], r["n"], r["k"], r["ta"], r["tb"], r["conj"], r["beta0"], r["N"])
        by.setdefault(key, np.full(NVAR, np.nan))[r["variant"]] = r["ms"]
    return by


def regret(times: np.ndarray, chosen: np.ndarray) -> np.ndarray:
    """t(chosen) / t(best) - 1 per class."""
    best = np.nanmin(times, axis=1)
    return times[np.arange(times.shape[0]), chosen] / best - 1.0


# candidate trust margins; 1.0 keeps the default rule for the whole type
MARGINS = (0.0, 0.02, 0.05, 0.1, 0.2, 1.0)
FOLDS = 4


def pick_margins(pred: np.ndarray, times: np.ndarray, nvalid: np.ndarray, dflt: np.ndarray,
                 dtypes) -> dict:
    """Per storage type, the margin of ``MARGINS`` whose choices (``rule_choice``
    on the predictions ``pred``) give the smallest total measured time over
    that type's classes; ties go to the larger margin.  ``pred`` must come
    from networks that did not see the classes (``out_of_fold``): on its own
    training classes a network looks better than it is."""
    dtypes = np.asarray(dtypes)
    out = {}
    for d in sorted(set(dtypes.tolist())):
        rows = np.where(dtypes == d)[0]
        total = {}
        for mg in MARGINS:
            ch = rule_choice(pred[rows], nvalid[rows], np.full(len(rows), mg), dflt[rows])
            total[mg] = float(np.nansum(times[rows, ch]))
        out[d] = min(MARGINS, key=lambda mg: (total[mg], -mg))
    return out


def out_of_fold(feats: np.ndarray, times: np.ndarray, folds=FOLDS, seed=0, steps=3000) -> np.ndarray:
    """Predicted relative times of every class from a network trained on the
    other folds (class i in fold i mod ``folds``)."""
    pred = np.full(times.shape, np.nan)
    fold = np.arange(len(feats)) % folds
    for f in range(folds):
        tr = fold != f
        net = CostModel(seed=seed + 1 + f)
        net.fit(feats[tr], times[tr], steps=steps)
        pred[~tr] = net.predict_rel(feats[~tr])
    return pred


def learn(feats, times, nvalid, dflt, dtypes, seed=0, steps=3000, folds=FOLDS):
    """The learned selector: per-type trust margins from out-of-fold
    predictions on the training classes, then one network trained on all of
    them.  Returns (network, margins, training-loss history)."""
    margins = pick_margins(out_of_fold(feats, times, folds, seed, steps), times, nvalid, dflt,
                           dtypes)
    net = CostModel(seed=seed)
    hist = net.fit(feats, times, steps=steps)
    return net, margins, hist


def evaluate(n_train_timings=2000, n_test=500, seed=11, reps=9, steps=3000, db_path=None,
             dtypes=("s", "d", "c", "z", "h", "b"), install_choices=False, log=print):
    """Collect autotuner timings for random problem classes until about
    `n_train_timings` (class, variant) rows exist for training, time every
    variant of `n_test` held-out classes, train the network, and report its
    selection regret against the exhaustive choice and the default variant."""
    import time as _time
    t0 = _time.time()
    db = TimingDB(db_path)
    tuner = Tuner(db, reps=reps)
    train, count, i = [], 0, 0
    pool = random_classes(4 * n_train_timings, seed, dtypes)
    while count < n_train_timings and i < len(pool):
        c = pool[i]
        i += 1
        train.append(c)
        count += sbgemm.num_variants(c[0], c[1], c[2], c[3])
    test = random_classes(n_test, seed + 1, dtypes)

    def table(classes):
        F = np.stack([features(*c) for c in classes])
        T = np.full((len(classes), NVAR), np.nan)
        nv = np.zeros(len(classes), dtype=np.int64)
        for j, c in enumerate(classes):
            t = tuner.time_class(*c)
            T[j, :len(t)] = t
            nv[j] = len(t)
        return F, T, nv

    Ftr, Ttr, nvtr = table(train)
    t1 = _time.time()
    Fte, Tte, nvte = table(test)
    t2 = _time.time()
    dtr, dte = default_choices(train), default_choices(test)
    ttr, tte = [c[0] for c in train], [c[0] for c in test]
    net, margins, hist = learn(Ftr, Ttr, nvtr, dtr, ttr, seed=seed, steps=steps)
    t3 = _time.time()
    chosen0 = net.choose(Fte, nvte, 0.0, dte)
    chosen = net.choose(Fte, nvte, margins, dte, tte)
    r_mlp = regret(Tte, chosen)
    r_def = regret(Tte, dte)
    # the method without any selection: one kernel per shape (variant 0)
    plain = np.zeros(len(test), dtype=np.int64)
    r_plain = regret(Tte, plain)
    multi = nvte > 1
    rep = {
        "device": tuner.name,
        "train_classes": len(train), "train_timings": int(np.isfinite(Ttr).sum()),
        "test_classes": len(test), "test_timings": int(np.isfinite(Tte).sum()),
        "test_classes_with_choice": int(multi.sum()),
        "loss_first": hist[0], "loss_last": hist[-1], "train_steps": steps,
        "l2_penalty": L2_PENALTY,
        "regret_mlp_mean": float(r_mlp.mean()), "regret_mlp_median": float(np.median(r_mlp)),
        "regret_mlp_p90": float(np.percentile(r_mlp, 90)),
        "regret_default_mean": float(r_def.mean()), "regret_default_median": float(np.median(r_def)),
        "regret_default_p90": float(np.percentile(r_def, 90)),
        "regret_mlp_mean_multi": float(r_mlp[multi].mean()) if multi.any() else 0.0,
        "regret_default_mean_multi": float(r_def[multi].mean()) if multi.any() else 0.0,
        "regret_plain_mean": float(r_plain.mean()),
        "mlp_picks_best": float((r_mlp == 0).mean()),
        "default_is_best": float((r_def == 0).mean()),
        "default_definition": "the library without a selection table (the tensor-core "
                              "variant for 16-bit m = n = k = 8, 16 and for fp64 at large "
                              "shapes; variant 2 for complex64 and for fp32 below 1e6 pairs; "
                              "variant 0 otherwise)",
        "plain_definition": "variant 0 for every class (one kernel per shape, no selection)",
        "trust_margins": margins, "folds": FOLDS,
        "regret_mlp_no_margin_mean": float(regret(Tte, chosen0).mean()),
        "time_mlp_no_margin_total_ms": float(Tte[np.arange(len(test)), chosen0].sum()),
        "time_mlp_total_ms": float(Tte[np.arange(len(test)), chosen].sum()),
        "time_default_total_ms": float(Tte[np.arange(len(test)), dte].sum()),
        "time_plain_total_ms": float(Tte[np.arange(len(test)), plain].sum()),
        "time_exhaustive_total_ms": float(np.nanmin(Tte, axis=1).sum()),
        "seconds": {"tune_train": round(t1 - t0, 1), "tune_test": round(t2 - t1, 1),
                    "train_network": round(t3 - t2, 1)},
    }
    if install_choices:
        install(test, chosen)
    log(json.dumps(rep))
    return rep, net


def install(classes, choices, path: str | None = None) -> None:
    """Write choices into the library's selection table, and the whole table
    to `path` when given (loadable by any process: ``sbgemm_load_table`` or
    the SBGEMM_TABLE environment setting)."""
    for (dtype, m, n, k, ta, tb, conj, beta0, N), v in zip(classes, choices):
        sbgemm.set_choice(dtype, m, n, k, ta, tb, beta0, size_class(N), int(v))
    if path:
        sbgemm.save_table(path)


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-timings", type=int, default=2000)
    ap.add_argument("--test", type=int, default=500)
    ap.add_argument("--db", default=None)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    rep, _ = evaluate(a.train_timings, a.test, seed=a.seed, db_path=a.db)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rep, f, indent=1)
