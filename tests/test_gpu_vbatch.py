"""GPU parity of the variable-size persistent path against the oracle's
problem-by-problem form of Eq. (1)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1304_7053_gb300 import inputs, sbgemm
from tests import gpu_helpers as H
from tests import refmath

pytestmark = pytest.mark.gpu


def vbound(dtype, desc, A, B, C, alpha, beta):
    """Per-entry bound of tests/gpu_helpers.py, problem by problem (grouped
    by shape and ops), laid out like the C arena."""
    cplx = dtype in "cz"
    out = np.zeros(C.size, dtype=np.float64)
    dec = lambda x: np.abs(H.decode(np.ascontiguousarray(x), dtype))
    Aa, Ba, Ca = dec(A), dec(B), dec(C)
    keys = {}
    for q in range(desc.shape[0]):
        keys.setdefault(tuple(int(v) for v in desc[q, :4]), []).append(q)
    u = H.U[dtype]
    for (m, n, k, fl), qs in keys.items():
        if m == 0 or n == 0:
            continue
        ta, tb = "NTC"[fl & 3], "NTC"[(fl >> 2) & 3]
        ar, ac = inputs.stored_shape(ta, m, k)
        br, bc = inputs.stored_shape(tb, k, n)
        qs = np.array(qs)
        oa, ob, oc = desc[qs, 4], desc[qs, 5], desc[qs, 6]
        ia = oa[:, None] + np.arange(m * k)[None, :]
        ib = ob[:, None] + np.arange(k * n)[None, :]
        ic = oc[:, None] + np.arange(m * n)[None, :]
        if k == 0:
            s = np.zeros((qs.size, m, n))
        else:
            Av = Aa[ia].reshape(-1, ac, ar).transpose(0, 2, 1)
            Bv = Ba[ib].reshape(-1, bc, br).transpose(0, 2, 1)
            opA = Av if ta == "N" else Av.transpose(0, 2, 1)
            opB = Bv if tb == "N" else Bv.transpose(0, 2, 1)
            s = abs(complex(alpha)) * np.matmul(opA, opB)
        if not (fl & 16) and complex(beta) != 0:
            s = s + abs(complex(beta)) * Ca[ic].reshape(-1, n, m).transpose(0, 2, 1)
        c = (2 * k + 5) if cplx else max(2 * k, k + 3)
        bd = c * u * s
        out[ic.ravel()] = bd.transpose(0, 2, 1).reshape(-1)
    return out


def run_vbatch(dtype, desc, A, B, C, alpha, beta, device_scalars=False, graph=False):
    tA, pA = H.to_dev(A)
    tB, pB = H.to_dev(B)
    tC, pC = H.to_dev(C, 64, 64)
    plan = sbgemm.VPlan(dtype, sbgemm.vproblems_from_desc(desc))
    keep = []
    if device_scalars:
        sd = {"s": np.float32, "h": np.float32, "b": np.float32, "d": np.float64,
              "c": np.complex64, "z": np.complex128}[dtype]
        ta_, pa = H.to_dev(np.array([alpha], dtype=sd))
        tb_, pb = H.to_dev(np.array([beta], dtype=sd))
        keep = [ta_, tb_]
        a_arg, b_arg = pa, pb
    else:
        a_arg, b_arg = alpha, beta
    if graph:
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        C0 = tC.clone()
        with torch.cuda.graph(g, stream=s):
            plan.run(a_arg, pA, pB, b_arg, pC, stream=s, device_scalars=device_scalars)
        for _ in range(2):          # replay twice from the same starting C
            tC.copy_(C0)
            g.replay()
    else:
        plan.run(a_arg, pA, pB, b_arg, pC, device_scalars=device_scalars)
    torch.cuda.synchronize()
    got, raw = H.from_dev(tC, C, 64)
    assert np.all(raw[:64] == 0x5A) and np.all(raw[64 + C.nbytes:] == 0x5A)
    info = plan.info()
    plan.close()
    del keep
    return got, info


def check(dtype, desc, A, B, C, alpha, beta, got, exact=False):
    ref = oracle.gemm_vbatch(dtype, desc, alpha, A, B, beta, C, threads=8)
    g = H.decode(got, dtype)
    if exact:
        bad = np.nonzero(g != ref)[0]
        assert bad.size == 0, f"not exact at {bad[:5]}"
        return
    bd = vbound(dtype, desc, A, B, C, alpha, beta)
    err = np.maximum(np.abs((g - ref).real), np.abs((g - ref).imag)) if dtype in "cz" else np.abs(g - ref)
    ratio = np.where(bd > 0, err / np.where(bd > 0, bd, 1), np.where(err > 0, np.inf, 0))
    i = int(np.argmax(ratio))
    assert ratio[i] <= 1.0, f"error {err[i]} > bound {bd[i]} at {i}"


def mixed_problems(count, seed, dtype):
    desc, la, lb, lc = inputs.vbatch_problems(count, seed=seed)
    return desc, la, lb, lc


@pytest.mark.parametrize("dtype", ["s", "d"])
def test_mixed_sizes_paper_distribution(dtype):
    """Sizes p + 1 with P(p) proportional to 1/p, beta per problem in {0, 1}."""
    desc, la, lb, lc = inputs.vbatch_problems(20000, seed=1)
    A, B, C = inputs.draw(dtype, la, 11), inputs.draw(dtype, lb, 12), inputs.draw(dtype, lc, 13)
    got, info = run_vbatch(dtype, desc, A, B, C, 1.0, 1.0)
    assert info["buckets"] == 15
    check(dtype, desc, A, B, C, 1.0, 1.0, got)
    Ai, Bi, Ci = (inputs.draw(dtype, n, s, int_valued=True) for n, s in ((la, 21), (lb, 22), (lc, 23)))
    got, _ = run_vbatch(dtype, desc, Ai, Bi, Ci, 1.5, -0.5)
    check(dtype, desc, Ai, Bi, Ci, 1.5, -0.5, got, exact=True)


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h", "b"])
def test_random_shapes_and_ops(dtype):
    """Random m, n, k in 0..16 (zeros included) and random ops: specialised
    and generic kinds in one launch."""
    count = 3000
    r = inputs.splitmix64(77, 5 * count).reshape(5, count)
    m = (r[0] % np.uint64(17)).astype(np.int64)
    n = (r[1] % np.uint64(17)).astype(np.int64)
    k = (r[2] % np.uint64(17)).astype(np.int64)
    sq = (r[3] % np.uint64(3)) == 0          # a third square N/N so kinds are hit too
    n[sq], k[sq] = m[sq], m[sq]
    ops = (r[4] % np.uint64(9)).astype(np.int64)
    opa, opb = ops // 3, ops % 3
    opa[sq], opb[sq] = 0, 0
    bz = ((r[4] >> np.uint64(8)) & np.uint64(1)).astype(np.int64)
    desc = np.zeros((count, 8), dtype=np.int64)
    desc[:, 0], desc[:, 1], desc[:, 2] = m, n, k
    desc[:, 3] = opa | (opb << 2) | (bz << 4)
    sa, sb, sc = m * k, k * n, m * n
    desc[:, 4] = np.concatenate([[0], np.cumsum(sa)[:-1]])
    desc[:, 5] = np.concatenate([[0], np.cumsum(sb)[:-1]])
    desc[:, 6] = np.concatenate([[0], np.cumsum(sc)[:-1]])
    A, B = inputs.draw(dtype, int(sa.sum()), 31), inputs.draw(dtype, int(sb.sum()), 32)
    C = inputs.draw(dtype, int(sc.sum()), 33)
    alpha, beta = (1.5 - 0.5j, -0.5 + 0.25j) if dtype in "cz" else (1.5, -0.5)
    got, _ = run_vbatch(dtype, desc, A, B, C, alpha, beta)
    if dtype in "hb":
        ref = oracle.gemm_vbatch(dtype, desc, alpha, A, B, beta, C, threads=8)
        g = H.decode(got, dtype)
        bd = (H.U16[dtype] * np.abs(ref) + (1 + H.U16[dtype]) * vbound(dtype, desc, A, B, C, alpha, beta)
              + H.SUB16[dtype])
        assert np.all(np.abs(g - ref) <= bd)
    else:
        check(dtype, desc, A, B, C, alpha, beta, got)


@pytest.mark.parametrize("dtype", ["s", "d", "z"])
def test_graph_capture_and_device_scalars(dtype):
    """Captured in a CUDA graph and replayed, and with device scalars; for
    fp64 and complex128 the plan's tensor-core record list is a second
    launch of the run."""
    desc, la, lb, lc = inputs.vbatch_problems(5000, seed=3)
    A, B, C = inputs.draw(dtype, la, 41), inputs.draw(dtype, lb, 42), inputs.draw(dtype, lc, 43)
    alpha, beta = (1.5 - 0.5j, -0.5 + 0.25j) if dtype in "cz" else (1.5, -0.5)
    got, _ = run_vbatch(dtype, desc, A, B, C, alpha, beta, graph=True)
    check(dtype, desc, A, B, C, alpha, beta, got)
    got, _ = run_vbatch(dtype, desc, A, B, C, alpha, beta, device_scalars=True)
    check(dtype, desc, A, B, C, alpha, beta, got)


def test_beta_zero_problems_never_read_c():
    desc, la, lb, lc = inputs.vbatch_problems(3000, seed=5, beta_mixed=False)
    desc[:, 3] |= 16
    A, B = inputs.draw("s", la, 51), inputs.draw("s", lb, 52)
    C = np.full(lc, np.nan, dtype=np.float32)
    got, _ = run_vbatch("s", desc, A, B, C, 1.0, 1.0)
    assert np.all(np.isfinite(got))
    check("s", desc, A, B, C, 1.0, 1.0, got)


def test_empty_plans():
    desc = np.zeros((4, 8), dtype=np.int64)
    desc[:, 0] = 0          # m = 0: no work
    desc[:, 1] = 3
    C = inputs.draw("s", 16, 1)
    got, info = run_vbatch("s", desc, np.zeros(1, np.float32), np.zeros(1, np.float32), C, 1.0, 0.0)
    assert info["tiles"] == 0 and np.array_equal(got, C)


def test_million_problems_sampled():
    """The full-size variable batch (N = 1,000,000, P(p) ~ 1/p, mixed beta),
    fp32, checked on a sample of problems the oracle computes one by one."""
    N = 1_000_000
    desc, la, lb, lc = inputs.vbatch_problems(N, seed=0)
    A, B, C = inputs.draw("s", la, 61), inputs.draw("s", lb, 62), inputs.draw("s", lc, 63)
    got, info = run_vbatch("s", desc, A, B, C, 1.0, 1.0)
    pick = np.unique((inputs.splitmix64(65, 3000) % np.uint64(N)).astype(np.int64))
    sub = desc[pick].copy()
    sizes = sub[:, 0] * sub[:, 0]
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    idx = np.concatenate([np.arange(o, o + s) for o, s in zip(desc[pick, 4], sizes)])
    sub[:, 4] = sub[:, 5] = sub[:, 6] = offs
    check("s", sub, A[idx], B[idx], C[idx], 1.0, 1.0, got[idx])


def test_tuned_window_installed_and_exact():
    """The autotuner times one plan per bucketing window, installs the
    fastest, and plans built afterwards give the oracle's result."""
    from paper_1304_7053_gb300 import selector
    desc, la, lb, lc = inputs.vbatch_problems(30000, seed=5)
    Ai, Bi, Ci = (inputs.draw("s", n, s, int_valued=True) for n, s in ((la, 31), (lb, 32), (lc, 33)))
    tA, tB, tC = (torch.from_numpy(x).cuda() for x in (Ai, Bi, Ci))
    try:
        best, times = selector.tune_vbatch("s", sbgemm.vproblems_from_desc(desc), tA, tB, tC,
                                           windows=(0, 4096, 1024), reps=3)
        assert set(times) == {0, 4096, 1024} and best in times
        assert all(t > 0 for t in times.values()) and times[best] == min(times.values())
        got, _ = run_vbatch("s", desc, Ai, Bi, Ci, 1.5, -0.5)
        check("s", desc, Ai, Bi, Ci, 1.5, -0.5, got, exact=True)
    finally:
        sbgemm.lib().sbgemm_vbatch_config(0)


ES = {"s": 4, "d": 8, "c": 8, "z": 16, "h": 2, "b": 2}


def phased_problems(dtype, reps, seed):
    """Square N/N problems of every size 1..16 with each matrix starting at
    every element offset within a 16-byte chunk (its phase), in a shuffled
    arena order with gaps between matrices; about half flagged beta = 0.
    Returns (desc, lenA, lenB, lenC)."""
    epc = 16 // ES[dtype]
    cases = np.array([(m, ph) for m in range(1, 17) for ph in range(epc) for _ in range(reps)],
                     dtype=np.int64)
    order = np.argsort(inputs.splitmix64(seed, len(cases)), kind="stable")
    cases = cases[order]
    r = inputs.splitmix64(seed + 1, 3 * len(cases)).reshape(3, -1)
    desc = np.zeros((len(cases), 8), dtype=np.int64)
    desc[:, 0] = desc[:, 1] = desc[:, 2] = cases[:, 0]
    desc[:, 3] = ((r[0] >> np.uint64(63)).astype(np.int64)) << 4
    ends = [0, 0, 0]
    for q, (m, ph) in enumerate(cases):
        for a in range(3):
            # the operand a starts at the next offset of phase ph (operand b,
            # c at phases shifted by the problem's own draw)
            want = (ph + a * int(r[1 + (a > 1), q] % np.uint64(epc))) % epc
            o = ends[a] + (want - ends[a]) % epc
            desc[q, 4 + a] = o
            ends[a] = o + m * m
    return desc, ends[0] + epc, ends[1] + epc, ends[2] + epc


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h", "b"])
def test_every_phase_every_square_kind(dtype):
    """Matrices at every 16-byte phase for every square size: the kinds that
    keep matrices in shifted slots (odd sizes of the 4- and 8-byte types,
    some 16-bit sizes) copy their middles in 16-byte chunks and their ragged
    heads and tails element by element.  Results against the oracle (exact
    on small integers for the 32- and 64-bit types), and the gaps of C
    between problems keep their values (the oracle leaves them as given)."""
    desc, la, lb, lc = phased_problems(dtype, 9, seed=91)
    Ai, Bi, Ci = (inputs.draw(dtype, n, s, int_valued=True) for n, s in ((la, 92), (lb, 93), (lc, 94)))
    cplx = dtype in "cz"
    for alpha, beta in (((1.5 - 0.5j, -0.5 + 0.25j) if cplx else (1.5, -0.5)),
                        ((0j, -0.5 + 0.25j) if cplx else (0.0, -0.5))):
        got, info = run_vbatch(dtype, desc, Ai, Bi, Ci, alpha, beta)
        assert info["buckets"] == 16
        if dtype in "hb":
            ref = oracle.gemm_vbatch(dtype, desc, alpha, Ai, Bi, beta, Ci, threads=8)
            g = H.decode(got, dtype)
            bd = (H.U16[dtype] * np.abs(ref) + (1 + H.U16[dtype]) *
                  vbound(dtype, desc, Ai, Bi, Ci, alpha, beta) + H.SUB16[dtype])
            assert np.all(np.abs(g - ref) <= bd)
        else:
            check(dtype, desc, Ai, Bi, Ci, alpha, beta, got, exact=True)
    covered = np.zeros(lc, dtype=bool)
    for q in range(desc.shape[0]):
        covered[desc[q, 6]:desc[q, 6] + desc[q, 0] ** 2] = True
    assert np.array_equal(got.view(np.uint8).reshape(lc, -1)[~covered],
                          Ci.view(np.uint8).reshape(lc, -1)[~covered])
