"""Generate ``tile_table.h``: the thread micro-tile of every specialised
kernel, chosen by a small cost model of one warp on sm_103a.

For a kernel that keeps each pair's A and B in shared memory and gives each
thread a TM x TN block of C, the model counts per pair:
  * shared-memory load instructions and the wavefronts they cost, by
    simulating the addresses one warp issues (32 banks of 4 bytes; 8-byte
    accesses in half-warps, 16-byte accesses in quarter-warps; identical
    addresses broadcast);
  * FMA instructions, including the duplicates of ragged tiles;
  * how many blocks fit an SM's shared memory (three pipeline stages of one
    compute round of pairs each, two for fp64 types) and so how many warps
    compute at once;
  * for fp64 types, the fp64 FMA pipe (2 per clock per SM), derated when
    fewer than eight warps compute;
and picks the configuration with the smallest
  max(issue cycles, shared-memory wavefronts)
under a register budget for accumulators plus fragments.  Rows and columns of
C may be assigned to threads in contiguous blocks or strided, and operands are
read with 16/8-byte vectors along whichever dimension is contiguous in shared
memory when the alignment allows it.

Run by the build when the table is missing or older than this script.
"""
from __future__ import annotations

import itertools
import os
import sys
from math import gcd

TYPES = {  # code: (element bytes, complex, fma per mac, unused)
    0: (4, False, 1, 32),   # S
    1: (8, False, 1, 16),   # D
    2: (8, True, 4, 16),    # C
    3: (16, True, 4, 8),    # Z
    4: (2, False, 1, 32),   # H
    5: (2, False, 1, 32),   # B
}
REG_LIMIT = 96                   # registers for accumulators plus fragments
STAGES = 3                       # pipeline depth of the default variant
FP64_TYPES = (1, 3)              # double and complex double: fp64-pipe bound, 2 stages
FP64_FMA_PER_CLK = 2.0           # measured fp64 FMA rate per SM per clock on GB300
SMEM_PER_SM = 227 * 1024
ISSUE_PER_CLK = 4 * 32 * 0.7     # thread-instructions per clock per SM (4 schedulers, derated)


def padded(elems, es):
    b = elems * es
    return elems + 16 // es if (b % 16 == 0 and (b // 16) % 2 == 0) else elems


def wavefronts(addrs_bytes, width):
    """Wavefronts for one warp-wide shared-memory load of `width` bytes per
    thread; addrs_bytes: 32 start addresses (None = thread inactive)."""
    group = {4: 32, 8: 16, 16: 8}.get(width, 32)
    total = 0
    for g0 in range(0, 32, group):
        banks = {}
        for a in addrs_bytes[g0:g0 + group]:
            if a is None:
                continue
            for w in range(width // 4 if width >= 4 else 1):
                word = a // 4 + w
                banks.setdefault(word % 32, set()).add(word)
        if banks:
            total += max(len(s) for s in banks.values())
    return total


def plan(code, M, N, K, TA, TB, TM, TN, SI, SJ):
    """Load plan of one thread for one l-chunk; returns None if not valid."""
    es, cplx, fpm, accbudget = TYPES[code]
    TI, TJ = -(-M // TM), -(-N // TN)
    rag_i, rag_j = TI * TM != M, TJ * TN != N
    SA_P, SB_P = padded(M * K, es), padded(K * N, es)
    # l-chunk width: operands contiguous along l (A^T stored, B stored)
    lcont = []
    if TA:
        lcont.append(SA_P)
    if not TB:
        lcont.append(SB_P)
    VL = 1
    for v in (16 // es, 8 // es, 4 // es, 2, 1):
        if v < 1 or v * es > 16:
            continue
        if K % v == 0 and all(s % v == 0 for s in lcont):
            VL = v
            break
    if not lcont:
        VL = 1
    # vector along rows for A stored as m x k (rows contiguous), along
    # columns for B stored as n x k (columns contiguous): the vector must
    # divide the block, the leading dimension and the matrix slot
    def vw(tblock, ld, slot):
        for v in (16 // es, 8 // es, 4 // es, 2, 1):
            if v >= 1 and v * es <= 16 and tblock % v == 0 and ld % v == 0 and slot % v == 0:
                return v
        return 1
    VI = vw(TM, M, SA_P) if (not TA and not SI and not rag_i) else 1
    VJ = vw(TN, N, SB_P) if (TB and not SJ and not rag_j) else 1
    words = max(1, es // 4)          # 32-bit registers per arithmetic value
    regs = (TM * TN + (TM + TN) * VL) * words
    if regs > REG_LIMIT:
        return None
    return dict(TI=TI, TJ=TJ, VL=VL, VI=VI, VJ=VJ, SA_P=SA_P, SB_P=SB_P, regs=regs,
                rag_i=rag_i, rag_j=rag_j)


def direct_store_width(es, M, N, TM, SI, rag_i):
    """Vector width (elements) for storing a thread's contiguous row block of
    a C column straight to global memory as 16-byte vectors, or 0 when rows
    are strided or ragged or the strides break 16-byte alignment."""
    if SI or rag_i:
        return 0
    SC = M * N
    v = 16 // es
    if TM % v == 0 and M % v == 0 and SC % v == 0:
        return v
    return 0


def row(ti, r, TI, TM, SI, M):
    i = ti + TI * r if SI else ti * TM + r
    return min(i, M - 1)


def cost(code, M, N, K, TA, TB, TM, TN, SI, SJ, NT):
    es, cplx, fpm, accbudget = TYPES[code]
    p = plan(code, M, N, K, TA, TB, TM, TN, SI, SJ)
    if p is None:
        return None
    TI, TJ, VL, VI, VJ = p["TI"], p["TJ"], p["VL"], p["VI"], p["VJ"]
    TPM = TI * TJ
    if TPM > NT:
        return None
    MPR = NT // TPM
    # load instructions per l-chunk per thread
    a_ins = TM if TA else VL * (-(-TM // VI))
    b_ins = TN if not TB else VL * (-(-TN // VJ))
    chunks = K // VL
    lds_thread = chunks * (a_ins + b_ins)
    fma_thread = K * TM * TN * fpm
    # simulate one warp for l0 = 0 (and l0 = VL when K > VL) -> wavefronts
    wf = 0
    threads = []
    for t in range(32):
        q, u = divmod(t, TPM)
        if q >= MPR:
            threads.append(None)
            continue
        threads.append((q, u % TI, u // TI))
    nmat_warp = max(1, len({th[0] for th in threads if th is not None}))
    frac_mat = min(1.0, 32 / TPM)   # matrices (or fraction) covered by one warp
    for l0 in sorted({0, VL % K if K > VL else 0}):
        # A loads
        if TA:
            for r in range(TM):
                addrs = [None if th is None else
                         es * (th[0] * p["SA_P"] + K * row(th[1], r, TI, TM, SI, M) + l0)
                         for th in threads]
                wf += wavefronts(addrs, VL * es)
        else:
            for dl in range(VL):
                for rg in range(0, TM, VI):
                    addrs = [None if th is None else
                             es * (th[0] * p["SA_P"] + row(th[1], rg, TI, TM, SI, M) + M * (l0 + dl))
                             for th in threads]
                    wf += wavefronts(addrs, VI * es)
        # B loads
        if not TB:
            for c in range(TN):
                addrs = [None if th is None else
                         es * (th[0] * p["SB_P"] + K * row(th[2], c, TJ, TN, SJ, N) + l0)
                         for th in threads]
                wf += wavefronts(addrs, VL * es)
        else:
            for dl in range(VL):
                for cg in range(0, TN, VJ):
                    addrs = [None if th is None else
                             es * (th[0] * p["SB_P"] + row(th[2], cg, TJ, TN, SJ, N) + N * (l0 + dl))
                             for th in threads]
                    wf += wavefronts(addrs, VJ * es)
    nsim = len({0, VL % K if K > VL else 0})
    wf_per_pair = wf / nsim * chunks * TPM / 32.0
    # epilogue: direct 16/8-byte stores of contiguous row blocks when the
    # layout allows, else scalar stores to a shared tile + coalesced copy-out
    VS = direct_store_width(es, M, N, TM, SI, p["rag_i"])
    if VS:
        epi_ins, epi_wf = TPM * TM * TN / VS, 0.0
    else:
        epi_ins = TPM * TM * TN + 2 * M * N * es / 16
        epi_wf = 2 * M * N / 32 + M * N * es / 128
    # occupancy: a block holds STAGES tiles of MPR pairs (plus an output tile
    # when C goes through shared memory); the warps of one tile compute while
    # the other stages load.  Few computing warps cannot fill the issue slots.
    quantum = 1
    for sz in (M * K, K * N, M * N):
        g = 16
        b = sz * es
        while b % g:
            g //= 2
        quantum = quantum * (16 // g) // gcd(quantum, 16 // g)
    P = MPR // quantum * quantum if MPR >= quantum else quantum
    busy = min(P, MPR) / MPR            # fraction of the round's threads with work
    bpp_in = (p["SA_P"] + p["SB_P"]) * es
    out_bpp = 0 if VS else padded(M * N, es) * es
    stages = 2 if code in FP64_TYPES else STAGES
    cta_smem = stages * P * bpp_in + P * out_bpp
    ctas = min(2048 // NT, SMEM_PER_SM // max(1, cta_smem))
    if ctas < 1:
        return None
    warps = ctas * MPR * TPM * busy / 32.0
    ipc = min(ISSUE_PER_CLK / 32.0, 0.35 * warps)      # warp-instructions per clock
    # issue: thread-instructions per pair (loads + fma + epilogue, ~20% overhead)
    ins_pair = (TPM * (lds_thread + fma_thread) + epi_ins) * 1.2
    issue_clk = ins_pair / 32.0 / ipc
    wf_total = wf_per_pair + epi_wf
    score = max(issue_clk, wf_total)
    if code in FP64_TYPES:
        # the fp64 pipe (2 FMA per clock per SM) binds; its four schedulers
        # need enough computing warps to stay busy
        fp64_clk = TPM * fma_thread / FP64_FMA_PER_CLK
        score = max(score, fp64_clk / min(1.0, warps / 8.0))
    if ctas == 1:
        # one block per SM: its barrier-separated phases leave bubbles that no
        # other block fills
        score *= 1.3
    return score, dict(p, TPM=TPM, MPR=MPR, wf=wf_total, issue=issue_clk, VS=VS, ctas=ctas)


def choose(code, M, N, K, TA, TB):
    best = None
    for NT in (128, 256):
        for TM in range(1, M + 1):
            for TN in range(1, N + 1):
                for SI, SJ in itertools.product((0, 1), (0, 1)):
                    if (SI and TM == 1) or (SJ and TN == 1):
                        continue
                    c = cost(code, M, N, K, TA, TB, TM, TN, SI, SJ, NT)
                    if c is None:
                        continue
                    score, info = c
                    # tie-break: fewer threads per matrix dividing 32 evenly
                    key = (round(score, 3), 0 if 32 % info["TPM"] == 0 or info["TPM"] % 32 == 0 else 1,
                           NT, info["TPM"])
                    if best is None or key < best[0]:
                        best = (key, dict(TM=TM, TN=TN, SI=SI, SJ=SJ, NT=NT, **info))
    return best[1]


SHAPES = [(s, s, s) for s in range(1, 17)] + [(3, 9, 3), (4, 16, 4), (16, 16, 1), (9, 16, 9), (16, 8, 16)]

# Measured replacements for the model's choice, keyed (type, M, N, K, TA, TB).
# The model sizes a block's shared memory from A and B alone; these fp64
# rectangular shapes are the FEM batches, run with beta != 0, where C is
# staged as well and the model's tiles (9x2, 2x8, 3x9: one compute round of
# 16-128 pairs) left one or two blocks per SM.  Timed on GB300 (N = 5e5,
# op(A) = T, op(B) = N, beta = 1): 1320 / 1831 / 115 us against 1407 / 2212 /
# 154 us.  The same idea measured 4% slower for 4x16x4 (2x4) and equal for
# 16x16x1 (2x8), which keep the model's choice.
MEASURED = {
    (1, 9, 16, 9, 1, 0): dict(TM=9, TN=1, SI=0, SJ=0, NT=128),
    (1, 16, 8, 16, 1, 0): dict(TM=2, TN=4, SI=0, SJ=0, NT=128),
    (1, 3, 9, 3, 1, 0): dict(TM=3, TN=3, SI=0, SJ=0, NT=128),
}


def main(out_path):
    lines = ["// Generated by gen_tiles.py: thread micro-tile per specialised kernel.",
             "// Fields: type, M, N, K, TA, TB -> TM, TN, SI (strided rows), SJ (strided",
             "// columns), NT (threads per block).  Model scores are in the comments.",
             "#pragma once", "", "namespace sbg {", "",
             "struct TileEntry { int type, m, n, k, ta, tb, tm, tn, si, sj, nt; };", "",
             "constexpr TileEntry kTileTable[] = {"]
    for code in sorted(TYPES):
        for (M, N, K) in SHAPES:
            for TA, TB in itertools.product((0, 1), (0, 1)):
                ov = MEASURED.get((code, M, N, K, TA, TB))
                if ov:
                    c = dict(ov, **cost(code, M, N, K, TA, TB, ov["TM"], ov["TN"], ov["SI"], ov["SJ"],
                                        ov["NT"])[1])
                else:
                    c = choose(code, M, N, K, TA, TB)
                lines.append(f"    {{{code}, {M}, {N}, {K}, {TA}, {TB}, {c['TM']}, {c['TN']}, {c['SI']}, "
                             f"{c['SJ']}, {c['NT']}}},  // wf {c['wf']:.1f} issue {c['issue']:.1f} "
                             f"TPM {c['TPM']} VL {c['VL']} VI {c['VI']} VJ {c['VJ']} VS {c['VS']} blocks/SM {c['ctas']}"
                             + (" (measured choice)" if ov else ""))
    lines += ["};", "",
              "constexpr TileEntry tile_for(int type, int m, int n, int k, int ta, int tb) {",
              "    for (const TileEntry& e : kTileTable)",
              "        if (e.type == type && e.m == m && e.n == n && e.k == k && e.ta == ta && e.tb == tb)",
              "            return e;",
              "    return TileEntry{type, m, n, k, ta, tb, 1, 1, 0, 0, 128};",
              "}", "", "}  // namespace sbg", ""]
    tmp = out_path + ".tmp"
    with open(tmp, "w") as f:
        f.write("\n".join(lines))
    os.replace(tmp, out_path)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)), "tile_table.h"))
