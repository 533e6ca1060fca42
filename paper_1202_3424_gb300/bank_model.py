"""Shared-memory bank model of the pencil-FFT exchanges; picks the row padding.

The FFT kernels stage TP pencils side by side in shared memory, element
(pos, t) of the plane at row pos, column t.  Between two radix stages every
thread stores its values at the positions the next stage's threads load
(csrc/fft.cuh, ``fft_stages``).  With TP * 8 bytes < 128 several rows share
one 128-byte bank window, and the stride patterns of those stores and loads
can put a whole half-warp on the same banks.  Inserting one padding row after
every 2^S rows (row pos stored at ``pos + (pos >> S)``) moves such rows
apart; since every exchange position is a per-thread base plus a multiple of
the radix stride, the shift folds into the constant offsets and costs almost
no address arithmetic.  This module counts the wavefronts of every exchange
instruction of every warp for each candidate S and picks the cheapest.  Its
choices are tabulated in ``exchange_pad_shift`` (csrc/fft.cuh);
``python -m paper_1202_3424_gb300.bank_model`` prints the table and
``--check`` compares it with the header.

Bank model: 32 banks of 4 bytes; a warp's 8-byte access is served in two
half-warp phases, each taking as many wavefronts as the largest number of
distinct 4-byte words any one bank must deliver (equal words broadcast).
"""
from __future__ import annotations

import os
import re
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
FFT_HEADER = os.path.join(HERE, "csrc", "fft.cuh")


def read_plans(path: str = FFT_HEADER):
    """{"Plan": {L: (NT, radices)}, "ZPlan": {...}} from the plan table of fft.cuh."""
    text = open(path).read()
    out = {"Plan": {}, "ZPlan": {}}
    for kind, L, NT, rad in re.findall(r"struct (Z?Plan)<(\d+)> : PlanDef<\d+, (\d+), ([\d, ]+)>", text):
        out[kind][int(L)] = (int(NT), [int(r) for r in rad.split(",")])
    for L, p in out["Plan"].items():
        out["ZPlan"].setdefault(L, p)
    return out


def read_table(path: str = FFT_HEADER):
    """{(L, NT, TP): S} from exchange_pad_shift in fft.cuh."""
    text = open(path).read()
    pat = r"if \(L == (\d+) && NT == (\d+) && TP == (\d+)\) return (\d+);"
    return {(int(a), int(b), int(c)): int(d) for a, b, c, d in re.findall(pat, text)}


def stage_radix(rad, direction, s):
    return rad[s] if direction < 0 else rad[len(rad) - 1 - s]


def stage_p(rad, direction, s):
    p = 1
    for i in range(s):
        p *= stage_radix(rad, direction, i)
    return p


def exchange_positions(L, NT, rad, direction):
    """Per exchange instruction: the position each thread u (0..NT-1) touches."""
    E = L // NT
    for S in range(len(rad) - 1):
        R, P = stage_radix(rad, direction, S), stage_p(rad, direction, S)
        for q in range(E // R):
            for m in range(R):
                pos = []
                for u in range(NT):
                    if NT % P == 0:
                        pos.append((u // P) * (P * R) + (u % P) + q * NT * R + m * P)
                    elif P % NT == 0:
                        pos.append(u + (q - q % (P // NT)) * NT * R + (q % (P // NT)) * NT + m * P)
                    else:
                        i = u + q * NT
                        k = i % P
                        pos.append((i - k) * R + k + m * P)
                yield pos
        R2 = stage_radix(rad, direction, S + 1)
        for q in range(E // R2):
            for j in range(R2):
                yield [u + q * NT + j * (L // R2) for u in range(NT)]


def wavefronts(byte_addrs, esize=8):
    total = 0
    phases = [byte_addrs[:16], byte_addrs[16:]] if esize == 8 else [byte_addrs]
    for ph in phases:
        banks: dict[int, set] = {}
        for a in ph:
            for w in range(esize // 4):
                word = a // 4 + w
                banks.setdefault(word % 32, set()).add(word)
        total += max((len(v) for v in banks.values()), default=0)
    return total


def padded_row(pos, shift):
    return pos + (pos >> shift) if shift else pos


def cost(L, NT, rad, TP, shift=0, groups=1):
    """(wavefronts, ideal) over both transform directions for a block of
    groups*TP*NT threads (thread -> column t = tid % TP, pencil thread
    u = (tid // TP) % NT); each group has its own plane."""
    rows = padded_row(L - 1, shift) + 1
    nthreads = groups * TP * NT
    act = ideal = 0
    for direction in (-1, +1):
        for pos in exchange_positions(L, NT, rad, direction):
            for w in range(nthreads // 32):
                addrs = []
                for lane in range(32):
                    tid = w * 32 + lane
                    t, u, g = tid % TP, (tid // TP) % NT, tid // (TP * NT)
                    addrs.append(((g * rows + padded_row(pos[u], shift)) * TP + t) * 8)
                act += wavefronts(addrs)
                ideal += 2
    return act, ideal


# Padding is kept only where it cuts the wavefronts by at least this factor.
# Measured on GB300: padding the 8-wide planes (cost 1.25 -> 1.0) made the
# register-capped schedule-0 z pass spill and run 10-13 % slower on the
# 128- and 512-point grids, while padding the 4-wide register-schedule planes
# (1.75 -> 1.0) made that z pass faster; an XOR swizzle showed the same split.
MIN_GAIN = 1.4


def best_shift(L, NT, rad, TP, groups=1):
    """(S, cost, plain cost): the cheapest padding shift if it pays
    (MIN_GAIN), else 0; ties go to the larger S (less padding)."""
    plain = cost(L, NT, rad, TP, 0, groups)
    plain = plain[0] / plain[1]
    best = (plain, 0)
    for s in range(6, 0, -1):
        a, i = cost(L, NT, rad, TP, s, groups)
        if a / i < best[0] - 1e-12:
            best = (a / i, s)
    r, s = best
    if s and plain < MIN_GAIN * r:
        return 0, plain, plain
    return s, r, plain


# Tile widths, as the kernels define them (csrc/matvec_impl.cuh) for
# complex64 elements.
def tp_strided(NT):
    tp = max(8, min(32, 256 // NT))
    return max(tp, 16)


def tp_zgroups(L, NT, table=None):
    """Schedule-0 z tile: halved until spectra (with the header's padding),
    Green tile and twiddles fit 216 KB."""
    table = read_table() if table is None else table
    tp = 256 // NT if NT >= 32 else 128 // NT
    tp = max(4, min(32, tp))
    while tp > 1:
        sh = table.get((L, NT, tp), 0)
        rows = L + ((L - 1) >> sh) if sh else L
        if ((3 * rows + 6 * (L // 2 + 1)) * tp + L) * 8 <= 216 * 1024:
            break
        tp //= 2
    return tp


def tp_zregs(NT):
    return max(4, min(32, 128 // NT))


def table(plans=None):
    """{(L, NT, TP): (S, padded cost, plain cost)} for every exchange plane of
    the three kernel families (strided passes, z groups, z registers)."""
    plans = plans or read_plans()
    out = {}
    for L, (NT, rad) in plans["Plan"].items():
        TP = tp_strided(NT)
        out[(L, NT, TP)] = best_shift(L, NT, rad, TP)
        if L // NT <= 8:
            TP = tp_zregs(NT)
            out[(L, NT, TP)] = best_shift(L, NT, rad, TP, groups=3)
    for L, (NT, rad) in plans["ZPlan"].items():
        TP = tp_zgroups(L, NT)
        out[(L, NT, TP)] = best_shift(L, NT, rad, TP, groups=3)
    return out


def main(argv):
    t = table()
    if "--check" in argv:
        want = {k: v[0] for k, v in t.items() if v[0] != 0}
        have = read_table()
        if want != have:
            print("exchange_pad_shift in fft.cuh differs from the model:")
            print("  model:", sorted(want.items()))
            print("  header:", sorted(have.items()))
            return 1
        print("exchange_pad_shift matches the model (%d padded planes)" % len(want))
        return 0
    for (L, NT, TP), (s, r, plain) in sorted(t.items()):
        print(f"L={L:4d} NT={NT:3d} TP={TP:3d}  pad shift S={s}  cost {r:.3f} of ideal (plain {plain:.3f})")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
