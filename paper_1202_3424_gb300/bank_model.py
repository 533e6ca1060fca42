"""Shared-memory bank model of the pencil-FFT exchanges; picks the row swizzle.

The FFT kernels stage TP pencils side by side in shared memory, element
(pos, t) of the plane at row pos, column t.  Between two radix stages every
thread stores its values at the positions the next stage's threads load
(csrc/fft.cuh, ``fft_stages``).  With TP * 8 bytes < 128 several rows share
one 128-byte bank window, and the stride patterns of those stores and loads
can put a whole half-warp on the same banks.  Storing row pos at
``pos ^ ((pos >> S) & M)`` moves such rows apart; this module counts the
wavefronts of every exchange instruction of every warp for each candidate
(S, M) and picks the cheapest.  Its choices are tabulated in
``exchange_swizzle`` (csrc/fft.cuh); ``python -m paper_1202_3424_gb300.bank_model``
prints the table and ``--check`` compares it with the header.

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
    """{(L, NT, TP): (S, M)} from exchange_swizzle in fft.cuh."""
    text = open(path).read()
    pat = r"if \(L == (\d+) && NT == (\d+) && TP == (\d+)\) return \{(\d+), (\d+)\};"
    return {(int(a), int(b), int(c)): (int(d), int(e)) for a, b, c, d, e in re.findall(pat, text)}


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


def cost(L, NT, rad, TP, swz=(0, 0), groups=1):
    """(wavefronts, ideal) over both transform directions for a block of
    groups*TP*NT threads (thread -> column t = tid % TP, pencil thread
    u = (tid // TP) % NT); each group has its own plane."""
    s, m = swz
    row = (lambda p: p ^ ((p >> s) & m)) if m else (lambda p: p)
    nthreads = groups * TP * NT
    act = ideal = 0
    for direction in (-1, +1):
        for pos in exchange_positions(L, NT, rad, direction):
            for w in range(nthreads // 32):
                addrs = []
                for lane in range(32):
                    tid = w * 32 + lane
                    t, u, g = tid % TP, (tid // TP) % NT, tid // (TP * NT)
                    addrs.append(((g * L + row(pos[u])) * TP + t) * 8)
                act += wavefronts(addrs)
                ideal += 2
    return act, ideal


def candidates():
    yield (0, 0)
    for s in range(1, 8):
        for m in (1, 3, 7):
            if m < (1 << s):
                yield (s, m)


# A swizzle adds address arithmetic to every exchange access.  Measured on
# GB300, removing a quarter of the wavefronts (plain cost 1.25 -> 1.0 on the
# 8-wide planes of the 512-point y and z passes) made those kernels ~10 %
# slower, while removing 40 % (1.75 -> 1.0 on the 4-wide register z plane)
# made the z pass 8 % faster; so a swizzle is kept only if it cuts the cost
# by this factor.
MIN_GAIN = 1.4


def best_swizzle(L, NT, rad, TP, groups=1):
    """Cheapest (S, M) if it pays (MIN_GAIN), else the identity; ties go to
    the smaller (M, S)."""
    scored = []
    for s, m in candidates():
        a, i = cost(L, NT, rad, TP, (s, m), groups)
        scored.append((a / i, m, s))
    scored.sort()
    r, m, s = scored[0]
    plain = [x for x in scored if x[1] == 0][0][0]
    if plain < MIN_GAIN * r:
        return (0, 0), plain, plain
    return (s, m), r, plain


# Tile widths, as the kernels define them (csrc/matvec_impl.cuh) for
# complex64 elements.
def tp_strided(NT):
    return max(8, min(32, 256 // NT))


def tp_zgroups(L, NT):
    tp = 256 // NT if NT >= 32 else 128 // NT
    tp = max(4, min(32, tp))
    while tp > 1 and (3 * L + 6 * (L // 2 + 1)) * tp * 8 > 200 * 1024:
        tp //= 2
    return tp


def tp_zregs(NT):
    return max(4, min(32, 128 // NT))


def table(plans=None):
    """{(L, NT, TP): ((S, M), swizzled cost, plain cost)} for every exchange plane
    of the three kernel families (strided passes, z groups, z registers)."""
    plans = plans or read_plans()
    out = {}
    for L, (NT, rad) in plans["Plan"].items():
        TP = tp_strided(NT)
        out[(L, NT, TP)] = best_swizzle(L, NT, rad, TP)
        if L // NT <= 8:
            TP = tp_zregs(NT)
            out[(L, NT, TP)] = best_swizzle(L, NT, rad, TP)
    for L, (NT, rad) in plans["ZPlan"].items():
        TP = tp_zgroups(L, NT)
        out[(L, NT, TP)] = best_swizzle(L, NT, rad, TP, groups=3)
    return out


def main(argv):
    t = table()
    if "--check" in argv:
        want = {k: v[0] for k, v in t.items() if v[0] != (0, 0)}
        have = read_table()
        if want != have:
            print("exchange_swizzle in fft.cuh differs from the model:")
            print("  model:", sorted(want.items()))
            print("  header:", sorted(have.items()))
            return 1
        print("exchange_swizzle matches the model (%d swizzled planes)" % len(want))
        return 0
    for (L, NT, TP), ((s, m), r, plain) in sorted(t.items()):
        print(f"L={L:4d} NT={NT:3d} TP={TP:3d}  swizzle (S={s}, M={m})  cost {r:.3f} of ideal (plain {plain:.3f})")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
