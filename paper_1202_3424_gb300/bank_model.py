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


# ---- warp-local pencils (x passes) ------------------------------------------
# The warp-local x passes (csrc/xwarp.cuh) hold each pencil in NT <= 32
# consecutive lanes and give it its own exchange plane of L + pad elements;
# the exchange after stage S of direction DIR stores and loads position pos
# at pos ^ ((pos >> K) & 15), with K chosen here per exchange.
XWARP_HEADER = os.path.join(HERE, "csrc", "xwarp.cuh")


def read_warp_plans(path: str = XWARP_HEADER):
    """{(L, V): (NT, radices)} from the XwPlan table of xwarp.cuh."""
    text = open(path).read()
    out = {}
    for L, V, L2, NT, rad in re.findall(r"struct XwPlan<(\d+), (\d+)> : PlanDef<(\d+), (\d+), ([\d, ]+)>", text):
        out[(int(L), int(V))] = (int(NT), [int(r) for r in rad.split(",")])
    return out


def read_warp_table(path: str = XWARP_HEADER):
    """({(L, NT, DIR, S): K}, {NT: pad}) as tabulated in xwarp.cuh."""
    text = open(path).read()
    pat = r"if \(L == (\d+) && NT == (\d+) && DIR == (-?\d+) && S == (\d+)\) return (\d+);"
    keys = {(int(a), int(b), int(c), int(d)): int(e) for a, b, c, d, e in re.findall(pat, text)}
    pads = {int(a): int(b) for a, b in re.findall(r"if \(NT == (\d+)\) return (\d+);", text)}
    return keys, pads


def warp_exchange_instrs(L, NT, rad, direction, S):
    """(store instructions, load instructions) of the exchange after stage S;
    each instruction lists the position of every pencil thread u."""
    stores = [p for i, p in enumerate(_stage_instrs(L, NT, rad, direction, S, stores=True))]
    loads = [p for p in _stage_instrs(L, NT, rad, direction, S, stores=False)]
    return stores, loads


def _stage_instrs(L, NT, rad, direction, S, stores):
    E = L // NT
    if stores:
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
    else:
        R2 = stage_radix(rad, direction, S + 1)
        for q in range(E // R2):
            for j in range(R2):
                yield [u + q * NT + j * (L // R2) for u in range(NT)]


def warp_swizzle(pos, key):
    return pos ^ ((pos >> key) & 15) if key else pos


def warp_exchange_cost(L, NT, rad, direction, S, key, plane):
    """(wavefronts, ideal) of one exchange for one warp (32 // NT pencils)."""
    act = ideal = 0
    st, ld = warp_exchange_instrs(L, NT, rad, direction, S)
    for instr in st + ld:
        addrs = [((lane // NT) * plane + warp_swizzle(instr[lane % NT], key)) * 8 for lane in range(32)]
        act += wavefronts(addrs)
        ideal += 2
    return act, ideal


WARP_PADS = (0, 8, 16, 24)


def warp_table(plans=None):
    """({(L, NT, DIR, S): K}, {NT: pad}, {(L, NT): (cost, plain cost)}): per
    exchange the key K (0: none) with the fewest wavefronts, ties to the
    smaller K; per pencil width NT the plane padding that is cheapest summed
    over every plan of that width."""
    plans = plans or read_warp_plans()
    by_nt = {}
    for (L, V), (NT, rad) in plans.items():
        by_nt.setdefault(NT, []).append((L, rad))
    keys, pads, costs = {}, {}, {}
    for NT, lst in sorted(by_nt.items()):
        best = None
        for pad in WARP_PADS:
            tot, ks, cs = 0, {}, {}
            for L, rad in lst:
                a_sum = i_sum = p_sum = 0
                for direction in (-1, +1):
                    for S in range(len(rad) - 1):
                        cands = []
                        for key in range(0, 7):
                            a, i = warp_exchange_cost(L, NT, rad, direction, S, key, L + pad)
                            cands.append((a, key, i))
                        a, key, i = min(cands)
                        ks[(L, NT, direction, S)] = key
                        a_sum += a
                        i_sum += i
                        p_sum += cands[0][0]
                cs[(L, NT)] = (a_sum / i_sum if i_sum else 1.0, p_sum / i_sum if i_sum else 1.0)
                tot += a_sum
            if best is None or tot < best[0]:
                best = (tot, pad, ks, cs)
        _, pad, ks, cs = best
        pads[NT] = pad
        keys.update(ks)
        costs.update(cs)
    return keys, pads, costs


def main(argv):
    t = table()
    if "--check-warp" in argv:
        keys, pads, costs = warp_table()
        want = {k: v for k, v in keys.items() if v}
        have, have_pads = read_warp_table()
        if want != have or pads != have_pads:
            print("warp_swizzle_key / warp_plane_pad in xwarp.cuh differ from the model:")
            print("  model:", sorted(want.items()), pads)
            print("  header:", sorted(have.items()), have_pads)
            return 1
        print("xwarp.cuh tables match the model (%d swizzled exchanges)" % len(want))
        return 0
    if "--warp" in argv:
        keys, pads, costs = warp_table()
        for (L, NT), (c, p) in sorted(costs.items()):
            print(f"L={L:4d} NT={NT:3d} pad {pads[NT]:2d}  cost {c:.3f} of ideal (unswizzled {p:.3f})")
        for k, v in sorted(keys.items()):
            if v:
                print(f"    if (L == {k[0]} && NT == {k[1]} && DIR == {k[2]} && S == {k[3]}) return {v};")
        for nt, pad in sorted(pads.items()):
            print(f"    if (NT == {nt}) return {pad};")
        return 0
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
