"""Index algebra of the two-pair FFT kernel's one-dimensional passes (CPU).

fft_x2_kernel stores element e of a table at shared-memory slot
swz(e) = e ^ ((e >> 3) & 7). Its one-dimensional passes take the span H = 2^LH
as a compile-time constant and use shortcuts for the slots of a group
e0 + t H (e0 = (g >> LH) << (LH + RL) | o, o < H), valid only for some
(RL, LH). This restates those shortcuts and checks them against swz for every
pass the kernel issues on tables of 2 to 2^12 points, and that each pass visits
every slot exactly once; the device results themselves are covered by the GPU
parity tests.
"""


def swz(e):
    return e ^ ((e >> 3) & 7)


def slots(rl, lh, e0):
    r = 1 << rl
    if lh >= 6:  # bits 0..5 of e0 + t H are those of e0
        a0 = swz(e0)
        return [a0 + t * (1 << lh) for t in range(r)]
    if lh == 3 and rl == 3:  # bits 3..5 of e0 + 8 t are t
        return [(e0 ^ t) + 8 * t for t in range(r)]
    if lh == 0 and rl == 3:  # e0 = 8 g: bits 3..5 are g & 7
        b = e0 ^ ((e0 >> 3) & 7)
        return [b ^ t for t in range(r)]
    return [swz(e0 + t * (1 << lh)) for t in range(r)]


def passes(ln):
    """(radix log, span log) of the passes of a 2^ln-point table, forward order."""
    full, rem = ln // 3, ln % 3
    if full == 0:
        return [(rem, 0)]
    out = [(rem, ln - rem)] if rem else []
    out += [(3, ln - rem - 3 * (k + 1)) for k in range(full - 1)]
    return out + [(3, 0)]


def test_slot_shortcuts_equal_the_swizzle():
    checked = 0
    for ln in range(1, 13):
        for rl, lh in passes(ln):
            h = 1 << lh
            seen = set()
            for g in range(1 << (ln - rl)):
                e0 = ((g >> lh) << (lh + rl)) + (g & (h - 1))
                got = slots(rl, lh, e0)
                assert got == [swz(e0 + t * h) for t in range(1 << rl)], (ln, rl, lh, g)
                seen.update(got)
                checked += 1
            assert seen == set(range(1 << ln)), (ln, rl, lh)
    assert checked > 4000


def test_the_span_8_shortcut_needs_radix_8():
    # the kernel issues radix-2/4 passes at span 8 only on tables of 2^4 and 2^5 points,
    # where bit 5 of e0 is zero and the shortcut would also hold; for a radix-4 pass at
    # span 8 in a larger table (bit 5 of e0 from g) it does not, hence the radix-8 condition
    rl, lh, ln = 2, 3, 6
    bad = 0
    for g in range(1 << (ln - rl)):
        e0 = ((g >> lh) << (lh + rl)) + (g & 7)
        if [(e0 ^ t) + 8 * t for t in range(4)] != [swz(e0 + 8 * t) for t in range(4)]:
            bad += 1
    assert bad > 0


def test_quarter_warps_hit_distinct_bank_groups():
    # eight consecutive lanes of every one-dimensional pass touch eight distinct
    # 16-byte groups of a 128-byte line (slot mod 8), for each element t
    for ln in range(3, 13):
        for rl, lh in passes(ln):
            if rl != 3:
                continue
            h = 1 << lh
            for g0 in range(0, 1 << (ln - rl), 8):
                for t in range(8):
                    groups = set()
                    for g in range(g0, g0 + 8):
                        e0 = ((g >> lh) << (lh + rl)) + (g & (h - 1))
                        groups.add(slots(rl, lh, e0)[t] % 8)
                    assert len(groups) == 8, (ln, lh, g0, t)
