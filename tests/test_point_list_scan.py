"""Host model of the 3D step kernels' point-list scan (injection and sampling
at one z level of a column).

A tile's entries are sorted by level z, and a cursor points at the first entry
not yet used. At level z the warp reads the 32 entries under the cursor, one
per lane (past the list's end a lane sees no level). A ballot counts the
lanes whose entry is at z; because the list is sorted, those lanes form a
prefix of the warp. The warp uses them, advances the cursor past them, and
takes the next cursor level from the lane just past the prefix, or reads the
next 32 when all of them matched.

The model replays that loop over random sorted lists and compares the entries
it uses and the final cursor with a direct filter of the list.
"""
import random

NONE = 2 ** 31 - 1
WARP = 32


def scan_level(zs, cur, end, cur_z, z):
    """One level of the kernel's loop: returns (entries used, cursor, cursor level)."""
    used = []
    while cur_z == z:
        lanes = [zs[cur + l] if cur + l < end else NONE for l in range(WARP)]
        here = [w == z for w in lanes]
        ballot = sum(1 << l for l in range(WARP) if here[l])
        n = bin(ballot).count("1")
        assert ballot == (1 << n) - 1, "entries at level z must be a prefix of the warp"
        used += [cur + l for l in range(WARP) if here[l]]
        cur += n
        cur_z = lanes[n & 31] if n < WARP else z
    return used, cur, cur_z


def run_column(zs, nz):
    cur, end = 0, len(zs)
    cur_z = zs[0] if zs else NONE
    seen = []
    for z in range(nz):
        if cur_z != z:
            continue
        used, cur, cur_z = scan_level(zs, cur, end, cur_z, z)
        assert used == [i for i, w in enumerate(zs) if w == z]
        seen += used
    assert seen == list(range(len(zs))) and cur == end and cur_z == NONE


def test_scan_uses_exactly_each_levels_entries():
    rng = random.Random(7)
    for counts in ([0], [1], [31], [32], [33], [64], [65], [100], [1, 32, 1], [31, 33, 64, 0, 2]):
        zs = []
        for i, c in enumerate(counts):
            zs += [3 + 2 * i] * c
        run_column(zs, 3 + 2 * len(counts) + 1)
    for _ in range(200):
        nz = rng.randint(1, 40)
        zs = sorted(rng.randrange(nz) for _ in range(rng.randint(0, 150)))
        run_column(zs, nz)


def test_scan_detects_an_unsorted_list():
    # a planted mistake: two levels interleaved breaks the prefix property
    zs = [5, 6, 5] + [7] * 3
    try:
        run_column(zs, 8)
    except AssertionError:
        return
    raise AssertionError("an unsorted list went unnoticed")
