"""Host model of the 3D multi-step launch's dependency protocol
(step3d_kernel with variant bits 3 and 4).

In one cooperative launch, CTA c runs the columns c, c + G, c + 2G, ... of
every step in order. A column (step n, unit u, tile) may start once every tile
of the 3 x 3 neighbourhood of the same unit has completed step n - 1 (a
progress flag per (unit, tile)). The column order (tile-major or
wavefield-fastest) maps a column index to (unit, tile) as the kernel's
column_of does.

The model runs the CTAs in random interleavings and checks three things. Every
item completes, so there is no deadlock. A column is never started before its
neighbours' previous step. Every flag index stays inside the units x tiles
array. Tile grids and grid sizes are those of the layered 3D batch (5 x 19
tiles of 64 x 16, or 5 x 37 pair tiles) and of small and degenerate cases.
"""
import random

import pytest


def column_of(it, nunits, ntiles, order3):
    if order3:
        return it % nunits, it // nunits
    return it // ntiles, it % ntiles


def run(ntx, nty, nunits, nsm, nsteps, order3, seed):
    ntiles = ntx * nty
    ncols = ntiles * nunits
    G = min(nsm, ncols)
    done = [[0] * ntiles for _ in range(nunits)]
    cols = [list(range(c, ncols, G)) for c in range(G)]
    pos = [0] * G
    total = [len(cl) * nsteps for cl in cols]
    rng = random.Random(seed)
    progress = True
    while progress:
        progress = False
        order = list(range(G))
        rng.shuffle(order)
        for c in order:
            if pos[c] >= total[c]:
                continue
            n, k = divmod(pos[c], len(cols[c]))
            u, t = column_of(cols[c][k], nunits, ntiles, order3)
            assert 0 <= u < nunits and 0 <= t < ntiles
            tx, ty = t % ntx, t // ntx
            ready = all(done[u][y * ntx + x] >= n
                        for y in range(max(ty - 1, 0), min(ty + 1, nty - 1) + 1)
                        for x in range(max(tx - 1, 0), min(tx + 1, ntx - 1) + 1))
            if ready:
                assert done[u][t] == n  # the CTA's own column of the previous step is done
                done[u][t] = n + 1
                pos[c] += 1
                progress = True
    assert pos == total, "deadlock"
    assert all(done[u][t] == nsteps for u in range(nunits) for t in range(ntiles))


CASES = [(5, 19, 8, 152), (5, 19, 4, 152), (5, 37, 4, 152), (2, 6, 16, 152), (2, 6, 4, 152),
         (1, 1, 1, 152), (3, 11, 8, 152), (5, 19, 8, 7), (2, 6, 16, 5), (5, 9, 8, 152)]


@pytest.mark.parametrize("ntx,nty,nunits,nsm", CASES)
@pytest.mark.parametrize("order3", [0, 1])
def test_multistep_protocol_completes_in_any_interleaving(ntx, nty, nunits, nsm, order3):
    for seed in range(3):
        run(ntx, nty, nunits, nsm, 6, order3, seed)


def test_model_detects_a_missing_dependency():
    # planted mistake in the model: a neighbourhood test that ignores the y
    # neighbours lets a column start before a neighbour's previous step; the
    # stricter check below must then see an out-of-order start
    ntx, nty, nunits = 3, 4, 1
    ntiles = ntx * nty
    done = [0] * ntiles
    started_early = False
    rng = random.Random(1)
    pending = {t: 0 for t in range(ntiles)}
    while any(v < 3 for v in pending.values()):
        t = rng.randrange(ntiles)
        n = pending[t]
        if n >= 3:
            continue
        tx, ty = t % ntx, t // ntx
        lax = all(done[ty * ntx + x] >= n for x in range(max(tx - 1, 0), min(tx + 1, ntx - 1) + 1))
        strict = all(done[y * ntx + x] >= n for y in range(max(ty - 1, 0), min(ty + 1, nty - 1) + 1)
                     for x in range(max(tx - 1, 0), min(tx + 1, ntx - 1) + 1))
        if lax:
            started_early |= not strict
            done[t] = n + 1
            pending[t] = n + 1
    assert started_early
