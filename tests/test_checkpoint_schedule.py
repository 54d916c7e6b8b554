"""The checkpoint schedule of fwi_gradient (wavefield checkpointing with
recomputation; the paper is silent on it), checked on the host for many step
counts and pool sizes by simulating it slot by slot.

- Every step reads the time level it needs: p^t and p^{t-1} for a forward
  step, q^{t+2}, q^{t+3} and the snapshot p^t for an adjoint step (levels
  before the start and after the end are the zero slot).
- The first pass runs steps 0..nt-1; the adjoint steps run nt-1..0, each once;
  the recomputed steps number what the plan reports.
- Inside one launch the reuse distances that the 2D multi-step kernel's
  tile-progress flags rely on hold: a slot is rewritten at the earliest three
  steps after it was written, two steps after it was read with a halo (the
  stepped level, the snapshot) and one step after a plain read.
The GPU tests check the same schedules end to end (checkpointed gradients
bit-identical to stored ones)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2512_12797_gb300 import _native
    return _native.lib()


def schedule(L, nt, slots):
    n, K, S, U = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    R = ctypes.c_int64()
    rc = L.fwi_checkpoint_schedule(nt, slots, None, 0, ctypes.byref(n), ctypes.byref(K), ctypes.byref(S),
                                   ctypes.byref(R), ctypes.byref(U))
    if rc == -3:
        return None
    assert rc == 0
    arr = np.zeros((n.value, 7), np.int32)
    assert L.fwi_checkpoint_schedule(nt, slots, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value - 1,
                                     ctypes.byref(n), None, None, None, None) == -1  # too small a buffer
    rc = L.fwi_checkpoint_schedule(nt, slots, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value,
                                   ctypes.byref(n), None, None, None, None)
    assert rc == 0
    return arr, K.value, S.value, R.value, U.value


def simulate(arr, nt, used):
    content = {}

    def expect(slot, kind, lev):
        if (kind == "p" and lev <= 0) or (kind == "q" and lev > nt):
            assert slot == 0, (kind, lev, slot)
        else:
            assert content.get(slot) == (kind, lev), (kind, lev, slot, content.get(slot))

    fwd_first, adj, recomputed = [], [], 0
    for launch, kind, cur, prev, out, snap, t in arr.tolist():
        assert out != 0 and max(cur, prev, out, snap) < used
        if kind == 0:
            expect(cur, "p", t)
            expect(prev, "p", t - 1)
            content[out] = ("p", t + 1)
            if launch == 0:
                fwd_first.append(t)
            else:
                recomputed += 1
        else:
            expect(cur, "q", t + 2)
            expect(prev, "q", t + 3)
            expect(snap, "p", t)
            content[out] = ("q", t + 1)
            adj.append(t)
    assert fwd_first == list(range(nt))
    assert adj == list(range(nt - 1, -1, -1))
    return recomputed


def reuse_distances(arr):
    for launch in np.unique(arr[:, 0]):
        steps = arr[arr[:, 0] == launch]
        last_write, last_halo, last_plain = {}, {}, {}
        for s, (_, kind, cur, prev, out, snap, t) in enumerate(steps.tolist()):
            assert out not in (cur, prev) and (kind == 0 or out != snap)
            if out in last_write:
                assert s - last_write[out] >= 3, (launch, s, out)
            if out in last_halo:
                assert s - last_halo[out] >= 2, (launch, s, out)
            if out in last_plain:
                assert s - last_plain[out] >= 1, (launch, s, out)
            last_write[out] = s
            last_halo[cur] = s
            if kind == 1:
                last_halo[snap] = s
            last_plain[prev] = s


@pytest.mark.parametrize("nt", [1, 2, 3, 4, 7, 10, 31, 64, 100, 257])
def test_schedules_read_the_right_levels_and_keep_reuse_distances(L, nt):
    prev_rec = None
    feasible = 0
    for slots in sorted({8, 9, 10, 12, 16, 20, 25, 32, 40, 60, 100, nt + 6, nt + 7, nt + 8, 3 * nt}):
        got = schedule(L, nt, slots)
        if got is None:
            assert prev_rec is None  # once a pool fits, larger pools fit too
            continue
        feasible += 1
        arr, K, nseg, rec, used = got
        assert used <= slots and 1 <= K <= nt and nseg == -(-nt // K)
        assert simulate(arr, nt, used) == rec == (nseg - 1) * (K - 1)
        reuse_distances(arr)
        if prev_rec is not None:
            assert rec <= prev_rec  # a larger pool never recomputes more
        prev_rec = rec
        if slots >= nt + 7:
            assert rec == 0  # every snapshot fits: nothing is recomputed
    assert feasible > 0


def test_schedule_rejects_pools_that_cannot_hold_a_plan(L):
    n = ctypes.c_int()
    assert L.fwi_checkpoint_schedule(100, 4, None, 0, ctypes.byref(n), None, None, None, None) == -3
    assert L.fwi_checkpoint_schedule(0, 100, None, 0, ctypes.byref(n), None, None, None, None) == -1


def test_the_simulation_catches_planted_slot_mistakes(L):
    arr, K, nseg, rec, used = schedule(L, 40, 30)
    assert rec > 0
    adj = np.nonzero(arr[:, 1] == 1)[0]
    for col, row in [(5, adj[len(adj) // 2]), (2, 7), (4, adj[3])]:
        bad = arr.copy()
        bad[row, col] = (bad[row, col] % (used - 1)) + 1 if bad[row, col] != 1 else 2
        with pytest.raises(AssertionError):
            simulate(bad, 40, used)
            reuse_distances(bad)
