"""A step-level model of the band-wavefront sweep's schedule (the transport sweep of Sec. 2.2 as the
band kernel orders it), run on the CPU to check three properties of that order that the GPU tests can
only observe indirectly:

  * no configuration the library accepts can deadlock: with fewer warps than bands (a warp takes bands
    w, w + W, w + 2W, ...), the producer of band b - 1 may be the consumer's own warp or one that is
    still on an earlier band, and its progress is published every 4 columns.  In the model a wait
    can block forever for nx <= 32 W + 2 and never from 32 W + 3 on; the library accepts
    nx >= 32 W + 4, one column of margin;
  * the shared-memory ring that hands band b's bottom trace to band b + 1 is never overwritten (by the
    owner's next band b + W) before band b + 1 has read it, whatever the interleaving of the warps;
  * the staged psi stores write every cell exactly once with its own value: lanes gather 4 cells of
    their row, the holders of completed row segments enter them in a per-warp table at their rank
    among the holders, and lane i copies cell i % 4 of entries i / 4, i / 4 + 8, ...

Model: lane l of a warp works at step s on its k = s - l th cell (local band k // nx, column k % nx of
the sweep's frame); a warp's step completes only when its lane 0's wait (band > 0) is satisfied, and
the lane-0 wait of step s sees the progress published by steps before s.  On the GPU the waiting lane
may also see its own warp's publication of the same step (the other lanes run on while it spins), so
the model sees at most the progress the kernel sees: a configuration free of deadlock here is free of
it there.  Every wait depends only on counters that never decrease, so a greedy schedule that runs
any warp able to advance reaches a deadlock exactly when some schedule does.  CPU only; no oracle
involved."""
import random

import numpy as np
import pytest

K_OUT = 4          # cells of a row gathered per lane before a segment is written


def band_cfg_accepted(nx, ny, W):
    """The library's rule for the band kernel's warp count (band meshes: nx >= 32, ny > 32)."""
    nb = (ny + 31) // 32
    if not (nx >= 32 and ny > 32) or W < 1 or W > 16 or W > nb:
        return False
    return not (W < nb and nx < 32 * W + 4)


class BandModel:
    """One ordinate of an nx x ny mesh swept by W warps; (px, py) the signs of the direction."""

    def __init__(self, nx, ny, W, px=True, py=True):
        self.nx, self.ny, self.W, self.px, self.py = nx, ny, W, px, py
        self.nb = (ny + 31) // 32
        self.nbw = [((self.nb - 1 - w) // W + 1) if w < self.nb else 0 for w in range(W)]
        self.nsteps = [self.nbw[w] * nx + 31 if self.nbw[w] else 0 for w in range(W)]
        self.step = [0] * W
        self.prog = [0] * W
        self.ring = {}                  # (warp, column) -> band whose trace the slot holds
        self.psi = {}                   # cell index -> list of values written
        self.obuf = {}                  # (warp, slot) -> cell value
        self.time = 0

    def lane_cell(self, w, s, lane):
        k = s - lane
        if not 0 <= k < self.nbw[w] * self.nx:
            return None
        lb, x = divmod(k, self.nx)
        band = w + lb * self.W
        row = band * 32 + lane
        if row >= self.ny:
            return None
        iy = row if self.py else self.ny - 1 - row
        ix = x if self.px else self.nx - 1 - x
        return k, band, x, iy * self.nx + ix

    def can_advance(self, w):
        s = self.step[w]
        if s >= self.nsteps[w]:
            return False
        c = self.lane_cell(w, s, 0)
        if c is None:
            return True
        k, band, x, _ = c
        if band == 0:
            return True
        wp = (w - 1) % self.W
        return self.prog[wp] >= ((band - 1) // self.W) * self.nx + x + 1

    def advance(self, w):
        """Run warp w's next step: lane 0's ring read, every lane's cell, lane 31's ring write and
        publication, then the flush of the row segments completed in this step."""
        s = self.step[w]
        wp = (w - 1) % self.W
        holders = []
        publish = None
        for lane in range(32):
            c = self.lane_cell(w, s, lane)
            if c is None:
                continue
            k, band, x, cell = c
            if lane == 0 and band > 0:
                assert self.ring.get((wp, x)) == band - 1, (w, s, band, x, self.ring.get((wp, x)))
            self.obuf[(w, (x % K_OUT) * 32 + lane)] = cell
            if x % K_OUT == K_OUT - 1 or x == self.nx - 1:
                holders.append((lane, x % K_OUT + 1, cell))
            if lane == 31 and band + 1 < self.nb:
                self.ring[(w, x)] = band
                if (x & 3) == 3 or x == self.nx - 1:
                    publish = k + 1
        if publish is not None:
            self.prog[w] = publish
        # the segment table: holders in lane order, entry r = the r-th holder
        table = [(end, length, lane) for lane, length, end in sorted(holders)]
        dc = 1 if self.px else -1
        for i in range(32):
            g, j = i // K_OUT, i % K_OUT
            while g < len(table):
                end, length, src = table[g]
                if j < length:
                    cell = end - (length - 1 - j) * dc
                    self.psi.setdefault(cell, []).append(self.obuf[(w, j * 32 + src)])
                g += 32 // K_OUT
        self.step[w] = s + 1
        self.time += 1

    def done(self):
        return all(self.step[w] >= self.nsteps[w] for w in range(self.W))

    def run(self, rng=None):
        """Advance until every warp is done (True) or none can advance (False: deadlock).  With rng,
        each move picks one advanceable warp at random and runs it for a random number of steps."""
        while not self.done():
            ready = [w for w in range(self.W) if self.can_advance(w)]
            if not ready:
                return False
            if rng is None:
                for w in ready:
                    while self.can_advance(w):
                        self.advance(w)
            else:
                w = rng.choice(ready)
                for _ in range(rng.randint(1, 40)):
                    if not self.can_advance(w):
                        break
                    self.advance(w)
        return True


@pytest.mark.parametrize("W", [1, 2, 3, 4])
def test_accepted_band_configurations_never_deadlock_and_the_rule_is_nearly_tight(W):
    for nb in (W + 1, W + 2, 2 * W + 1):
        ny = 32 * (nb - 1) + 7                       # a ragged last band
        for nx in range(max(32, 32 * W - 3), 32 * W + 9):
            ok = BandModel(nx, ny, W).run()
            if band_cfg_accepted(nx, ny, W):
                assert ok, (nx, ny, W)
            # the model's own threshold: the library's rule keeps one column above it
            assert ok == (nx >= 32 * W + 3), (nx, ny, W)


def test_one_warp_per_band_never_waits_forever():
    for nb in (2, 3, 5):
        for nx in (32, 33, 35, 47):
            assert band_cfg_accepted(nx, 32 * nb, nb)
            assert BandModel(nx, 32 * nb, nb).run()


def test_batched_blocks_sized_for_the_tallest_mesh_never_wait_forever():
    """The batched sweep gives every block one warp per band of the batch's tallest mesh (at most
    16): on a smaller mesh the warps beyond its band count idle, and the others never wait forever,
    whatever the mesh width (no cyclic ownership, so no width rule)."""
    for W in (4, 8, 16):
        for ny in (33, 64, 100, 32 * W):
            if (ny + 31) // 32 > W:
                continue
            for nx in (32, 33, 47, 64):
                m = BandModel(nx, ny, W)
                assert m.run(), (nx, ny, W)
                assert sorted(m.psi) == list(range(nx * ny))


@pytest.mark.parametrize("px,py", [(True, True), (False, True), (True, False), (False, False)])
def test_staged_stores_write_every_cell_once_with_its_value(px, py):
    for nx, ny, W in ((32, 33, 2), (37, 70, 3), (41, 100, 4), (69, 100, 2), (36, 64, 1), (130, 90, 1)):
        assert band_cfg_accepted(nx, ny, W)
        m = BandModel(nx, ny, W, px, py)
        assert m.run()
        assert sorted(m.psi) == list(range(nx * ny))
        for cell, vals in m.psi.items():
            assert vals == [cell], (nx, ny, W, cell, vals)


def test_ring_slots_are_read_before_they_are_rewritten_under_random_interleavings():
    rng = random.Random(20260105)
    for nx, ny, W in ((36, 100, 1), (68, 160, 2), (100, 200, 3), (132, 300, 4), (40, 96, 3)):
        assert band_cfg_accepted(nx, ny, W)
        for _ in range(12):
            m = BandModel(nx, ny, W, rng.random() < 0.5, rng.random() < 0.5)
            assert m.run(rng)            # the ring assertion runs inside every step
            assert len(m.psi) == nx * ny


def test_model_counts_match_the_kernel_step_counts():
    """Each warp runs its bands' columns plus the 31-step lane skew; a sweep of nb bands over W warps
    takes ceil((nb - w) / W) bands for warp w."""
    m = BandModel(101, 32 * 7 + 3, 3)
    assert band_cfg_accepted(101, 32 * 7 + 3, 3)
    assert m.nb == 8 and m.nbw == [3, 3, 2]
    assert m.nsteps == [3 * 101 + 31, 3 * 101 + 31, 2 * 101 + 31]
    assert m.run()
    assert np.sum(m.step) == np.sum(m.nsteps)
