"""CPU model of the synchronisation protocol of the fused colour-class kernel
(`k_vb_packed_colour` in paper_1906_11195_gb300/csrc/vb_kernels.cu), explored over random
interleavings.

The model restates, step for step, what the kernel's actors wait for and release: per CTA one
producer warp (stream ring of NSS stages with "full" and "empty" mbarriers) and W consumer warps
(gather ring of NG buffers with "gfree" mbarriers, cp.async groups with wait_group<L>), and the
grid-wide barrier between colour classes.  Copies and gathers complete asynchronously at any
later step.  Each run must finish (no deadlock), and every step must respect:

  * mbarrier parity waits are never ambiguous: when a warp tests the phase it waits for, the
    barrier is in that phase or the next one (never two phases on, never one behind);
  * a stream stage is refilled only after every consumer released its previous group, and a
    gather buffer only after every consumer released the group it held;
  * the data a consumer uses (its stage, its gathers) belongs to the group it is updating;
  * colour order: every neighbour gather of class c starts after every update of a class < c
    has been written (all CTAs) and completes before any update of a class > c is written.

Planted protocol mistakes in the model (no gather-buffer wait, no grid barrier) must be caught.
Forms of a launch running several sweeps (which the kernel does not do) show what that needs
beyond the ring waits: holding the next sweep's first stage until the previous sweep's last
group is released deadlocks against the consumers' look at that stage; the ring waits alone can
stage a group's own words before the previous sweep wrote them; waiting for the release of the
same group in the previous sweep keeps every order when each CTA owns at least two groups.  The model checks the design
of the waits, not the CUDA code itself.
"""
import random

import pytest


class ProtocolError(AssertionError):
    pass


class MBar:
    """An mbarrier: a phase completes when `count` arrivals and all expected bytes are in."""

    def __init__(self, count):
        self.count = count
        self.pending = count
        self.tx = 0
        self.phase = 0  # completed phases

    def _step(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def arrive(self):
        self.pending -= 1
        self._step()

    def arrive_expect_tx(self, nbytes):
        self.tx += nbytes
        self.arrive()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        self._step()

    def done(self, phase_index):
        """try_wait.parity for the phase with absolute index phase_index (parity = index & 1)."""
        if not (phase_index <= self.phase <= phase_index + 1):
            raise ProtocolError(f"ambiguous parity wait: barrier at phase {self.phase}, waiting for {phase_index}")
        return (self.phase & 1) != (phase_index & 1)


class Sim:
    def __init__(self, grid, warps, nss, ng, lookahead, class_groups, seed, sweeps=1,
                 mutant=None):
        self.G, self.W, self.NSS, self.NG, self.L = grid, warps, nss, ng, lookahead
        self.nc = len(class_groups)
        self.class_groups = class_groups  # groups per colour class (whole grid)
        self.sweeps = sweeps
        self.mutant = mutant
        self.rng = random.Random(seed)
        self.time = 0
        self.gbar = 0
        self.writes = []   # (time, sweep, class)
        self.reads = []    # (t_issue, t_done, sweep, class)
        self.actors = []   # generators yielding wait predicates
        self.events = []   # pending asynchronous completions: callables
        for cta in range(grid):
            self._make_cta(cta)

    # ---------------------------------------------------------------- per-CTA state and actors
    def _make_cta(self, cta):
        G, W, NSS, NG = self.G, self.W, self.NSS, self.NG
        # this CTA's groups per class: static round robin over the grid, as in the kernel
        per_class = [len(range(cta, n, G)) for n in self.class_groups]
        kc = [0]
        for n in per_class:
            kc.append(kc[-1] + n)
        n_mine = kc[-1]
        c = {"full": [MBar(1) for _ in range(NSS)], "empty": [MBar(W) for _ in range(NSS)],
             "gfree": [MBar(W) for _ in range(NG)], "kc": kc, "n_mine": n_mine,
             "stage": [None] * NSS, "gbuf": [None] * NG, "released": {},
             "bar_arrived": {}, "id": cta}
        self.actors.append(self._producer(c))
        for w in range(W):
            self.actors.append(self._consumer(c, w))

    def _class_of(self, c, k):
        kk = k % c["n_mine"]
        j = 0
        while kk >= c["kc"][j + 1]:
            j += 1
        return j

    def _producer(self, c):
        NSS = self.NSS
        n_total = c["n_mine"] * self.sweeps
        for k in range(n_total):
            s = k % NSS
            if k >= NSS:
                yield lambda k=k, s=s: c["empty"][s].done(k // NSS - 1)
            if self.mutant == "hold_next_sweep" and k > 0 and k % c["n_mine"] == 0:
                kp = k - 1
                yield lambda kp=kp: c["empty"][kp % NSS].done(kp // NSS)
            if self.mutant == "own_word_wait" and k >= c["n_mine"] and c["n_mine"] < NSS:
                # wait for the release of the same group in the previous sweep, which is more
                # recent than the ring's own k - NSS
                kp = k - c["n_mine"]
                yield lambda kp=kp: c["empty"][kp % NSS].done(kp // NSS)
            # refill stage s with group k: every consumer must have released group k - NSS
            if k >= NSS and c["released"].get(k - NSS, 0) != self.W:
                raise ProtocolError(f"stage {s} refilled while group {k - NSS} is in use")
            # the stage carries the group's own words: in a later sweep of the same launch they
            # were written by this group's update in the previous sweep
            if k >= c["n_mine"] and c["released"].get(k - c["n_mine"], 0) != self.W:
                raise ProtocolError(f"own words of group {k} staged before the previous sweep wrote them")
            c["stage"][s] = None  # in flight
            full = c["full"][s]
            full.arrive_expect_tx(1)

            def land(s=s, k=k, full=full):
                c["stage"][s] = k
                full.complete_tx(1)
            self.events.append(land)

    def _grid_barrier(self, c, target, w):
        key = target
        c["bar_arrived"][key] = c["bar_arrived"].get(key, 0) + 1
        yield lambda: c["bar_arrived"][key] == self.W  # bar.red over the CTA's consumers
        if w == 0:
            self.gbar += 1  # one arrival per CTA
        yield lambda: self.gbar >= target

    def _consumer(self, c, w):
        NSS, NG, L = self.NSS, self.NG, self.L
        n_mine = c["n_mine"]
        n_total = n_mine * self.sweeps
        groups = []  # this warp's cp.async groups: [done flag holder or None for empty]

        def gathers(k, k_end, sweep):
            if k < k_end:
                s, b = k % NSS, k % NG
                yield lambda: c["full"][s].done(k // NSS)
                if k >= NG and self.mutant != "no_gfree":
                    yield lambda: c["gfree"][b].done(k // NG - 1)
                if c["stage"][s] != k:
                    raise ProtocolError(f"gathers of group {k} read stage {s} holding {c['stage'][s]}")
                if k >= NG and c["released"].get(k - NG, 0) != self.W:
                    raise ProtocolError(f"gather buffer {b} overwritten while group {k - NG} is in use")
                c["gbuf"][b] = k
                cls = self._class_of(c, k)
                rec = {"done": False, "k": k, "b": b}
                t_issue = self.time

                def land(rec=rec, cls=cls, t_issue=t_issue, sweep=sweep):
                    rec["done"] = True
                    self.reads.append((t_issue, self.time, sweep, cls))
                self.events.append(land)
                groups.append(rec)
            else:
                groups.append(None)

        if n_mine:
            yield lambda: c["full"][0].done(0)
        bar_idx = 0
        for sweep in range(self.sweeps):
            base = sweep * n_mine
            for j in range(self.nc):
                kb, ke = base + c["kc"][j], base + c["kc"][j + 1]
                if j > 0 or sweep > 0:
                    bar_idx += 1
                    if self.mutant != "no_grid_barrier":
                        yield from self._grid_barrier(c, bar_idx * self.G, w)
                for k in range(kb, kb + L):
                    yield from gathers(k, ke, sweep)
                for k in range(kb, ke):
                    yield from gathers(k + L, ke, sweep)
                    if k + 1 < n_total:
                        kn = k + 1
                        if kn >= ke:
                            yield lambda kn=kn: c["full"][kn % NSS].done(kn // NSS)
                        if c["stage"][kn % NSS] != kn:
                            raise ProtocolError(f"acceptance of group {kn} read a stage holding {c['stage'][kn % NSS]}")
                    # cp.async.wait_group L: all but the newest L groups complete
                    pending = groups[:-L] if L else groups
                    yield lambda pending=pending: all(g is None or g["done"] for g in pending)
                    s, b = k % NSS, k % NG
                    if c["stage"][s] != k:
                        raise ProtocolError(f"update of group {k} read stage {s} holding {c['stage'][s]}")
                    if c["gbuf"][b] != k:
                        raise ProtocolError(f"update of group {k} read gather buffer {b} holding {c['gbuf'][b]}")
                    mine = [g for g in groups if g is not None and g["k"] == k]
                    if not all(g["done"] for g in mine):
                        raise ProtocolError(f"update of group {k} before its gathers landed")
                    self.writes.append((self.time, sweep, self._class_of(c, k)))
                    c["released"][k] = c["released"].get(k, 0) + 1
                    c["empty"][s].arrive()
                    c["gfree"][b].arrive()
        yield lambda: all(g is None or g["done"] for g in groups)  # wait_group 0

    # ---------------------------------------------------------------- scheduler
    def run(self, max_steps=200000):
        waits = [None] * len(self.actors)
        live = set(range(len(self.actors)))
        for i in list(live):
            waits[i] = self._advance(i, live)
        for _ in range(max_steps):
            if not live and not self.events:
                break
            runnable = [i for i in live if waits[i] is None or waits[i]()]
            choices = runnable + (["event"] if self.events else [])
            if not choices:
                raise ProtocolError("deadlock: every actor waits and no copy is in flight")
            pick = self.rng.choice(choices)
            self.time += 1
            if pick == "event":
                self.events.pop(self.rng.randrange(len(self.events)))()
            else:
                waits[pick] = self._advance(pick, live)
        else:
            raise ProtocolError("step limit reached")
        self._check_order()

    def _advance(self, i, live):
        try:
            return next(self.actors[i])
        except StopIteration:
            live.discard(i)
            return None

    def _check_order(self):
        for t_issue, t_done, sweep, cls in self.reads:
            for t_w, sw, c_w in self.writes:
                earlier = (sw, c_w) < (sweep, cls)
                later = (sw, c_w) > (sweep, cls)
                if earlier and t_w >= t_issue:
                    raise ProtocolError(f"gather of class {cls} started before an update of class {c_w} was written")
                if later and t_w <= t_done:
                    raise ProtocolError(f"gather of class {cls} landed after an update of class {c_w} was written")


# (stream stages, gather buffers, lookahead): the kernel's shapes, then two it could take
SHAPES = [(3, 3, 1), (4, 2, 1), (2, 2, 1), (4, 3, 1), (4, 3, 2)]
LAYOUTS = [
    [7, 5, 3, 1],        # classes shrinking to a one-group tail
    [2, 9, 0, 4],        # an empty class
    [1, 1, 1],           # fewer groups than CTAs in every class
    [12],                # a single class (no grid barrier)
]


@pytest.mark.parametrize("nss,ng,L", SHAPES)
@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("grid,warps", [(1, 2), (3, 2), (2, 3)])
def test_kernel_protocol_is_safe_and_finishes(nss, ng, L, layout, grid, warps):
    for seed in range(25):
        Sim(grid, warps, nss, ng, L, layout, seed).run()


@pytest.mark.parametrize("mutant,layout", [("no_gfree", [9, 6]), ("no_grid_barrier", [6, 6, 3])])
def test_planted_protocol_mistakes_are_caught(mutant, layout):
    caught = 0
    for seed in range(60):
        try:
            Sim(2, 2, 3, 2, 1, layout, seed, mutant=mutant).run()
        except ProtocolError:
            caught += 1
    assert caught > 0, mutant


def test_multi_sweep_launch_with_held_first_stage_deadlocks():
    # a multi-sweep launch whose producer holds the next sweep's first stage until the previous
    # sweep's last group is released, while the consumers of that last group wait for the next
    # stage to compute its acceptance: the waits form a cycle
    with pytest.raises(ProtocolError, match="deadlock"):
        Sim(1, 2, 3, 3, 1, [4, 3], 0, sweeps=2, mutant="hold_next_sweep").run()


def test_multi_sweep_launch_with_own_word_wait_is_consistent():
    # the form to use: the producer also waits for the release of the same group in the previous
    # sweep; with at least two groups per CTA it keeps every order and finishes (the memory
    # fences the own-word copies need on the GPU are outside the model)
    for layout, grid in (([2, 2, 1], 2), ([5, 3, 1], 2), ([3, 3], 3), ([9, 1, 1], 4)):
        for seed in range(25):
            Sim(grid, 2, 3, 3, 1, layout, seed, sweeps=3, mutant="own_word_wait").run()


def test_multi_sweep_launch_with_one_group_per_cta_deadlocks():
    # one group per CTA: the group's own previous-sweep release is the one its consumers hold
    # while they look at the next sweep's first stage
    with pytest.raises(ProtocolError, match="deadlock"):
        Sim(2, 2, 3, 3, 1, [2, 1], 0, sweeps=2, mutant="own_word_wait").run()  # CTA 1: one group


def test_multi_sweep_launch_with_ring_waits_only_stages_stale_own_words():
    # with fewer groups per CTA than stream stages, the ring waits alone let the producer stage
    # a group of the next sweep before the previous sweep's update of that group is written
    caught = 0
    for seed in range(40):
        try:
            Sim(3, 2, 3, 3, 1, [2, 2, 1], seed, sweeps=3).run()
        except ProtocolError as e:
            assert "own words" in str(e) or "deadlock" in str(e)
            caught += 1
    assert caught > 0
