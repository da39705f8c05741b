"""A randomized model of the tensor-core step kernels' warp roles and mbarrier
protocol, for race checking on the CPU.

Roles are generators that yield waits on mbarriers (with the phase index the
role means to wait for) and perform actions (arrivals, TMA loads, MMAs and
commits).  The scheduler interleaves runnable roles and completes outstanding
asynchronous work (TMA loads in any order, MMAs in issue order, a commit once
every MMA issued before it completed) at random.  mbarrier semantics are the
hardware's: a phase completes when its pending arrival count and its
transaction bytes reach zero; `wait(parity p)` passes when the number of
completed phases has the other parity.  A wait meant for phase k that passes
with fewer than k + 1 completed phases is a stale pass (the parity aliased); a
state where nothing can move while roles still wait is a deadlock.  Every
shared resource carries a data tag that readers check: staging slots (which
tile and slot was loaded), A-operand chunks, tensor-memory accumulators and
the resident table.
"""
import random


class ProtocolError(AssertionError):
    pass


class Barrier:
    def __init__(self, name, count):
        self.name, self.count = name, count
        self.pending, self.tx, self.completed = count, 0, 0

    def arrive(self, n=1):
        self.pending -= n
        if self.pending < 0:
            raise ProtocolError(f"{self.name}: more arrivals than expected in phase {self.completed}")
        self._maybe_complete()

    def expect_tx(self, nbytes):            # mbarrier.arrive.expect_tx: one arrival plus bytes
        self.tx += nbytes
        self.arrive()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        self._maybe_complete()

    def _maybe_complete(self):
        if self.pending == 0 and self.tx == 0:
            self.completed += 1
            self.pending = self.count

    def passes(self, parity):
        return (self.completed & 1) != parity


class Wait:
    """Yielded by a role: wait on `bar` for the completion of phase `k`
    (k = -1: the phase before the first, passes on a fresh barrier)."""

    def __init__(self, bar, k, who):
        self.bar, self.k, self.who = bar, k, who

    def ready(self):
        return self.bar.passes(self.k & 1)

    def check_pass(self):
        if self.bar.completed < self.k + 1:
            raise ProtocolError(f"{self.who}: stale pass on {self.bar.name} waiting for phase {self.k} "
                                f"with {self.bar.completed} completed")


class Machine:
    """`slow` maps a role-name prefix to a scheduling weight (default 1):
    roles given a small weight run rarely, which lets a test reach orders
    where one role lags far behind the others."""

    def __init__(self, seed, slow=None):
        self.rng = random.Random(seed)
        self.slow = dict(slow or {})
        self.roles = {}                 # name -> [generator, pending Wait or None]
        self.tma = []                   # outstanding TMA loads: callables run on completion
        self.mma = []                   # FIFO of ("mma", fn) / ("commit", barrier)
        self.steps = 0

    def add_role(self, name, gen):
        self.roles[name] = [gen, None]

    # actions used by roles -------------------------------------------------
    def tma_load(self, on_land):
        self.tma.append(on_land)

    def issue_mma(self, on_complete):
        self.mma.append(("mma", on_complete))

    def commit(self, bar):
        self.mma.append(("commit", bar))

    # scheduler ---------------------------------------------------------------
    def _advance(self, name):
        gen, _ = self.roles[name]
        try:
            w = next(gen)
        except StopIteration:
            del self.roles[name]
            return
        self.roles[name][1] = w

    def run(self, max_steps=2_000_000):
        for name in list(self.roles):
            self._advance(name)
        while self.roles or self.tma or self.mma:
            self.steps += 1
            if self.steps > max_steps:
                raise ProtocolError("model did not finish")
            choices = [("role", n) for n, (g, w) in self.roles.items() if w is None or w.ready()]
            if self.tma:
                choices.append(("tma", None))
            if self.mma:
                choices.append(("mma", None))
            if not choices:
                waits = {n: f"{w.bar.name}[phase {w.k}, {w.bar.completed} done]" for n, (g, w) in self.roles.items()}
                raise ProtocolError(f"deadlock: {waits}")
            if self.slow:
                weights = [next((w for pre, w in self.slow.items() if k == "role" and n.startswith(pre)), 1.0)
                           for k, n in choices]
                kind, name = self.rng.choices(choices, weights)[0]
            else:
                kind, name = self.rng.choice(choices)
            if kind == "role":
                w = self.roles[name][1]
                if w is not None:
                    w.check_pass()
                self._advance(name)
            elif kind == "tma":
                self.tma.pop(self.rng.randrange(len(self.tma)))()
            else:
                what, obj = self.mma.pop(0)
                if what == "mma":
                    obj()
                else:
                    obj.arrive()


def _groups(n):
    return n // 8                        # 8-direction staging slots per tile


def _chunks(n):
    return (4 * n + 63) // 64            # 64-wide bf16 K chunks per tile


def bf16_step(items, stages, seed, shared_ring=False, gather=False, edge_tiles=(), skip_fill_wait=False,
              gather_ring_flaw=False, slow=None):
    """The single-CTA tensor-core step (and the batch kernel, whose items may
    differ in n and table): `items` lists (n, table key) per tile in the order
    a CTA processes them.  Roles as in the kernels: one producer thread (TMA of
    the table on a key change, after `z_free`; one staging slot per 8
    directions into its group's ring), eight converter warps (quadrant q,
    group grp: slot j = 2c + grp of every 64-wide chunk c; TMEM init, then the
    A chunk once the previous tile's MMAs released it), one MMA thread (a
    commit per chunk barrier for every chunk the widest item has, then the
    accumulator barrier, then `z_free` before a key change) and eight epilogue
    warps (quadrant q, half of the directions).  shared_ring: the earlier form
    in which both converter groups consumed one ring of `stages` slots.
    gather: the gather form of bilinear streaming -- staging slots of four
    directions (n / 4 per tile), slot j to group (j >> 1) & 1, group grp
    taking slots 4c + 2 grp and 4c + 2 grp + 1 of chunk c; in the tiles listed
    in `edge_tiles` each of the group's four warps first writes its part of
    the window's ghost values, arrives on the group's fill barrier (count 4)
    and waits for it before reading the window.  skip_fill_wait: the warps
    read without that wait; gather_ring_flaw: the producer keeps the
    eight-direction form's group of a slot (j & 1) (planted flaws)."""
    M = Machine(seed, slow)
    T = len(items)
    ring = stages // 2
    max_c = max(_chunks(n) for n, _ in items)
    st_full = [Barrier(f"st_full[{s}]", 1) for s in range(stages)]
    st_empty = [Barrier(f"st_empty[{s}]", 4) for s in range(stages)]
    a_empty = [Barrier(f"a_empty[{c}]", 1) for c in range(max_c)]
    t_ready = [Barrier(f"t_ready[{b}]", 8) for b in range(2)]
    acc_full = [Barrier(f"acc_full[{b}]", 1) for b in range(2)]
    acc_empty = [Barrier(f"acc_empty[{b}]", 8) for b in range(2)]
    z_full, z_free = Barrier("z_full", 1), Barrier("z_free", 1)
    fill_bar = [Barrier(f"fill_bar[{g}]", 4) for g in range(2)]
    stage = [None] * stages
    filled = {}                  # (staging slot, quadrant) -> (tile, slot) whose ghost values it holds
    A, acc, z = {}, {}, [None]
    base = [0]
    for n, _ in items:
        base.append(base[-1] + (n // 4 if gather else _groups(n)))

    def slot_of(i, j, grp, local):
        if shared_ring:
            qg = base[i] + j
            return qg % stages, qg // stages
        return grp * ring + local % ring, local // ring

    def producer():
        prev, zr, gq = None, 0, [0, 0]
        for i, (n, key) in enumerate(items):
            if key != prev:
                if i > 0:
                    yield Wait(z_free, zr, "producer")
                    zr += 1
                z_full.expect_tx(1)

                def land_z(key=key):
                    z[0] = key
                    z_full.complete_tx(1)
                M.tma_load(land_z)
                prev = key
            for j in range(n // 4 if gather else _groups(n)):
                gr = (j >> 1) & 1 if gather and not gather_ring_flaw else j & 1
                local = gq[gr]
                gq[gr] += 1
                s, k = slot_of(i, j, gr, local)
                yield Wait(st_empty[s], k - 1, "producer")
                st_full[s].expect_tx(1)

                def land(s=s, tag=(i, j)):
                    stage[s] = tag
                    st_full[s].complete_tx(1)
                M.tma_load(land)

    def converter(q, grp):
        who = f"converter(q{q},g{grp})"
        gq = fq = 0
        for i, (n, key) in enumerate(items):
            b = i & 1
            yield Wait(acc_empty[b], (i >> 1) - 1, who)
            for c in range(_chunks(n)):
                j = 2 * c + grp
                mine = j < _groups(n)
                for h in range(2 if gather else 1):
                    if not mine:
                        break
                    sj = 4 * c + 2 * grp + h if gather else j
                    local = gq
                    gq += 1
                    s, k = slot_of(i, sj, grp, local)
                    yield Wait(st_full[s], k, who)
                    if stage[s] != (i, sj):
                        raise ProtocolError(f"{who} tile {i} slot {sj}: staging slot {s} holds {stage[s]}")
                    if gather and i in edge_tiles:
                        filled[(s, q)] = (i, sj)
                        fill_bar[grp].arrive()
                        if not skip_fill_wait:
                            yield Wait(fill_bar[grp], fq, who)
                        fq += 1
                        for q2 in range(4):
                            if filled.get((s, q2)) != (i, sj):
                                raise ProtocolError(f"{who} tile {i} slot {sj}: window part {q2} of staging slot {s} "
                                                    f"holds {filled.get((s, q2))}")
                    if h == 0:
                        cell = acc.get((b, j, q))
                        if cell is not None and cell[0] != "free":
                            raise ProtocolError(f"{who} tile {i}: accumulator {b} slot {j} still {cell[0]} "
                                                f"for tile {cell[1]}")
                        acc[(b, j, q)] = ["init", i, 0]
                    st_empty[s].arrive()
                yield Wait(a_empty[c], i - 1, who)
                if mine:
                    A[(c, grp, q)] = i
            t_ready[b].arrive()

    def mma():
        prev, zl = None, 0
        for i, (n, key) in enumerate(items):
            b = i & 1
            if key != prev:
                yield Wait(z_full, zl, "mma")
                zl += 1
                prev = key
            yield Wait(t_ready[b], i >> 1, "mma")
            for c in range(max_c):
                if c < _chunks(n):
                    def done(i=i, b=b, c=c, n=n, key=key):
                        for grp in (0, 1):
                            if 2 * c + grp < _groups(n):
                                for q in range(4):
                                    if A.get((c, grp, q)) != i:
                                        raise ProtocolError(f"MMA tile {i} chunk {c}: A part ({grp},{q}) holds "
                                                            f"tile {A.get((c, grp, q))}")
                        if z[0] != key:
                            raise ProtocolError(f"MMA tile {i}: table {z[0]} resident, {key} needed")
                        for j in range(_groups(n)):
                            for q in range(4):
                                cell = acc.get((b, j, q))
                                if cell is None or cell[1] != i or cell[0] not in ("init", "partial"):
                                    raise ProtocolError(f"MMA tile {i} chunk {c}: accumulator {b} slot {j} is {cell}")
                                cell[0] = "done" if c == _chunks(n) - 1 else "partial"
                    M.issue_mma(done)
                M.commit(a_empty[c])
            M.commit(acc_full[b])
            if i + 1 < T and items[i + 1][1] != key:
                M.commit(z_free)

    def epilogue(q, dh):
        who = f"epilogue(q{q},h{dh})"
        for i, (n, key) in enumerate(items):
            b = i & 1
            yield Wait(acc_full[b], i >> 1, who)
            dn = n // 2
            readers = 2 if dn < 8 else 1
            for j in sorted({d // 8 for d in range(dh * dn, dh * dn + dn)}):
                cell = acc.get((b, j, q))
                if cell is None or cell[0] != "done" or cell[1] != i:
                    raise ProtocolError(f"{who} tile {i}: accumulator {b} slot {j} is {cell}")
                cell[2] += 1
                if cell[2] == readers:
                    cell[0] = "free"
            acc_empty[b].arrive()

    M.add_role("producer", producer())
    M.add_role("mma", mma())
    for q in range(4):
        for grp in range(2):
            M.add_role(f"conv{q}{grp}", converter(q, grp))
        for dh in range(2):
            M.add_role(f"epi{q}{dh}", epilogue(q, dh))
    M.run()
    return M.steps


def fp8_step(items, stages, seed, gate_t_ready=True):
    """The FP8 kernel: one TMEM accumulator handed back by the epilogue one
    8-direction slot at a time (`d_free[j]`, arrived by every epilogue warp
    whose directions touch slot j), no A-chunk barriers (a converter past the
    slot's hand-off knows the previous tile's MMAs completed), a single
    `t_ready` and `acc_full`.  The converter reads a staging slot twice (block
    maximum, then conversion), the second time after the hand-off, and arrives
    on `t_ready` for tile i only after its phase for tile i - 1 completed
    (gate_t_ready=False: the first form, without that wait, in which a warp
    with no slot in a tile -- group 1 at n = 8 -- runs ahead)."""
    M = Machine(seed)
    T = len(items)
    n = items[0][0]
    assert all(it[0] == n for it in items)
    G, ring = _groups(n), stages // 2
    dfree_count = 4 if (n // 2) % 8 == 0 else 8
    st_full = [Barrier(f"st_full[{s}]", 1) for s in range(stages)]
    st_empty = [Barrier(f"st_empty[{s}]", 4) for s in range(stages)]
    d_free = [Barrier(f"d_free[{j}]", dfree_count) for j in range(G)]
    t_ready, acc_full = Barrier("t_ready", 8), Barrier("acc_full", 1)
    z_full, z_free = Barrier("z_full", 1), Barrier("z_free", 1)
    stage = [None] * stages
    A, acc, z, mma_done = {}, {}, [None], [-1]

    def producer():
        prev, zr, gq = None, 0, [0, 0]
        for i, (_, key) in enumerate(items):
            if key != prev:
                if i > 0:
                    yield Wait(z_free, zr, "producer")
                    zr += 1
                z_full.expect_tx(1)

                def land_z(key=key):
                    z[0] = key
                    z_full.complete_tx(1)
                M.tma_load(land_z)
                prev = key
            for j in range(G):
                gr = j & 1
                local = gq[gr]
                gq[gr] += 1
                s = gr * ring + local % ring
                yield Wait(st_empty[s], local // ring - 1, "producer")
                st_full[s].expect_tx(1)

                def land(s=s, tag=(i, j)):
                    stage[s] = tag
                    st_full[s].complete_tx(1)
                M.tma_load(land)

    def converter(q, grp):
        who = f"converter(q{q},g{grp})"
        gq = 0
        for i, _ in enumerate(items):
            for j in range(grp, G, 2):
                local = gq
                gq += 1
                s = grp * ring + local % ring
                yield Wait(st_full[s], local // ring, who)
                if stage[s] != (i, j):                       # first pass: block maximum
                    raise ProtocolError(f"{who} tile {i} slot {j}: staging slot {s} holds {stage[s]}")
                yield Wait(d_free[j], i - 1, who)
                if stage[s] != (i, j):                       # second pass: conversion
                    raise ProtocolError(f"{who} tile {i} slot {j}: staging slot {s} changed to {stage[s]}")
                cell = acc.get((j, q))
                if cell is not None and cell[0] != "free":
                    raise ProtocolError(f"{who} tile {i}: accumulator slot {j} still {cell[0]} for tile {cell[1]}")
                acc[(j, q)] = ["init", i, 0]
                st_empty[s].arrive()
                if mma_done[0] < i - 1:
                    raise ProtocolError(f"{who} tile {i}: A slot {j} rewritten before tile {i - 1}'s MMAs completed")
                A[(j, q)] = i
            if gate_t_ready:
                yield Wait(t_ready, i - 1, who)
            t_ready.arrive()

    def mma():
        prev, zl = None, 0
        for i, (_, key) in enumerate(items):
            if key != prev:
                yield Wait(z_full, zl, "mma")
                zl += 1
                prev = key
            yield Wait(t_ready, i, "mma")

            def done(i=i, key=key):
                for j in range(G):
                    for q in range(4):
                        if A.get((j, q)) != i:
                            raise ProtocolError(f"MMA tile {i}: A slot ({j},{q}) holds tile {A.get((j, q))}")
                        cell = acc.get((j, q))
                        if cell is None or cell[0] != "init" or cell[1] != i:
                            raise ProtocolError(f"MMA tile {i}: accumulator slot ({j},{q}) is {cell}")
                        cell[0] = "done"
                if z[0] != key:
                    raise ProtocolError(f"MMA tile {i}: table {z[0]} resident, {key} needed")
                mma_done[0] = i
            M.issue_mma(done)
            M.commit(acc_full)
            if i + 1 < T and items[i + 1][1] != key:
                M.commit(z_free)

    def epilogue(q, dh):
        who = f"epilogue(q{q},h{dh})"
        dn = n // 2
        for i, _ in enumerate(items):
            yield Wait(acc_full, i, who)
            for d0 in range(dh * dn, dh * dn + dn, 4):
                j = d0 // 8
                cell = acc.get((j, q))
                if cell is None or cell[0] not in ("done", "read") or cell[1] != i:
                    raise ProtocolError(f"{who} tile {i}: accumulator slot {j} is {cell}")
                cell[0] = "read"
                nxt = d0 + 4
                if nxt % 8 == 0 or nxt == dh * dn + dn:
                    cell[2] += 1
                    if cell[2] == (2 if dn < 8 else 1):
                        cell[0] = "free"
                    d_free[j].arrive()

    M.add_role("producer", producer())
    M.add_role("mma", mma())
    for q in range(4):
        for grp in range(2):
            M.add_role(f"conv{q}{grp}", converter(q, grp))
        for dh in range(2):
            M.add_role(f"epi{q}{dh}", epilogue(q, dh))
    M.run()
    return M.steps


def _slot_order(G):
    """Order in which the FP8X kernel loads and converts a tile's staging
    slots (its slot_of): 0, 1, 4, 5, 2, 3, 6, 7 at eight slots, in order
    otherwise."""
    if G == 8:
        return [(k & 1) | ((k >> 1) & 1) << 2 | (k >> 2) << 1 for k in range(8)]
    return list(range(G))


def fp8x_step(items, stages, seed, early_handback=False, slow=None):
    """The split-FP8 kernel (FP8X): as fp8_step (one accumulator handed back
    per slot through d_free, one t_ready gated on its previous phase, one
    acc_full), with the slots loaded and converted in the order the epilogue
    hands them back (_slot_order), the staging slot released before the wait
    for the slot's hand-off (its values are kept in registers), the A terms
    and init written after it, each group's packed scale cell written once all
    of its slots of the tile passed their hand-off, and an epilogue that loads
    up to two slots at a time and hands them back before storing.
    early_handback=True: the epilogue arrives on d_free before it has read
    the columns (a planted flaw)."""
    M = Machine(seed, slow)
    T = len(items)
    n = items[0][0]
    assert all(it[0] == n for it in items)
    G, ring = _groups(n), stages // 2
    order = _slot_order(G)
    dn = n // 2
    step = 16 if dn >= 16 else (8 if dn >= 8 else 4)
    dfree_count = 4 if dn % 8 == 0 else 8
    st_full = [Barrier(f"st_full[{s}]", 1) for s in range(stages)]
    st_empty = [Barrier(f"st_empty[{s}]", 4) for s in range(stages)]
    d_free = [Barrier(f"d_free[{j}]", dfree_count) for j in range(G)]
    t_ready, acc_full = Barrier("t_ready", 8), Barrier("acc_full", 1)
    z_full, z_free = Barrier("z_full", 1), Barrier("z_free", 1)
    stage = [None] * stages
    A, SA, acc, z, mma_done = {}, {}, {}, [None], [-1]

    def producer():
        prev, zr, gq = None, 0, [0, 0]
        for i, (_, key) in enumerate(items):
            if key != prev:
                if i > 0:
                    yield Wait(z_free, zr, "producer")
                    zr += 1
                z_full.expect_tx(1)

                def land_z(key=key):
                    z[0] = key
                    z_full.complete_tx(1)
                M.tma_load(land_z)
                prev = key
            for j in order:
                gr = j & 1
                local = gq[gr]
                gq[gr] += 1
                s = gr * ring + local % ring
                yield Wait(st_empty[s], local // ring - 1, "producer")
                st_full[s].expect_tx(1)

                def land(s=s, tag=(i, j)):
                    stage[s] = tag
                    st_full[s].complete_tx(1)
                M.tma_load(land)

    def converter(q, grp):
        who = f"converter(q{q},g{grp})"
        gq = 0
        mine = [j for j in order if j & 1 == grp]
        for i, _ in enumerate(items):
            for j in mine:
                local = gq
                gq += 1
                s = grp * ring + local % ring
                yield Wait(st_full[s], local // ring, who)
                if stage[s] != (i, j):
                    raise ProtocolError(f"{who} tile {i} slot {j}: staging slot {s} holds {stage[s]}")
                st_empty[s].arrive()                       # values kept in registers
                yield Wait(d_free[j], i - 1, who)
                cell = acc.get((j, q))
                if cell is not None and cell[0] != "free":
                    raise ProtocolError(f"{who} tile {i}: accumulator slot {j} still {cell[0]} for tile {cell[1]}")
                acc[(j, q)] = ["init", i, 0]
                if mma_done[0] < i - 1:
                    raise ProtocolError(f"{who} tile {i}: A slot {j} rewritten before tile {i - 1}'s MMAs completed")
                A[(j, q)] = i
            if mine:
                if mma_done[0] < i - 1:
                    raise ProtocolError(f"{who} tile {i}: scale cell rewritten before tile {i - 1}'s MMAs completed")
                SA[(grp, q)] = i
            yield Wait(t_ready, i - 1, who)
            t_ready.arrive()

    def mma():
        prev, zl = None, 0
        for i, (_, key) in enumerate(items):
            if key != prev:
                yield Wait(z_full, zl, "mma")
                zl += 1
                prev = key
            yield Wait(t_ready, i, "mma")

            def done(i=i, key=key):
                for j in range(G):
                    for q in range(4):
                        if A.get((j, q)) != i:
                            raise ProtocolError(f"MMA tile {i}: A slot ({j},{q}) holds tile {A.get((j, q))}")
                        cell = acc.get((j, q))
                        if cell is None or cell[0] != "init" or cell[1] != i:
                            raise ProtocolError(f"MMA tile {i}: accumulator slot ({j},{q}) is {cell}")
                        cell[0] = "done"
                for g in range(min(2, G)):
                    for q in range(4):
                        if SA.get((g, q)) != i:
                            raise ProtocolError(f"MMA tile {i}: scale cell ({g},{q}) holds tile {SA.get((g, q))}")
                if z[0] != key:
                    raise ProtocolError(f"MMA tile {i}: table {z[0]} resident, {key} needed")
                mma_done[0] = i
            M.issue_mma(done)
            M.commit(acc_full)
            if i + 1 < T and items[i + 1][1] != key:
                M.commit(z_free)

    def epilogue(q, dh):
        who = f"epilogue(q{q},h{dh})"
        for i, _ in enumerate(items):
            yield Wait(acc_full, i, who)
            for d0 in range(dh * dn, dh * dn + dn, step):
                slots = sorted({d // 8 for d in range(d0, d0 + step)})
                if early_handback:
                    for j in slots:
                        d_free[j].arrive()
                    yield None                              # the converters may run here
                for j in slots:
                    cell = acc.get((j, q))
                    if cell is None or cell[0] not in ("done", "read") or cell[1] != i:
                        raise ProtocolError(f"{who} tile {i}: accumulator slot {j} is {cell}")
                    cell[0] = "read"
                    cell[2] += 1
                    if cell[2] == (2 if dn < 8 else 1):
                        cell[0] = "free"
                if not early_handback:
                    for j in slots:
                        d_free[j].arrive()

    M.add_role("producer", producer())
    M.add_role("mma", mma())
    for q in range(4):
        for grp in range(2):
            M.add_role(f"conv{q}{grp}", converter(q, grp))
        for dh in range(2):
            M.add_role(f"epi{q}{dh}", epilogue(q, dh))
    M.run()
    return M.steps


def tf32_step(items, stages, seed, gate_ring=True, slow=None):
    """The 3xTF32 kernel (4n <= 128): two accumulators D and two exact-part
    regions E in TMEM, a ring of split state chunks in shared memory (Rg
    slots per converter group: 1 at n = 32, 2 below).  Per tile the
    converters wait for the epilogue of tile i - 2 (acc_empty[b]) before
    writing E[b]; per staging slot j (group j & 1) they wait for the slot's
    load and for the MMAs on their next ring slot (a_empty), write the hi and
    lo chunk and E's columns, release the staging slot and report the ring
    slot (a_full, count 4).  The MMA thread waits for acc_empty[b], then
    chunk by chunk on a_full (the first MMA of a tile starts D from zero)
    and commits a_empty per chunk, acc_full per tile.  gate_ring=False: the
    converters skip the a_empty wait (a planted flaw)."""
    M = Machine(seed, slow)
    T = len(items)
    n = items[0][0]
    assert all(it[0] == n for it in items) and 4 * n <= 128
    G, ring = _groups(n), stages // 2
    Rg = 1 if 4 * n >= 128 else 2
    st_full = [Barrier(f"st_full[{s}]", 1) for s in range(stages)]
    st_empty = [Barrier(f"st_empty[{s}]", 4) for s in range(stages)]
    a_full = [Barrier(f"a_full[{k}]", 4) for k in range(2 * Rg)]
    a_empty = [Barrier(f"a_empty[{k}]", 1) for k in range(2 * Rg)]
    acc_full = [Barrier(f"acc_full[{b}]", 1) for b in range(2)]
    acc_empty = [Barrier(f"acc_empty[{b}]", 8) for b in range(2)]
    z_full, z_free = Barrier("z_full", 1), Barrier("z_free", 1)
    stage = [None] * stages
    ringd, E, D, z = {}, {}, {}, [None]

    def producer():
        prev, zr, gq = None, 0, [0, 0]
        for i, (_, key) in enumerate(items):
            if key != prev:
                if i > 0:
                    yield Wait(z_free, zr, "producer")
                    zr += 1
                z_full.expect_tx(1)

                def land_z(key=key):
                    z[0] = key
                    z_full.complete_tx(1)
                M.tma_load(land_z)
                prev = key
            for j in range(G):
                gr = j & 1
                local = gq[gr]
                gq[gr] += 1
                s = gr * ring + local % ring
                yield Wait(st_empty[s], local // ring - 1, "producer")
                st_full[s].expect_tx(1)

                def land(s=s, tag=(i, j)):
                    stage[s] = tag
                    st_full[s].complete_tx(1)
                M.tma_load(land)

    def converter(q, grp):
        who = f"converter(q{q},g{grp})"
        gq, mc = 0, 0
        for i, _ in enumerate(items):
            b = i & 1
            yield Wait(acc_empty[b], (i >> 1) - 1, who)
            for j in range(grp, G, 2):
                local = gq
                gq += 1
                s = grp * ring + local % ring
                m = mc
                mc += 1
                k = grp * Rg + m % Rg
                yield Wait(st_full[s], local // ring, who)
                if gate_ring:
                    yield Wait(a_empty[k], m // Rg - 1, who)
                if stage[s] != (i, j):
                    raise ProtocolError(f"{who} tile {i} slot {j}: staging slot {s} holds {stage[s]}")
                cell = ringd.get((k, q))
                if cell is not None and cell[1] != "used":
                    raise ProtocolError(f"{who} tile {i} slot {j}: ring slot {k} still holds {cell} unread")
                ringd[(k, q)] = [(i, j), "written"]
                e = E.get((b, j, q))
                if e is not None and e[1] != "read":
                    raise ProtocolError(f"{who} tile {i}: exact part {b} slot {j} still {e}")
                E[(b, j, q)] = [i, "written"]
                st_empty[s].arrive()
                a_full[k].arrive()

    def mma():
        prev, zl, mc = None, 0, [0, 0]
        for i, (_, key) in enumerate(items):
            b = i & 1
            if key != prev:
                yield Wait(z_full, zl, "mma")
                zl += 1
                prev = key
            yield Wait(acc_empty[b], (i >> 1) - 1, "mma")
            for j in range(G):
                g = j & 1
                m = mc[g]
                mc[g] += 1
                k = g * Rg + m % Rg
                yield Wait(a_full[k], m // Rg, "mma")

                def done(i=i, b=b, j=j, k=k, key=key):
                    if z[0] != key:
                        raise ProtocolError(f"MMA tile {i}: table {z[0]} resident, {key} needed")
                    for q in range(4):
                        cell = ringd.get((k, q))
                        if cell is None or cell[0] != (i, j) or cell[1] != "written":
                            raise ProtocolError(f"MMA tile {i} chunk {j}: ring slot {k} ({q}) is {cell}")
                        cell[1] = "used"
                        for dh in range(2):
                            d = D.get((b, q, dh))
                            if j == 0:
                                if d is not None and d[1] != "read":
                                    raise ProtocolError(f"MMA tile {i}: accumulator {b} ({q},{dh}) still {d}")
                            elif d != [i, "partial"]:
                                raise ProtocolError(f"MMA tile {i} chunk {j}: accumulator {b} ({q},{dh}) is {d}")
                            D[(b, q, dh)] = [i, "done" if j == G - 1 else "partial"]
                M.issue_mma(done)
                M.commit(a_empty[k])
            M.commit(acc_full[b])
            if i + 1 < T and items[i + 1][1] != key:
                M.commit(z_free)

    def epilogue(q, dh):
        who = f"epilogue(q{q},h{dh})"
        for i, _ in enumerate(items):
            b = i & 1
            yield Wait(acc_full[b], i >> 1, who)
            d = D.get((b, q, dh))
            if d != [i, "done"]:
                raise ProtocolError(f"{who} tile {i}: accumulator {b} is {d}")
            d[1] = "read"
            for j in sorted({dd // 8 for dd in range(dh * n // 2, (dh + 1) * n // 2)}):
                e = E.get((b, j, q))
                if e is None or e[0] != i:
                    raise ProtocolError(f"{who} tile {i}: exact part {b} slot {j} is {e}")
                e[1] = "read"
            acc_empty[b].arrive()

    M.add_role("producer", producer())
    M.add_role("mma", mma())
    for q in range(4):
        for grp in range(2):
            M.add_role(f"conv{q}{grp}", converter(q, grp))
        for dh in range(2):
            M.add_role(f"epi{q}{dh}", epilogue(q, dh))
    M.run()
    return M.steps


def table_step(masks, stages, seed, gate_done=True, slow=None):
    """The adjoint's tensor-core table gradient: `masks` lists the class mask
    of each 32-site chunk a CTA reduces.  A producer thread fills a ring of
    `stages` staging slots (st_full by transaction bytes; it waits on
    st_empty, count 16, before reusing a slot); sixteen converter warps take
    each chunk's passes (one per class present), write operand buffer
    pass % 2 after the MMAs of the pass two before it completed (done), and
    report on op_full (count 16); the MMA thread waits op_full, issues and
    commits done; every converter warp releases the slot after the chunk's
    last pass.  gate_done=False drops the converters' wait on done (a planted
    flaw)."""
    M = Machine(seed, slow)
    W = 16
    st_full = [Barrier(f"st_full[{k}]", 1) for k in range(stages)]
    st_empty = [Barrier(f"st_empty[{k}]", W) for k in range(stages)]
    op_full = [Barrier(f"op_full[{b}]", W) for b in range(2)]
    done = [Barrier(f"done[{b}]", 1) for b in range(2)]
    stage = [None] * stages
    ops = {}                               # (buffer, warp) -> (pass, state)
    passes = [(ch, c) for ch, m in enumerate(masks) for c in range(4) if m >> c & 1]

    def producer():
        for it, _ in enumerate(masks):
            k = it % stages
            if it >= stages:
                yield Wait(st_empty[k], it // stages - 1, "producer")
            st_full[k].expect_tx(1)

            def land(k=k, it=it):
                stage[k] = it
                st_full[k].complete_tx(1)
            M.tma_load(land)

    def converter(w):
        who = f"converter{w}"
        p = 0
        for it, m in enumerate(masks):
            k = it % stages
            yield Wait(st_full[k], it // stages, who)
            for c in range(4):
                if not m >> c & 1:
                    continue
                b = p & 1
                if p >= 2 and gate_done:
                    yield Wait(done[b], (p >> 1) - 1, who)
                if stage[k] != it:
                    raise ProtocolError(f"{who} pass {p}: staging slot {k} holds chunk {stage[k]}, {it} needed")
                cell = ops.get((b, w))
                if cell is not None and cell[1] != "used":
                    raise ProtocolError(f"{who} pass {p}: operand buffer {b} still holds unread pass {cell[0]}")
                ops[(b, w)] = [p, "written"]
                op_full[b].arrive()
                p += 1
            st_empty[k].arrive()

    def mma():
        for p, (ch, c) in enumerate(passes):
            b = p & 1
            yield Wait(op_full[b], p >> 1, "mma")

            def read(p=p, b=b):
                for w in range(W):
                    cell = ops.get((b, w))
                    if cell is None or cell != [p, "written"]:
                        raise ProtocolError(f"MMA pass {p}: operand buffer {b} part {w} is {cell}")
                    cell[1] = "used"
            M.issue_mma(read)
            M.commit(done[b])

    M.add_role("producer", producer())
    M.add_role("mma", mma())
    for w in range(W):
        M.add_role(f"conv{w}", converter(w))
    M.run()
    return M.steps


def pair_step(keys, stages, seed, n=64, gate_acc_empty=True, slow=None):
    """The CTA-pair kernel (cta_group::2, bf16 state operand and split table):
    each entry of `keys` is one pair of tiles (one per CTA) of the same table
    key.  Per CTA: a producer (its half of the table and its own tile's
    staging), eight converter warps and eight epilogue warps as in bf16_step.
    The even CTA's MMA thread issues M = 256 MMAs reading both CTAs' A chunks
    and table halves and writing both accumulators; its commits arrive on the
    barriers of both CTAs.  The odd CTA's converters arrive on a local
    barrier that one thread forwards to the even CTA's t_ready (count 9); the
    odd producer forwards the completion of its table half to the even z_full
    (count 2).  gate_acc_empty=False lets the converters write a tile's
    accumulator init without waiting for the epilogue of two tiles before (a
    planted flaw)."""
    M = Machine(seed, slow)
    T = len(keys)
    G, C, ring = _groups(n), _chunks(n), stages // 2
    R = (0, 1)
    st_full = {(r, s): Barrier(f"st_full[{r}][{s}]", 1) for r in R for s in range(stages)}
    st_empty = {(r, s): Barrier(f"st_empty[{r}][{s}]", 4) for r in R for s in range(stages)}
    a_empty = {(r, c): Barrier(f"a_empty[{r}][{c}]", 1) for r in R for c in range(C)}
    acc_full = {(r, b): Barrier(f"acc_full[{r}][{b}]", 1) for r in R for b in range(2)}
    acc_empty = {(r, b): Barrier(f"acc_empty[{r}][{b}]", 8) for r in R for b in range(2)}
    z_free = {r: Barrier(f"z_free[{r}]", 1) for r in R}
    t_ready = [Barrier(f"t_ready[{b}]", 9) for b in range(2)]          # even CTA
    t_local = [Barrier(f"t_local[{b}]", 8) for b in range(2)]          # odd CTA
    z_full = {0: Barrier("z_full[0]", 2), 1: Barrier("z_full[1]", 1)}
    stage = {(r, s): None for r in R for s in range(stages)}
    A, acc, z = {}, {}, {0: None, 1: None}

    def mcast(bars):
        for bar in bars:
            M.commit(bar)

    def producer(r):
        who = f"producer{r}"
        prev, zr, zl, gq = None, 0, 0, [0, 0]
        for i, key in enumerate(keys):
            if key != prev:
                if i > 0:
                    yield Wait(z_free[r], zr, who)
                    zr += 1
                z_full[r].expect_tx(1)

                def land_z(key=key, r=r):
                    z[r] = key
                    z_full[r].complete_tx(1)
                M.tma_load(land_z)
                if r == 1:
                    yield Wait(z_full[1], zl, who)
                    z_full[0].arrive()                      # forward to the even CTA
                zl += 1
                prev = key
            for j in range(G):
                gr = j & 1
                local = gq[gr]
                gq[gr] += 1
                s = gr * ring + local % ring
                yield Wait(st_empty[(r, s)], local // ring - 1, who)
                st_full[(r, s)].expect_tx(1)

                def land(r=r, s=s, tag=(i, j)):
                    stage[(r, s)] = tag
                    st_full[(r, s)].complete_tx(1)
                M.tma_load(land)

    def converter(r, q, grp):
        who = f"converter{r}(q{q},g{grp})"
        gq = 0
        for i, key in enumerate(keys):
            b = i & 1
            if gate_acc_empty:
                yield Wait(acc_empty[(r, b)], (i >> 1) - 1, who)
            for c in range(C):
                j = 2 * c + grp
                local = gq
                gq += 1
                s = grp * ring + local % ring
                yield Wait(st_full[(r, s)], local // ring, who)
                if stage[(r, s)] != (i, j):
                    raise ProtocolError(f"{who} tile {i} slot {j}: staging holds {stage[(r, s)]}")
                cell = acc.get((r, b, j, q))
                if cell is not None and cell[0] != "free":
                    raise ProtocolError(f"{who} tile {i}: accumulator {b} slot {j} still {cell[0]}")
                acc[(r, b, j, q)] = ["init", i, 0]
                st_empty[(r, s)].arrive()
                yield Wait(a_empty[(r, c)], i - 1, who)
                A[(r, c, grp, q)] = i
            (t_ready[b] if r == 0 else t_local[b]).arrive()

    def forwarder():
        for i, _ in enumerate(keys):
            b = i & 1
            yield Wait(t_local[b], i >> 1, "forwarder")
            t_ready[b].arrive()

    def mma():
        prev, zl = None, 0
        for i, key in enumerate(keys):
            b = i & 1
            if key != prev:
                yield Wait(z_full[0], zl, "mma")
                zl += 1
                prev = key
            yield Wait(t_ready[b], i >> 1, "mma")
            for c in range(C):
                def done(i=i, b=b, c=c, key=key):
                    for r in R:
                        if z[r] != key:
                            raise ProtocolError(f"MMA pair {i}: CTA {r} holds table {z[r]}, {key} needed")
                        for grp in (0, 1):
                            for q in range(4):
                                if A.get((r, c, grp, q)) != i:
                                    raise ProtocolError(f"MMA pair {i} chunk {c}: CTA {r} A part ({grp},{q}) holds "
                                                        f"{A.get((r, c, grp, q))}")
                        for j in range(G):
                            for q in range(4):
                                cell = acc.get((r, b, j, q))
                                if cell is None or cell[1] != i or cell[0] not in ("init", "partial"):
                                    raise ProtocolError(f"MMA pair {i}: CTA {r} accumulator slot {j} is {cell}")
                                cell[0] = "done" if c == C - 1 else "partial"
                M.issue_mma(done)
                mcast([a_empty[(0, c)], a_empty[(1, c)]])
            mcast([acc_full[(0, b)], acc_full[(1, b)]])
            if i + 1 < T and keys[i + 1] != key:
                mcast([z_free[0], z_free[1]])

    def epilogue(r, q, dh):
        who = f"epilogue{r}(q{q},h{dh})"
        dn = n // 2
        for i, _ in enumerate(keys):
            b = i & 1
            yield Wait(acc_full[(r, b)], i >> 1, who)
            for j in sorted({d // 8 for d in range(dh * dn, dh * dn + dn)}):
                cell = acc.get((r, b, j, q))
                if cell is None or cell[0] != "done" or cell[1] != i:
                    raise ProtocolError(f"{who} tile {i}: accumulator {b} slot {j} is {cell}")
                cell[0] = "free"
            acc_empty[(r, b)].arrive()

    M.add_role("mma", mma())
    M.add_role("forwarder", forwarder())
    for r in R:
        M.add_role(f"producer{r}", producer(r))
        for q in range(4):
            for grp in range(2):
                M.add_role(f"conv{r}{q}{grp}", converter(r, q, grp))
            for dh in range(2):
                M.add_role(f"epi{r}{q}{dh}", epilogue(r, q, dh))
    M.run()
    return M.steps
