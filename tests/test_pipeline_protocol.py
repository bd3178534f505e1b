"""The barrier protocol of the FP32 tensor-core pipeline (`k_tc_gemm<MODE, 1>`),
checked on the CPU by a model with random interleavings.

The model has the kernel's agents:
  - the producer: one copy per term into a ring of `nst` stages;
  - four splitter warps: [B; B_lo] into one of `kASlots` TMEM A slots, with
    the look-ahead that tests the next term's stage and slot barriers;
  - two MMA issuers, taking the terms by parity;
  - four epilogue warps, reading one of `nacc` TMEM accumulators per term.

They use mbarriers with the PTX phase semantics. A barrier counts arrivals
(and, for a copy, transaction bytes) and completes a phase when both are
done. `try_wait.parity(P)` succeeds once the phase of parity P has completed,
which on a fresh barrier holds for P = 1. `tcgen05.commit` arrives when all of
the committing thread's earlier MMAs have finished. Each agent waits with the
kernel's own stage, slot, accumulator and parity formulas.

The checker asserts what the waits exist for:
  - no stage is refilled before the MMA that read it finished;
  - no A slot is rewritten before its MMA finished;
  - no accumulator is overwritten before all epilogue warps read it;
  - every consumer sees the term it expects;
  - every run ends without deadlock.

Each planted mistake must be caught: a wrong parity in any agent, a
look-ahead that ignores the stage test, and a look-ahead that tests the
wrong slot. The model also shows that the two issuers do not need even
accumulator and slot counts: every reuse of a barrier waits on the previous
use's consumer, so its arrivals come in order either way."""
import random

import pytest


class Barrier:
    def __init__(self, count):
        self.count, self.arrived, self.tx, self.phase = count, 0, 0, 0  # phase = completed phases

    def _maybe_complete(self):
        if self.arrived == self.count and self.tx == 0:
            self.phase += 1
            self.arrived = 0

    def arrive(self, tx=0):
        self.arrived += 1
        self.tx += tx
        self._maybe_complete()

    def complete_tx(self, tx):
        self.tx -= tx
        self._maybe_complete()

    def test(self, parity):
        return (self.phase & 1) != parity


class Hazard(AssertionError):
    pass


def run_pipeline(T, nst=6, nacc=4, nslots=4, seed=0, mutate=None, max_steps=200000, splitter_warps=True,
                 items=None):
    """Simulate one CTA on T terms; raises Hazard or returns normally.  Without
    splitter warps (the BF16 kernel) the issuers wait on the copies directly.
    With `items` (term counts of the CTA's items; the BF16 kernel's protocol)
    one issuer accumulates all terms of an item into one accumulator and the
    epilogue reads each accumulator once per item."""
    if items is not None:
        T = sum(items)
        splitter_warps = False
    rng = random.Random(seed)
    full = [Barrier(1) for _ in range(nst)]
    split = [Barrier(4) for _ in range(nst)]
    empty = [Barrier(1) for _ in range(nst)]
    aempty = [Barrier(1) for _ in range(nslots)]
    accf = [Barrier(1) for _ in range(nacc)]
    acce = [Barrier(4) for _ in range(nacc)]
    END = -1
    stage_term = [None] * nst          # term whose data sits (or is landing) in the stage
    stage_landed = [False] * nst
    stage_readers = [0] * nst          # MMAs in flight that read the stage
    slot_term = [[None] * 4 for _ in range(nslots)]  # per splitter warp: term written to the slot
    slot_readers = [0] * nslots
    acc_term = [None] * nacc           # term whose result the accumulator holds (None: being written)
    acc_unread = [0] * nacc            # epilogue warps that still have to read it
    pending = []                       # async events: [remaining delay, callback]
    mma_queue = {0: [], 1: []}         # per issuer, in-order MMA completions

    def later(fn, lo=1, hi=6):
        pending.append([rng.randint(lo, hi), fn])

    def W(bar, parity):
        return ("wait", bar, parity)

    # ---------------- producer ----------------
    def producer():
        stage, phase = 0, 0
        for t in range(T):
            p = phase if mutate == "producer_parity" else phase ^ 1
            yield W(empty[stage], p)
            if stage_readers[stage] or (stage_term[stage] is not None and not consumed.get(stage_term[stage])):
                raise Hazard(f"stage {stage} refilled for term {t} before term {stage_term[stage]} was consumed")
            stage_term[stage], stage_landed[stage] = t, False
            full[stage].arrive(tx=1)

            def land(s=stage, tt=t):
                if stage_term[s] != tt:
                    raise Hazard("copy landed in a stage that moved on")
                stage_landed[s] = True
                full[s].complete_tx(1)
            later(land, 2, 12)
            stage += 1
            if stage == nst:
                stage, phase = 0, phase ^ 1
        yield W(empty[stage], phase ^ 1)
        stage_term[stage], stage_landed[stage] = END, True
        full[stage].arrive()

    # ---------------- splitter warps ----------------
    def splitter(w):
        stage, phase, sit, pre = 0, 0, 0, False
        while True:
            if not pre:
                yield W(full[stage], phase)
            if stage_term[stage] == END:
                split[stage].arrive()
                return
            if not stage_landed[stage] or stage_term[stage] != sit:
                raise Hazard(f"splitter {w} read stage {stage} for term {sit}, found {stage_term[stage]}")
            a = sit % nslots
            if not pre:
                yield W(aempty[a], ((sit // nslots) & 1) ^ (0 if mutate == "splitter_parity" else 1))
            nstage = 0 if stage + 1 == nst else stage + 1
            nphase = phase ^ 1 if stage + 1 == nst else phase
            pf = full[nstage].test(nphase)
            nx = sit + (2 if mutate == "probe_wrong_slot" else 1)
            pa = aempty[nx % nslots].test((((sit + 1) // nslots) & 1) ^ 1)
            yield ("step",)
            if slot_readers[a]:
                raise Hazard(f"A slot {a} rewritten for term {sit} while an MMA reads it")
            slot_term[a][w] = sit
            yield ("step",)
            sit += 1
            pre = (pf or mutate == "no_lookahead_test") and pa
            split[stage].arrive()
            stage += 1
            if stage == nst:
                stage, phase = 0, phase ^ 1

    consumed = {}

    # ---------------- MMA issuers ----------------
    def issuer(j):
        for it in range(j, T, 2):
            stage = it % nst
            yield W(split[stage] if splitter_warps else full[stage], (it // nst) & 1)
            acc = it % nacc
            yield W(acce[acc], ((it // nacc) & 1) ^ (0 if mutate == "issuer_acce_parity" else 1))
            a = it % nslots
            if stage_term[stage] != it or not stage_landed[stage]:
                raise Hazard(f"MMA of term {it} found stage {stage} holding {stage_term[stage]}")
            if splitter_warps and any(x != it for x in slot_term[a]):
                raise Hazard(f"MMA of term {it} found A slot {a} holding {slot_term[a]}")
            if acc_unread[acc]:
                raise Hazard(f"MMA of term {it} overwrites accumulator {acc} before its epilogue read")
            stage_readers[stage] += 1
            slot_readers[a] += 1
            acc_term[acc] = None
            mma_queue[j].append(it)

            def finish(j=j):
                # MMAs of one issuer complete in order; the commit arrives with them
                t2 = mma_queue[j].pop(0)
                s2, a2, c2 = t2 % nst, t2 % nslots, t2 % nacc
                stage_readers[s2] -= 1
                slot_readers[a2] -= 1
                consumed[t2] = True
                acc_term[c2], acc_unread[c2] = t2, 4
                empty[s2].arrive()
                aempty[a2].arrive()
                accf[c2].arrive()
            later(finish, 1, 8)
            yield ("step",)

    # ---------------- epilogue warps ----------------
    def epilogue(e):
        for it in range(T):
            acc = it % nacc
            yield W(accf[acc], ((it // nacc) & 1) ^ (1 if mutate == "epilogue_parity" else 0))
            if acc_term[acc] != it:
                raise Hazard(f"epilogue {e} expected term {it} in accumulator {acc}, found {acc_term[acc]}")
            yield ("step",)
            acc_unread[acc] -= 1
            acce[acc].arrive()

    # ---------------- per-item accumulation (BF16): one issuer, one accumulator per item ----------------
    def issuer_items():
        it = 0
        for idx, cnt in enumerate(items):
            acc = (it if mutate == "acc_by_term" else idx) % nacc
            for t in range(cnt):
                stage = it % nst
                yield W(full[stage], (it // nst) & 1)
                if t == 0:
                    yield W(acce[acc], ((idx // nacc) & 1) ^ (0 if mutate == "issuer_acce_parity" else 1))
                    if acc_unread[acc]:
                        raise Hazard(f"item {idx} overwrites accumulator {acc} before its epilogue read")
                    acc_term[acc] = None
                if stage_term[stage] != it or not stage_landed[stage]:
                    raise Hazard(f"MMA of term {it} found stage {stage} holding {stage_term[stage]}")
                if acc_term[acc] is not None:
                    raise Hazard(f"term {it} accumulates into accumulator {acc} that holds item {acc_term[acc]}")
                stage_readers[stage] += 1
                last = t == cnt - 1
                mma_queue[0].append((it, acc, idx, last))

                def finish():
                    t2, c2, i2, l2 = mma_queue[0].pop(0)
                    s2 = t2 % nst
                    stage_readers[s2] -= 1
                    consumed[t2] = True
                    empty[s2].arrive()
                    if l2:
                        acc_term[c2], acc_unread[c2] = i2, 4
                        accf[c2].arrive()
                later(finish, 1, 8)
                it += 1
                yield ("step",)

    def epilogue_items(e):
        for idx in range(len(items)):
            acc = idx % nacc
            yield W(accf[acc], ((idx // nacc) & 1) ^ (1 if mutate == "epilogue_parity" else 0))
            if acc_term[acc] != idx:
                raise Hazard(f"epilogue {e} expected item {idx} in accumulator {acc}, found {acc_term[acc]}")
            yield ("step",)
            acc_unread[acc] -= 1
            acce[acc].arrive()

    if items is not None:
        agents = [producer(), issuer_items()] + [epilogue_items(e) for e in range(4)]
    else:
        agents = ([producer()] + ([splitter(w) for w in range(4)] if splitter_warps else []) + [issuer(0), issuer(1)]
                  + [epilogue(e) for e in range(4)])
    state = [None] * len(agents)   # the pending request of each agent
    done = [False] * len(agents)
    for step in range(max_steps):
        runnable = []
        for i, g in enumerate(agents):
            if done[i]:
                continue
            req = state[i]
            if req is None or req[0] == "step" or (req[0] == "wait" and req[1].test(req[2])):
                runnable.append(i)
        if not runnable and not pending and all(done):
            return
        if not runnable and not pending:
            raise Hazard("deadlock: " + ", ".join(f"agent {i} waits" for i in range(len(agents)) if not done[i]))
        if pending and (not runnable or rng.random() < 0.3):
            k = rng.randrange(len(pending))
            pending[k][0] -= 1
            if pending[k][0] <= 0:
                pending.pop(k)[1]()
            continue
        i = rng.choice(runnable)
        try:
            state[i] = next(agents[i])
        except StopIteration:
            done[i] = True
    raise Hazard("no progress within the step limit")


# stage counts the kernel takes (6 and 4 for FP32, 14 and 9 for BF16), and
# small and odd ones
@pytest.mark.parametrize("T", [1, 2, 5, 6, 7, 13, 40])
@pytest.mark.parametrize("nst", [2, 3, 4, 5, 6, 9, 14])
def test_protocol_is_hazard_and_deadlock_free(T, nst):
    for seed in range(12):
        run_pipeline(T, nst=nst, seed=seed)


@pytest.mark.parametrize("nacc,nslots", [(3, 4), (4, 3), (2, 2), (5, 5)])
def test_odd_and_small_ring_sizes_are_safe(nacc, nslots):
    for seed in range(12):
        run_pipeline(30, nacc=nacc, nslots=nslots, seed=seed)


@pytest.mark.parametrize("mutate", ["producer_parity", "splitter_parity", "issuer_acce_parity", "epilogue_parity",
                                    "no_lookahead_test", "probe_wrong_slot"])
def test_planted_protocol_mistakes_are_caught(mutate):
    caught = False
    for seed in range(60):
        try:
            run_pipeline(24, seed=seed, mutate=mutate)
        except Hazard:
            caught = True
            break
    assert caught, mutate


# The BF16 kernel has no splitter: each issuer waits on the copy of its own
# term, and the stage's previous use may belong to the other issuer.  A parity
# wait is then safe only while that earlier copy is known to have landed.  It
# is when the stage count is even (each stage stays with one issuer), and when
# nst >= nacc + 2 (the issuer's accumulator wait for its previous term covers
# the earlier copy).  The kernel's BF16 stage counts are 14, and 9 for R > 64.
@pytest.mark.parametrize("nst", [4, 6, 7, 9, 14])
def test_bf16_protocol_with_its_stage_counts(nst):
    for T in (1, 7, 40):
        for seed in range(12):
            run_pipeline(T, nst=nst, seed=seed, splitter_warps=False)


@pytest.mark.parametrize("nst", [3, 5])
def test_bf16_protocol_unsafe_with_few_odd_stages(nst):
    caught = False
    for seed in range(80):
        try:
            run_pipeline(40, nst=nst, seed=seed, splitter_warps=False)
        except Hazard:
            caught = True
            break
    assert caught


# The BF16 kernel accumulates all terms of an item in one TMEM accumulator (its
# error budget is far above the accumulator's rounding): one issuer takes every
# term in order, and the epilogue reads one accumulator per item.  One issuer
# waits on every stage in order, so any stage count is safe.
ITEM_SHAPES = [[1], [3], [1, 1, 1, 1, 1, 1, 1], [5, 1, 7, 2, 13, 1, 1, 4], [2] * 20, [17, 3, 9]]


@pytest.mark.parametrize("nst", [2, 3, 4, 5, 9, 14])
@pytest.mark.parametrize("shape", range(len(ITEM_SHAPES)))
def test_bf16_item_protocol_is_hazard_and_deadlock_free(nst, shape):
    for nacc in (2, 3, 4):
        for seed in range(8):
            run_pipeline(0, nst=nst, nacc=nacc, seed=seed, items=ITEM_SHAPES[shape])


@pytest.mark.parametrize("mutate", ["producer_parity", "issuer_acce_parity", "epilogue_parity", "acc_by_term"])
def test_bf16_item_protocol_planted_mistakes_are_caught(mutate):
    caught = False
    for seed in range(80):
        try:
            run_pipeline(0, nst=4, seed=seed, mutate=mutate, items=[5, 1, 7, 2, 13, 1, 1, 4, 3, 3])
        except Hazard:
            caught = True
            break
    assert caught, mutate

