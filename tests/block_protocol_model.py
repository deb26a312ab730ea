"""Randomised-interleaving model of one thread block's protocol in the persistent filter kernels
(a test aid; it shares no code with the CUDA library).

A block has one coordinator warp and W compute warps; each compute warp filters one group of every
tile the block takes.  The model keeps the synchronisation the kernels use and checks it under
random schedules:

* tickets: tile numbers drawn from a global counter into a ring of R slots, each announced on its
  own mbarrier (phase k // R of barrier k mod R for iteration k); the block's first A tickets are
  drawn at start, and the fold of iteration k draws that of iteration k + A;
* the fold: the last compute warp of iteration k to finish its pass arrives on the local-carry
  barrier of slot k mod NS, which the coordinator waits on;
* the coordinator resolves the tile (a random delay stands for its lookback over other blocks) and
  posts the groups' incoming states in slot k mod NS, announced on incoming-state barrier k mod NZ
  (NZ = NS in the kernels: one barrier per slot);
* the correction of the tile of iteration k runs in iteration k + D - 1 of each compute warp, from
  row buffer k mod D, after that warp's fold of its own later tile;
* the samples of the next tile go to row buffer (k + 1) mod D: held in registers and stored at the
  start of iteration k + 1 (the kernels), or, with `load="after_correction"`, loaded straight into
  that buffer once the correction of iteration k has freed it (`load="early"` issues that load
  before the correction: a planted mistake).

mbarrier waits are on a phase parity: a wait for phase m of a barrier that has already completed
phase m + 1 waits for another phase, which never comes.  Every wait therefore checks that its
barrier is at most one phase ahead.  Slots (tickets, local carries, incoming states) and row
buffers are checked not to be overwritten before their readers are done, and every (tile, warp)
must be corrected exactly once.  The model has no notion of time beyond the order of steps: the
scheduler gives the agents shares of the steps that it redraws from a heavy-tailed distribution
every few dozen steps, so that any agent is now and then starved for long stretches, as a warp can
be on the GPU.
"""
import random


class Hazard(Exception):
    """A schedule under which the protocol would misbehave on the GPU."""


def run_block(W, n_tiles, *, R=8, A=3, D=2, NS=2, NZ=2, load="registers", seed=0, max_steps=500000):
    """One block taking every tile of a launch of `n_tiles` tiles.  Raises Hazard on a violation."""
    rng = random.Random(seed)
    bar_ticket = [0] * R        # completed phases per barrier
    bar_local = [0] * NS
    bar_zready = [0] * NZ
    counter = [0]
    ring = [None] * R           # (iteration, tile) of the current occupant
    ring_readers = [set() for _ in range(R)]
    a_slot = [[None] * W for _ in range(NS)]  # iteration whose local carry each warp left there
    a_consumed = [True] * NS
    z_slot = [None] * NS
    z_readers = [set() for _ in range(NS)]
    fold_count = [0] * NS
    corrected = []

    def draw():
        t = counter[0]
        counter[0] += 1
        return t if t < n_tiles else -1

    def post_ticket(k):
        j = k % R
        if ring[j] is not None and ring[j][1] >= 0:
            everyone = {"coordinator"} | set(range(W))
            if not everyone <= ring_readers[j]:
                raise Hazard(f"ticket slot {j} of iteration {ring[j][0]} overwritten by {k} "
                             f"before {everyone - ring_readers[j]} read it")
        ring[j] = (k, draw())
        ring_readers[j] = set()
        bar_ticket[j] += 1

    def take_ticket(k, who):
        j = k % R
        if ring[j] is None or ring[j][0] != k:
            raise Hazard(f"{who} reads ticket slot {j} for iteration {k}, which holds {ring[j]}")
        ring_readers[j].add(who)
        return ring[j][1]

    def wait(bars, b, m, who):
        if bars[b] > m + 1:
            raise Hazard(f"{who} waits for phase {m} of a barrier that has completed {bars[b]}")
        while bars[b] < m + 1:
            yield

    def pause(n):
        for _ in range(rng.randrange(0, n)):
            yield

    def coordinator():
        k = 0
        while True:
            yield from wait(bar_ticket, k % R, k // R, "coordinator")
            if take_ticket(k, "coordinator") < 0:
                return
            s = k % NS
            yield from wait(bar_local, s, k // NS, "coordinator")
            if any(a != k for a in a_slot[s]):
                raise Hazard(f"coordinator {k}: local carries of iterations {a_slot[s]}")
            a_consumed[s] = True
            yield from pause(30)  # the lookback over other blocks' tiles
            if z_slot[s] is not None and len(z_readers[s]) < W:
                raise Hazard(f"coordinator {k}: incoming states of iteration {z_slot[s]} not yet read")
            z_slot[s] = k
            z_readers[s] = set()
            bar_zready[k % NZ] += 1
            k += 1

    def compute(w):
        rows = [None] * D  # tile held by each row buffer
        yield from wait(bar_ticket, 0, 0, w)
        tile = take_ticket(0, w)
        if tile < 0:
            return
        pending = []       # (iteration, tile) awaiting correction, oldest first

        def correct(j, t):
            yield from wait(bar_zready, j % NZ, j // NZ, w)
            z = j % NS
            if z_slot[z] != j:
                raise Hazard(f"warp {w} corrects iteration {j} with incoming states of {z_slot[z]}")
            z_readers[z].add(w)
            if rows[j % D] != t:
                raise Hazard(f"warp {w} corrects tile {t} from a buffer holding {rows[j % D]}")
            yield from pause(5)
            rows[j % D] = None
            corrected.append((t, w))

        def land(k, t):  # the samples of tile t arrive in the buffer of iteration k
            if rows[k % D] is not None:
                raise Hazard(f"warp {w}: tile {t} lands in buffer {k % D}, which still holds tile {rows[k % D]}")
            rows[k % D] = t

        k = 0
        landed = load == "registers"
        if not landed:
            land(0, tile)
        while True:
            if landed:
                land(k, tile)
            landed = load == "registers"
            yield from wait(bar_ticket, (k + 1) % R, (k + 1) // R, w)
            nxt = take_ticket(k + 1, w)
            if load == "early" and nxt >= 0:
                land(k + 1, nxt)
            elif load == "after_correction" and nxt >= 0 and len(pending) < D - 1:
                land(k + 1, nxt)  # the buffer is free from the start
            yield from pause(10)  # the pass over the group and the lane scan
            s = k % NS
            if a_slot[s][w] is not None and not a_consumed[s]:
                raise Hazard(f"warp {w}, iteration {k}: local-carry slot {s} of iteration "
                             f"{a_slot[s][w]} not yet consumed")
            a_slot[s][w] = k
            fold_count[s] += 1
            if fold_count[s] == W:  # the last warp folds
                fold_count[s] = 0
                a_consumed[s] = False
                post_ticket(k + A)
                bar_local[s] += 1
            pending.append((k, tile))
            yield from pause(4)  # between the fold and the wait for the incoming states
            if len(pending) == D:
                yield from correct(*pending.pop(0))
                if load == "after_correction" and nxt >= 0:
                    land(k + 1, nxt)
            if nxt < 0:
                break
            tile = nxt
            k += 1
        while pending:
            yield from correct(*pending.pop(0))

    for k in range(A):
        post_ticket(k)
    agents = [coordinator()] + [compute(w) for w in range(W)]
    alive = list(range(len(agents)))
    steps = 0
    share = [1.0] * len(agents)
    while alive:
        if steps % 40 == 0:
            share = [rng.expovariate(1.0) ** 4 + 1e-9 for _ in agents]
        i = rng.choices(alive, weights=[share[a] for a in alive])[0]
        try:
            next(agents[i])
        except StopIteration:
            alive.remove(i)
        steps += 1
        if steps > max_steps:
            raise Hazard("no progress: every agent waits")
    if sorted(corrected) != sorted((t, w) for t in range(n_tiles) for w in range(W)):
        raise Hazard("not every (tile, warp) was corrected exactly once")
