"""The scheduling rules of the persistent PCG kernels, played out on the host
(no GPU): a discrete-event model of CTAs taking items from a counter under
the kernels' wait rules, for random batches, solve lengths, CTA counts and
item durations.  It checks the properties the kernels' comments argue:
every wait ends (no state where all CTAs wait), every env runs exactly the
iterations its solve needs within the launch, an env's update of round k
starts only after all its products of round k, and its products of round
k + 1 only after its update of round k.

The rules modelled are those of k_pcg_multi (W rounds of [pair groups,
row items, update items], each env after env; products of round k wait for
the env's completed-update count to reach k, updates of round k for its
product count to reach (k + 1) x its product items; an env whose solve
ended skips its later items) and of k_pcg_iter in ready-slot order (the
env whose last product finishes publishes its update items into slots that
CTAs take in order)."""
import random

import pytest


def _simulate_multi(env_items, solve_len, W, n_cta, rng):
    """env_items: per env (row items, pair groups); solve_len: per env the
    iterations until its solve stops.  Returns per env the iterations run
    and the event log."""
    n_env = len(env_items)
    items = []
    for k in range(W):
        for e, (_, p) in enumerate(env_items):
            items += [("prod", k, e)] * p
        for e, (r, _) in enumerate(env_items):
            items += [("prod", k, e)] * r
        for e, (r, _) in enumerate(env_items):
            items += [("upd", k, e)] * r
    need = [r + p for r, p in env_items]
    phase = [0] * n_env          # products completed, across the launch
    updk = [0] * n_env           # update rounds completed
    upd_done = [[0] * W for _ in range(n_env)]
    pcg = [solve_len[e] > 0 for e in range(n_env)]
    iters = [0] * n_env
    nxt = 0
    ctas = [None] * n_cta        # (item, remaining time) or None
    log = []
    t = 0
    while True:
        # idle CTAs take the next item
        for c in range(n_cta):
            if ctas[c] is None and nxt < len(items):
                ctas[c] = [items[nxt], None]
                nxt += 1
        if all(c is None for c in ctas) and nxt >= len(items):
            break
        progressed = False
        for c in range(n_cta):
            if ctas[c] is None:
                continue
            (kind, k, e), rem = ctas[c]
            if rem is None:
                # the item's wait: ends when the condition holds or the env stopped
                if not pcg[e]:
                    ctas[c] = None        # skip
                    progressed = True
                    continue
                ready = updk[e] >= k if kind == "prod" else phase[e] >= (k + 1) * need[e]
                if not ready:
                    continue
                if kind == "upd":
                    assert phase[e] == (k + 1) * need[e]      # all products of round k, none of k + 1
                    log.append(("upd_start", k, e))
                else:
                    assert updk[e] == k                      # the previous update, not a later one
                ctas[c][1] = rng.randint(1, 5)
                progressed = True
                continue
            ctas[c][1] -= 1
            progressed = True
            if ctas[c][1] > 0:
                continue
            ctas[c] = None
            if kind == "prod":
                phase[e] += 1
            else:
                upd_done[e][k] += 1
                if upd_done[e][k] == env_items[e][0]:     # the env's last update CTA of the round
                    iters[e] += 1
                    if iters[e] >= solve_len[e]:
                        pcg[e] = False                    # cleared before the round is counted
                    updk[e] += 1
        assert progressed, "every CTA waits: a wait that never ends"
        t += 1
    return iters, log


@pytest.mark.parametrize("seed", range(40))
def test_multi_iteration_rules_end_every_wait_and_run_each_solve(seed):
    rng = random.Random(seed)
    n_env = rng.randint(1, 9)
    env_items = [(rng.randint(1, 6), rng.randint(0, 3)) for _ in range(n_env)]
    solve_len = [rng.randint(0, 12) for _ in range(n_env)]
    W = rng.choice([1, 2, 4, 8])
    n_cta = rng.randint(1, 40)
    iters, log = _simulate_multi(env_items, solve_len, W, n_cta, rng)
    assert iters == [min(s, W) for s in solve_len]
    # an env's update rounds start in order
    for e in range(n_env):
        ks = [k for kind, k, ee in log if ee == e]
        assert ks == sorted(ks)


def _simulate_ready_slots(env_items, n_cta, rng):
    """k_pcg_iter, ready-slot order: products first (pairs, then rows), the
    env's last product publishes its update items, CTAs then take slots in
    order and wait only for their slot to be written."""
    n_env = len(env_items)
    prods = []
    for e, (_, p) in enumerate(env_items):
        prods += [e] * p
    for e, (r, _) in enumerate(env_items):
        prods += [e] * r
    need = [r + p for r, p in env_items]
    n_upd = sum(r for r, _ in env_items)
    phase = [0] * n_env
    slots = [None] * n_upd
    alloc = 0
    nxt, take = 0, 0
    ctas = [None] * n_cta
    done_upd = [0] * n_env
    order = []
    while True:
        for c in range(n_cta):
            if ctas[c] is None:
                if nxt < len(prods):
                    ctas[c] = ["prod", prods[nxt], rng.randint(1, 5)]
                    nxt += 1
                elif take < n_upd:
                    ctas[c] = ["slot", take, None]
                    take += 1
        if all(c is None for c in ctas):
            break
        progressed = False
        for c in range(n_cta):
            if ctas[c] is None:
                continue
            kind, x, rem = ctas[c]
            if kind == "slot" and rem is None:
                if slots[x] is None:
                    continue              # waits for its slot
                e = slots[x]
                assert phase[e] == need[e]   # its env's products are all in
                order.append(e)
                ctas[c] = ["upd", e, rng.randint(1, 5)]
                progressed = True
                continue
            ctas[c][2] -= 1
            progressed = True
            if ctas[c][2] > 0:
                continue
            ctas[c] = None
            if kind == "prod":
                phase[x] += 1
                if phase[x] == need[x]:   # the env's last product publishes
                    for j in range(env_items[x][0]):
                        slots[alloc + j] = x
                    alloc += env_items[x][0]
            else:
                done_upd[x] += 1
        assert progressed, "every CTA waits: a wait that never ends"
    assert alloc == n_upd and all(s is not None for s in slots)
    assert done_upd == [r for r, _ in env_items]
    return order


@pytest.mark.parametrize("seed", range(40))
def test_ready_slot_rules_end_every_wait_and_update_every_row_item(seed):
    rng = random.Random(1000 + seed)
    n_env = rng.randint(1, 9)
    env_items = [(rng.randint(1, 6), rng.randint(0, 3)) for _ in range(n_env)]
    _simulate_ready_slots(env_items, rng.randint(1, 40), rng)
