"""The named-barrier hand-off of the two-warp pipelined kernels, modelled on the
CPU: each warp's sequence of barrier operations as the kernels issue them, run
under many random interleavings.  A barrier instance completes when one warp
arrives and the other waits; the checks are that no interleaving deadlocks, that
a warp never arrives twice at a barrier before the other warp's matching wait
(which would complete a barrier instance with the wrong partner), and that every
arrival is matched.  This is the property that keeps the kernels from hanging.
"""
import random

import pytest


def adjoint_ops(Tn):
    """k_backward_pipe: tape b = t & 1; FULL(b) / EMPTY(b)."""
    producer, consumer = [], []
    for t in range(Tn - 1, -1, -1):
        b = t & 1
        if t < Tn - 2:
            producer.append(("sync", f"EMPTY{b}"))
        producer.append(("arrive", f"FULL{b}"))
        consumer.append(("sync", f"FULL{b}"))
        if t >= 2:
            consumer.append(("arrive", f"EMPTY{b}"))
    return producer, consumer


def rollout_ops(Tn, links):
    """k_rollout_pipe: LINK(l) per link, Q per step."""
    inertia, bias = [], []
    if Tn > 0:
        bias.append(("arrive", "Q"))
    for t in range(Tn):
        inertia.append(("sync", "Q"))
        for l in range(links - 1, -1, -1):
            inertia.append(("arrive", f"LINK{l}"))
        for l in range(links - 1, -1, -1):
            bias.append(("sync", f"LINK{l}"))
        if t + 1 < Tn:
            bias.append(("arrive", "Q"))
    return inertia, bias


def run(a, b, seed):
    rnd = random.Random(seed)
    ops = [a, b]
    pos = [0, 0]
    arrived, waited = {}, {}
    while pos[0] < len(a) or pos[1] < len(b):
        order = [w for w in (0, 1) if pos[w] < len(ops[w])]
        rnd.shuffle(order)
        for w in order:
            op, bar = ops[w][pos[w]]
            n_arr, n_wait = arrived.get(bar, 0), waited.get(bar, 0)
            if op == "arrive":
                assert n_arr - n_wait < 1, f"second arrival at {bar} before the matching wait"
                arrived[bar] = n_arr + 1
            else:
                if n_arr <= n_wait:
                    continue                       # blocked: the partner has not arrived yet
                waited[bar] = n_wait + 1
            pos[w] += 1
            break
        else:
            raise AssertionError("deadlock")
    assert arrived == waited


@pytest.mark.parametrize("Tn", list(range(0, 30)))
def test_adjoint_protocol(Tn):
    p, c = adjoint_ops(Tn)
    for seed in range(100):
        run(p, c, seed)


@pytest.mark.parametrize("links", [1, 2, 7, 14])
@pytest.mark.parametrize("Tn", [0, 1, 2, 3, 11])
def test_rollout_protocol(Tn, links):
    i, b = rollout_ops(Tn, links)
    for seed in range(100):
        run(i, b, seed)


def test_model_catches_a_broken_protocol():
    """A producer that waits on EMPTY one step too often deadlocks in the model."""
    p, c = adjoint_ops(5)
    p.insert(0, ("sync", "EMPTY0"))
    with pytest.raises(AssertionError):
        run(p, c, 0)
