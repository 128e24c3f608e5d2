"""Placement of the batched form's ensemble members on the GPUs of a job.

The members of an ensemble are independent problems, so the ensemble
shards with no exchange on the data path: each GPU advances its own members
and only statistics are gathered.  A member's work per step grows with its
grid size N and the square of its rank cap (the roundings factor N x cap-class
cores, O(N cap^2) each), so members are placed by longest processing time
first on cost N * cap^2: the costliest member not yet placed goes to the
GPU with the least load.  Greedy list scheduling keeps every load within the
mean load plus one member's cost (Graham's bound), and LPT within 4/3 of the
optimal makespan.
"""


def member_cost(n, cap):
    """Work estimate of one ensemble member per step: N * cap^2."""
    return float(n) * float(cap) * float(cap)


def partition(costs, world):
    """Indices of the members placed on each of `world` GPUs (each list
    ascending), by longest processing time first; ties go to the lower
    member index and the lower GPU."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    shards = [[] for _ in range(world)]
    for i in order:
        g = min(range(world), key=lambda r: (loads[r], r))
        shards[g].append(i)
        loads[g] += costs[i]
    return [sorted(s) for s in shards]


def shard_loads(costs, shards):
    return [sum(costs[i] for i in s) for s in shards]
