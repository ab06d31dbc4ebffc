"""Test-side splitmix64 (Steele, Lea, Flood 2014) and priority comparisons, written
independently of the oracle's C code for brute-force cross-checks."""
import numpy as np

M64 = (1 << 64) - 1


def splitmix64(seed, counter):
    z = (seed + (counter + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def priorities(n, seed):
    """key(v) = (hash, -v): larger key = higher priority."""
    return [(splitmix64(seed, v), -v) for v in range(n)]


def adjacency(rowptr, col):
    n = len(rowptr) - 1
    return [set(int(c) for c in col[rowptr[i]:rowptr[i + 1]] if c != i) for i in range(n)]


def mis2_rounds(adj, seed):
    """Synchronous rounds: an undecided node becomes a root when its priority beats every
    undecided node within distance 2; nodes within distance 2 of new roots are decided."""
    n = len(adj)
    key = priorities(n, seed)
    n2 = []
    for v in range(n):
        s = set(adj[v])
        for w in adj[v]:
            s |= adj[w]
        s.discard(v)
        n2.append(s)
    undecided = set(range(n))
    roots = set()
    while undecided:
        new = [v for v in undecided if all(key[v] > key[w] for w in n2[v] if w in undecided)]
        assert new
        for v in new:
            roots.add(v)
        for v in new:
            undecided.discard(v)
            undecided -= n2[v]
    return roots


def jp_colour(adj, seed):
    n = len(adj)
    key = priorities(n, seed)
    colour = [-1] * n
    left = set(range(n))
    while left:
        ready = [v for v in left if all(key[v] > key[w] for w in adj[v] if colour[w] < 0)]
        assign = {}
        for v in ready:
            used = {colour[w] for w in adj[v] if colour[w] >= 0}
            c = 0
            while c in used:
                c += 1
            assign[v] = c
        for v, c in assign.items():
            colour[v] = c
            left.discard(v)
    return np.array(colour)
