"""Synthetic workloads for the kicked-Ising benchmarks of arXiv 2506.13241.

This module only builds inputs -- lattices, edge colourings, gate lists and
observables -- and holds none of the method's arithmetic.  Both the CUDA
library (through its Python binding) and the CPU oracle consume what it
returns, so it must not import either of them.

Gate tuples are ``(kind, q0, q1, theta)``: ``("rx", q, None, theta)`` is
exp(-i theta/2 sigma_x^q) and ``("rzz", i, j, theta)`` is
exp(-i theta/2 sigma_z^i sigma_z^j) (Eq. eq:u).  Qubits are 0-based.
"""
from __future__ import annotations

import math
from collections import deque

THETA_ZZ = -math.pi / 2  # fixed interaction angle (Sec. III)


# --------------------------------------------------------------------------
# Lattices
# --------------------------------------------------------------------------

def chain_edges(n: int):
    """Open chain 0-1-...-(n-1)."""
    return [(i, i + 1) for i in range(n - 1)]


def heavy_hex_eagle():
    """127-qubit heavy-hexagon lattice of the IBM Eagle layout (Fig. 1a).

    Seven rows of 14, 15, 15, 15, 15, 15, 14 qubits are numbered
    consecutively, each row followed (except the last) by a block of four
    bridge qubits.  Row r spans columns 0..14; the first row covers columns
    0..13 and the last columns 1..14.  The bridge block after row k joins
    (row k, column c) to (row k+1, column c) through one bridge qubit, with
    c in {0, 4, 8, 12} after even k and c in {2, 6, 10, 14} after odd k.
    Returns (n_qubits, edges) with edges sorted as (min, max) pairs.
    """
    row_len = [14, 15, 15, 15, 15, 15, 14]
    row_first_col = [0, 0, 0, 0, 0, 0, 1]
    pos = {}  # (row, col) -> qubit
    edges = []
    q = 0
    bridges_after = []
    for r, length in enumerate(row_len):
        start = q
        for k in range(length):
            pos[(r, row_first_col[r] + k)] = q
            q += 1
        for k in range(length - 1):
            edges.append((start + k, start + k + 1))
        if r < len(row_len) - 1:
            block = list(range(q, q + 4))
            q += 4
            bridges_after.append(block)
    for r, block in enumerate(bridges_after):
        cols = (0, 4, 8, 12) if r % 2 == 0 else (2, 6, 10, 14)
        for b, c in zip(block, cols):
            edges.append((pos[(r, c)], b))
            edges.append((b, pos[(r + 1, c)]))
    edges = sorted((min(a, b), max(a, b)) for a, b in edges)
    return q, edges


def adjacency(n: int, edges):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    for lst in adj:
        lst.sort()
    return adj


def bfs_order(n: int, edges, source: int):
    """Qubits ordered by graph distance from ``source`` (ties by index),
    with their distances."""
    adj = adjacency(n, edges)
    dist = [-1] * n
    dist[source] = 0
    dq = deque([source])
    while dq:
        u = dq.popleft()
        for v in adj[u]:
            if dist[v] < 0:
                dist[v] = dist[u] + 1
                dq.append(v)
    order = sorted((d, q) for q, d in enumerate(dist) if d >= 0)
    return [q for _, q in order], dist


def edge_colouring(n: int, edges):
    """Proper edge colouring of a bipartite graph with max-degree colours
    (Koenig's theorem), by alternating-path recolouring.  Returns a list of
    colour classes, each a list of disjoint edges in input order."""
    adj = adjacency(n, edges)
    ncol = max((len(a) for a in adj), default=0)
    # colour_at[v][c] = neighbour joined to v by an edge of colour c
    colour_at = [dict() for _ in range(n)]

    def free(v):
        for c in range(ncol):
            if c not in colour_at[v]:
                return c
        raise AssertionError("no free colour")

    for (u, v) in edges:
        a = free(u)
        b = free(v)
        if a != b and a in colour_at[v]:
            # flip the a/b alternating path starting at v
            path = []
            w, c = v, a
            while c in colour_at[w]:
                nxt = colour_at[w][c]
                path.append((w, nxt, c))
                w = nxt
                c = b if c == a else a
            for (x, y, c) in path:
                del colour_at[x][c]
                del colour_at[y][c]
            for (x, y, c) in path:
                c2 = b if c == a else a
                colour_at[x][c2] = y
                colour_at[y][c2] = x
        colour_at[u][a] = v
        colour_at[v][a] = u
    classes = [[] for _ in range(ncol)]
    for (u, v) in edges:
        for c, w in colour_at[u].items():
            if w == v:
                classes[c].append((u, v))
                break
    return classes


# --------------------------------------------------------------------------
# Kicked-Ising circuit (Eq. eq:u)
# --------------------------------------------------------------------------

def kicked_ising_layers(n: int, edges, theta_x: float, theta_zz: float = THETA_ZZ):
    """One Trotter step in Heisenberg order: the U_zz layer (all edges,
    colour class by colour class) and then the U_x layer (qubits ascending).

    For U = U_zz U_x the conjugation U^dagger O U acts with U_zz first and
    U_x second, so an observable is pushed through these two lists in order.
    """
    classes = edge_colouring(n, edges)
    zz = [("rzz", a, b, theta_zz) for cls in classes for (a, b) in cls]
    xx = [("rx", q, None, theta_x) for q in range(n)]
    return [zz, xx]


def z_label(n: int, sites) -> str:
    s = ["I"] * n
    for q in sites:
        s[q] = "Z"
    return "".join(s)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

def workload(name: str):
    """Named workloads: returns a dict with n, edges, layers, observable,
    steps, delta.  The observable is a list of (label, coefficient)."""
    if name == "chain12":
        n = 12
        edges = chain_edges(n)
        return dict(name=name, n=n, edges=edges,
                    layers=kicked_ising_layers(n, edges, math.pi / 4),
                    observable=[(z_label(n, [6]), 1.0)], steps=5, delta=0.0,
                    theta_x=math.pi / 4)
    if name.startswith("heavyhex"):
        n, edges = heavy_hex_eagle()
        # heavyhex[_theta=<rad>][_t=<steps>][_delta=<d>]
        theta, steps, delta = math.pi / 4, 5, 1e-4
        for part in name.split("_")[1:]:
            k, v = part.split("=")
            if k == "theta":
                theta = float(v)
            elif k == "t":
                steps = int(v)
            elif k == "delta":
                delta = float(v)
        return dict(name=name, n=n, edges=edges,
                    layers=kicked_ising_layers(n, edges, theta),
                    observable=[(z_label(n, [62]), 1.0)], steps=steps, delta=delta,
                    theta_x=theta)
    raise KeyError(name)


def weighted_z_observable(n: int, edges, centre: int, weight: int):
    """Z-string on the ``weight`` qubits nearest ``centre`` by graph distance
    (ties broken by qubit index)."""
    order, _ = bfs_order(n, edges, centre)
    return z_label(n, order[:weight])


def sweep_workload(n_theta: int = 32, steps: int = 10, delta: float = 1e-4, weights=(1, 3, 17)):
    """Batched theta_h x observable sweep on the heavy-hex: n_theta angles
    uniform in [0, pi/2] (both ends included) times Z-strings of the given
    weights around qubit 62.  Problem p = i_theta * len(weights) + i_obs.
    Returns n, edges, the layer template (angles of the X layer are
    replaced per problem), the observables per problem, and theta[p]."""
    n, edges = heavy_hex_eagle()
    thetas = [0.5 * math.pi * k / (n_theta - 1) for k in range(n_theta)] if n_theta > 1 else [math.pi / 4]
    obs = [weighted_z_observable(n, edges, 62, w) for w in weights]
    problems, theta_p = [], []
    for th in thetas:
        for lab in obs:
            problems.append([(lab, 1.0)])
            theta_p.append(th)
    return dict(name="sweep_%dx%d_t=%d_delta=%g" % (n_theta, len(weights), steps, delta), n=n, edges=edges,
                layers=kicked_ising_layers(n, edges, math.pi / 4), problems=problems, theta=theta_p,
                steps=steps, delta=delta, weights=list(weights))
