"""Synthetic inputs: the heavy-hex lattice and the batched sweep's problem
definitions (angle grid with both ends, Z-strings around qubit 62)."""
import math

from paper_2506_13241_gb300 import workloads as W


def test_sweep_definition():
    wl = W.sweep_workload(32, 10, 1e-4)
    n, edges = wl["n"], wl["edges"]
    assert n == 127 and len(wl["problems"]) == 96
    thetas = sorted(set(wl["theta"]))
    assert len(thetas) == 32 and thetas[0] == 0.0 and abs(thetas[-1] - math.pi / 2) < 1e-15
    assert all(abs(thetas[k] - k * math.pi / 62) < 1e-15 for k in range(32))
    # problem p = 3 * i_theta + i_obs
    for p, terms in enumerate(wl["problems"]):
        assert wl["theta"][p] == thetas[p // 3]
        assert len(terms) == 1 and terms[0][1] == 1.0
    sites = [[q for q, ch in enumerate(wl["problems"][k][0][0]) if ch == "Z"] for k in range(3)]
    assert sites[0] == [62] and sites[1] == [61, 62, 63] and len(sites[2]) == 17
    # the weight-17 string is a ball around 62 in graph distance: every site
    # but 62 has a neighbour that is closer to 62
    _, dist = W.bfs_order(n, edges, 62)
    adj = W.adjacency(n, edges)
    for q in sites[2]:
        if q != 62:
            assert any(dist[r] < dist[q] and r in sites[2] for r in adj[q])
    assert max(dist[q] for q in sites[2]) <= min(dist[q] for q in range(n) if q not in sites[2])


def test_heavy_hex_shape():
    n, edges = W.heavy_hex_eagle()
    adj = W.adjacency(n, edges)
    assert n == 127 and len(edges) == 144
    assert max(len(a) for a in adj) == 3
    assert sorted(adj[62]) == [61, 63, 72]
