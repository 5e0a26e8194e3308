"""Test-only helpers: small independent reference computations (dense linear
algebra, graph components) used to pin the oracle, plus the mapping between
the oracle's edge numbering and the library's device layout."""
from __future__ import annotations

import numpy as np


def dense(A):
    return A.toarray() if hasattr(A, "toarray") else np.asarray(A)


def conductor_node_components(disc):
    """Connected components of the graph whose vertices are nodes touched by a
    conducting edge and whose arcs are the conducting edges (plain BFS)."""
    G = disc.G.tocsr()
    adj = {}
    for e in disc.c_idx:
        cols = G.indices[G.indptr[e]:G.indptr[e + 1]]
        a, b = int(cols[0]), int(cols[1])
        adj.setdefault(a, set()).add(b)
        adj.setdefault(b, set()).add(a)
    seen, comps = set(), []
    for s in adj:
        if s in seen:
            continue
        comp, stack = [], [s]
        seen.add(s)
        while stack:
            u = stack.pop()
            comp.append(u)
            for v in adj[u]:
                if v not in seen:
                    seen.add(v)
                    stack.append(v)
        comps.append(comp)
    return comps


def interior_nodes(N):
    r = np.arange(1, N)
    k, j, i = np.meshgrid(r, r, r, indexing="ij")
    return (i + (N + 1) * (j + (N + 1) * k)).ravel()


def kn_null_vectors(disc):
    """Null vectors of K_n predicted by the topology: gradients of the hat
    function of every interior node touched by no conducting edge, and of the
    indicator of every connected conductor."""
    comps = conductor_node_components(disc)
    cnodes = set(u for c in comps for u in c)
    vecs = []
    G = disc.G
    for nd in interior_nodes(disc.N):
        if nd in cnodes:
            continue
        phi = np.zeros(disc.grid.n_nodes)
        phi[nd] = 1.0
        vecs.append((G @ phi)[disc.n_idx])
    for c in comps:
        phi = np.zeros(disc.grid.n_nodes)
        phi[c] = 1.0
        vecs.append((G @ phi)[disc.n_idx])
    return vecs, comps


# --- oracle numbering <-> device layout -------------------------------------
def layout_index_of_oracle_edges(N):
    """For every oracle edge, its index in the device layout (3 N^3 doubles,
    component-major, x fastest, storage index range [0, N) per axis), or -1
    where the edge is not stored (Dirichlet edges at node index N)."""
    out = []
    N1 = N + 1
    for comp, shape in ((0, (N, N1, N1)), (1, (N1, N, N1)), (2, (N1, N1, N))):
        k, j, i = np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]), indexing="ij")
        i, j, k = i.ravel(), j.ravel(), k.ravel()
        ok = (i < N) & (j < N) & (k < N)
        idx = np.where(ok, comp * N ** 3 + i + N * (j + N * k), -1)
        out.append(idx)
    return np.concatenate(out)


def oracle_to_layout(N, v_oracle):
    m = layout_index_of_oracle_edges(N)
    out = np.zeros(3 * N ** 3)
    ok = m >= 0
    out[m[ok]] = v_oracle[ok]
    return out


def layout_to_oracle(N, v_layout):
    m = layout_index_of_oracle_edges(N)
    out = np.zeros(m.size)
    ok = m >= 0
    out[ok] = v_layout[m[ok]]
    return out


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
