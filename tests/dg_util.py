"""Checks of a discrete gradient that hold by Forman's definition or by
topology, independent of how the gradient was built (Section 5.1,
DiscreteGradient), and conversion of the consumer's id arrays to vertex
tuples."""
from itertools import combinations

import numpy as np


def all_simplices(rows):
    """Every simplex of a pure tetrahedral complex, as sorted tuples, by dimension."""
    S = [set(), set(), set(), set()]
    for r in rows:
        r = tuple(sorted(int(x) for x in r))
        for d in range(4):
            S[d].update(combinations(r, d + 1))
    return S


def pairs_from_ids(g, E, F, rows):
    """(set of (face, coface) tuples, set of critical tuples) from the
    consumer's v_up / e_up / f_up arrays, checking that the down arrays
    mirror the up arrays."""
    E = [tuple(int(x) for x in e) for e in E]
    F = [tuple(int(x) for x in f) for f in F]
    T = [tuple(int(x) for x in r) for r in rows]
    pairs = set()
    for v, e in enumerate(g["v_up"]):
        if e >= 0:
            assert g["e_down"][e] == v
            pairs.add(((v,), E[e]))
    for e, f in enumerate(g["e_up"]):
        if f >= 0:
            assert g["f_down"][f] == e
            pairs.add((E[e], F[f]))
    for f, t in enumerate(g["f_up"]):
        if t >= 0:
            assert g["t_down"][t] == f
            pairs.add((F[f], T[t]))
    down = sum(int((np.asarray(g[k]) >= 0).sum()) for k in ("e_down", "f_down", "t_down"))
    assert down == len(pairs)
    crit = set()
    for v in range(len(g["v_up"])):
        if g["v_up"][v] < 0:
            crit.add((v,))
    for e in range(len(E)):
        if g["e_down"][e] < 0 and g["e_up"][e] < 0:
            crit.add(E[e])
    for f in range(len(F)):
        if g["f_down"][f] < 0 and g["f_up"][f] < 0:
            crit.add(F[f])
    for t in range(len(T)):
        if g["t_down"][t] < 0:
            crit.add(T[t])
    return pairs, crit


def violations(rows, field, inid, pairs, critical):
    """Problems with a claimed gradient (empty list: none):
    * every simplex is critical or in exactly one pair;
    * a pair is a face and a coface one dimension higher;
    * both lie in the same lower star (share their highest vertex);
    * no closed V-path (the gradient is acyclic);
    * the critical cells' alternating count is the Euler characteristic."""
    out = []
    S = all_simplices(rows)
    key = lambda v: (float(field[v]), int(inid[v]))
    top = lambda s: max(s, key=key)
    seen = {}
    for a, b in pairs:
        a, b = tuple(a), tuple(b)
        for s in (a, b):
            seen[s] = seen.get(s, 0) + 1
        if len(b) != len(a) + 1 or not set(a) < set(b):
            out.append(("not a facet pair", a, b))
        elif top(a) != top(b):
            out.append(("pair across lower stars", a, b))
        if b not in S[len(b) - 1]:
            out.append(("not a simplex", b))
    for c in critical:
        seen[tuple(c)] = seen.get(tuple(c), 0) + 1
    for d in range(4):
        for s in S[d]:
            if seen.get(s, 0) != 1:
                out.append(("classified %d times" % seen.get(s, 0), s))
    chi = len(S[0]) - len(S[1]) + len(S[2]) - len(S[3])
    cc = [0, 0, 0, 0]
    for c in critical:
        cc[len(c) - 1] += 1
    if cc[0] - cc[1] + cc[2] - cc[3] != chi:
        out.append(("Euler characteristic", cc, chi))
    # V-paths: sigma -> tau (paired), tau -> sigma' (other facets of tau)
    partner = {}
    for a, b in pairs:
        partner[tuple(a)] = tuple(b)
    for k in range(3):
        nodes = list(S[k]) + list(S[k + 1])
        succ = {s: [] for s in nodes}
        indeg = {s: 0 for s in nodes}
        for s in S[k]:
            t = partner.get(s)
            if t is not None and len(t) == k + 2:
                succ[s].append(t)
                indeg[t] += 1
        for t in S[k + 1]:
            for i in range(len(t)):
                f = t[:i] + t[i + 1:]
                if partner.get(f) == t:
                    continue
                succ[t].append(f)
                indeg[f] += 1
        queue = [s for s in nodes if indeg[s] == 0]
        n = 0
        while queue:
            s = queue.pop()
            n += 1
            for x in succ[s]:
                indeg[x] -= 1
                if indeg[x] == 0:
                    queue.append(x)
        if n != len(nodes):
            out.append(("closed V-path", k))
    return out


def lower_link_prediction(rows, field, inid):
    """Per vertex, the critical cells of each dimension that a lower star
    whose gradient is optimal must hold: the reduced Betti numbers of the
    lower link LL (the link simplices with every vertex below v), shifted up
    one dimension.  On a 3-manifold mesh the link is a 2-sphere or a disk,
    so LL has no 2-cycle unless it is the whole closed link; b1 follows from
    the Euler characteristic of LL."""
    nv = int(np.max(rows)) + 1 if len(rows) else 0
    key = lambda v: (float(field[v]), int(inid[v]))
    star = [[] for _ in range(nv)]
    for r in rows:
        for x in r:
            star[int(x)].append([int(y) for y in r if int(y) != int(x)])
    pred = {}
    for v in range(nv):
        tris = [tuple(sorted(o)) for o in star[v]]
        edges = {e for t in tris for e in combinations(t, 2)}
        verts = {x for t in tris for x in t}
        ecount = {}
        for t in tris:
            for e in combinations(t, 2):
                ecount[e] = ecount.get(e, 0) + 1
        closed = all(c == 2 for c in ecount.values())
        low = lambda x: key(x) < key(v)
        Lv = [x for x in verts if low(x)]
        Le = [e for e in edges if low(e[0]) and low(e[1])]
        Lt = [t for t in tris if all(low(x) for x in t)]
        if not Lv:
            pred[v] = (1, 0, 0, 0)
            continue
        parent = {x: x for x in Lv}

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x
        for a, b in Le:
            parent[find(a)] = find(b)
        b0 = len({find(x) for x in Lv})
        b2 = 1 if closed and len(Lt) == len(tris) else 0
        chi = len(Lv) - len(Le) + len(Lt)
        b1 = b0 + b2 - chi
        pred[v] = (0, b0 - 1, b1, b2)
    return pred


def critical_by_vertex(critical, field, inid, nv):
    key = lambda v: (float(field[v]), int(inid[v]))
    got = {v: [0, 0, 0, 0] for v in range(nv)}
    for c in critical:
        got[max(c, key=key)][len(c) - 1] += 1
    return {v: tuple(x) for v, x in got.items()}
