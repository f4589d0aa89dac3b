"""Seeded synthetic inputs: typed HINs and metapath query workloads.

This module only draws random numbers. It builds no CSR, evaluates no constraint
and multiplies nothing, so the CPU oracle and the CUDA path can both take their
inputs from it without sharing any of the method's arithmetic.

A HIN is returned as a plain dict::

    {"types":     {"P": 2000, "A": 1500, ...},          # node type -> node count
     "relations": [("P", "A", src_u32, dst_u32), ...],  # one direction per schema edge
     "props":     {("P", "year"): int32 array, ...}}

Every schema edge is bidirectional (Sec. 2, Def. 1 and the HIN tables of Sec. 4.1.1):
the generator lists each relation once, as drawn, and each consumer builds both
directions from it. Edge lists may contain repeated (src, dst) pairs when asked for
(``dup_frac``); the 0/1 adjacency of Def. 1 collapses them.

A query is a plain dict::

    {"types": ["A", "P", "T", "P", "A"],
     "constraints": [{"pos": 1, "prop": "year", "op": "range", "lo": 2010, "hi": 2020},
                     {"pos": 0, "prop": None,   "op": "in",    "set": uint32 array}]}

``prop=None`` constrains the node id itself. ``op`` is ``range`` (lo <= v <= hi),
``eq`` (v == lo) or ``in`` (v in set). Constraint semantics follow Def. 3.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "stream", "zipf_sampler", "uniform_sampler", "draw_links",
    "scholarly_hin", "news_hin", "tiny_hin", "config1_hin", "config2_hin", "config4_hin",
    "config1_query", "config2_queries", "batched_queries", "long_queries",
    "serving_stream", "random_queries", "schema_walk",
]


def stream(seed: int, *tag: int) -> np.random.Generator:
    """Independent PCG64 stream for (seed, tag...)."""
    return np.random.default_rng(np.random.SeedSequence([int(seed)] + [int(t) for t in tag]))


def zipf_sampler(n: int, s: float, perm_rng: np.random.Generator):
    """Zipf(s) over n ranks by inverse CDF; rank r maps to node id perm[r], so hubs
    are scattered over the id range instead of sitting at low ids."""
    w = np.arange(1, n + 1, dtype=np.float64) ** (-float(s))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    perm = perm_rng.permutation(n).astype(np.uint32)

    def sample(rng: np.random.Generator, size: int) -> np.ndarray:
        r = np.searchsorted(cdf, rng.random(size), side="right")
        np.minimum(r, n - 1, out=r)
        return perm[r]

    return sample


def uniform_sampler(n: int):
    def sample(rng: np.random.Generator, size: int) -> np.ndarray:
        return rng.integers(0, n, size=size, dtype=np.int64).astype(np.uint32)

    return sample


def draw_links(rng, n_src: int, counts: np.ndarray, n_dst: int, sample):
    """Per source node, draw counts[i] distinct destinations (clipped to n_dst) with
    `sample`, re-drawing repeats until each source's list has no duplicate."""
    counts = np.minimum(np.asarray(counts, dtype=np.int64), n_dst)
    src = np.repeat(np.arange(n_src, dtype=np.uint32), counts)
    dst = sample(rng, src.size)
    active = np.ones(n_src, dtype=bool)
    for _ in range(100000):
        sel = np.nonzero(active[src])[0]
        if sel.size == 0:
            break
        key = src[sel].astype(np.int64) * n_dst + dst[sel]
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(ks.size, dtype=bool)
        dup[1:] = ks[1:] == ks[:-1]
        if not dup.any():
            break
        redo = sel[order[dup]]
        dst[redo] = sample(rng, redo.size)
        active[:] = False
        active[src[redo]] = True
    return src, dst


def _with_dups(rng, src, dst, dup_frac):
    if dup_frac <= 0 or src.size == 0:
        return src, dst
    k = max(1, int(src.size * dup_frac))
    pick = rng.integers(0, src.size, size=k)
    s = np.concatenate([src, src[pick]])
    d = np.concatenate([dst, dst[pick]])
    o = rng.permutation(s.size)
    return s[o], d[o]


def scholarly_hin(n_p, n_a, n_v, n_t, seed, *, s_author=1.2, s_topic=1.0,
                  mean_authors=3.0, mean_topics=4.0, year=True, dup_frac=0.0):
    """Scholarly-shaped HIN (papers P, authors A, venues V, topics T).

    Each paper has 1+Poisson(mean_authors-1) distinct Zipf(s_author) authors, exactly
    one uniform venue and 1+Poisson(mean_topics-1) distinct Zipf(s_topic) topics.
    With `year`, P carries an int32 'year' uniform on 1980..2021.
    """
    g = stream(seed, 0)
    c_a = 1 + g.poisson(mean_authors - 1.0, n_p)
    c_t = 1 + g.poisson(mean_topics - 1.0, n_p)
    pa = draw_links(stream(seed, 1), n_p, c_a, n_a, zipf_sampler(n_a, s_author, stream(seed, 11)))
    pv = draw_links(stream(seed, 2), n_p, np.ones(n_p, np.int64), n_v, uniform_sampler(n_v))
    pt = draw_links(stream(seed, 3), n_p, c_t, n_t, zipf_sampler(n_t, s_topic, stream(seed, 13)))
    rels = []
    for k, (a, b, (s, d)) in enumerate((("P", "A", pa), ("P", "V", pv), ("P", "T", pt))):
        s, d = _with_dups(stream(seed, 20 + k), s, d, dup_frac)
        rels.append((a, b, s, d))
    props = {}
    if year:
        props[("P", "year")] = stream(seed, 4).integers(1980, 2022, n_p, dtype=np.int64).astype(np.int32)
    return {"types": {"P": n_p, "A": n_a, "V": n_v, "T": n_t}, "relations": rels, "props": props}


CONFIG1_COUNTS = {"P": 2000, "A": 1500, "V": 50, "T": 200}


def config1_hin(seed: int = 1):
    """2,000 papers, 1,500 authors, 50 venues, 200 topics."""
    c = CONFIG1_COUNTS
    return scholarly_hin(c["P"], c["A"], c["V"], c["T"], seed)


def config2_hin(seed: int = 2, scale: float = 1.0):
    """5 M papers, 4 M authors, 5 k venues, 50 k topics (scale shrinks every count)."""
    f = lambda n: max(2, int(round(n * scale)))
    return scholarly_hin(f(5_000_000), f(4_000_000), f(5_000), f(50_000), seed)


def news_hin(n_art, n_per, n_org, n_loc, n_thm, seed, *, s=1.3, means=(5, 3, 2, 8), days=730,
             dup_frac=0.0):
    """News-shaped HIN: articles (R) linked to persons (E), organisations (O),
    locations (L) and themes (H); each article draws 1+Poisson(mean-1) distinct
    Zipf(s) targets per type and carries an int32 'date' uniform on 0..days-1."""
    g = stream(seed, 0)
    rels = []
    for k, (t, n) in enumerate((("E", n_per), ("O", n_org), ("L", n_loc), ("H", n_thm))):
        cnt = 1 + g.poisson(means[k] - 1.0, n_art)
        s_, d_ = draw_links(stream(seed, 1 + k), n_art, cnt, n,
                            zipf_sampler(n, s, stream(seed, 11 + k)))
        s_, d_ = _with_dups(stream(seed, 20 + k), s_, d_, dup_frac)
        rels.append(("R", t, s_, d_))
    props = {("R", "date"): stream(seed, 9).integers(0, days, n_art, dtype=np.int64).astype(np.int32)}
    return {"types": {"R": n_art, "E": n_per, "O": n_org, "L": n_loc, "H": n_thm},
            "relations": rels, "props": props}


def config4_hin(seed: int = 4, scale: float = 1.0):
    f = lambda n: max(2, int(round(n * scale)))
    return news_hin(f(10_000_000), f(2_000_000), f(1_000_000), f(200_000), f(20_000), seed)


def tiny_hin(seed: int, max_nodes: int = 12, dup_frac: float = 0.2):
    """A few-dozen-node scholarly HIN for brute-force enumeration, with repeated
    edges, isolated nodes and a 'year' property on every type."""
    g = stream(seed, 100)
    n = {t: int(g.integers(2, max_nodes + 1)) for t in ("P", "A", "V", "T")}
    h = scholarly_hin(n["P"], n["A"], n["V"], n["T"], seed + 1000, mean_authors=2.0,
                      mean_topics=2.0, dup_frac=dup_frac)
    for t in ("A", "V", "T"):
        h["props"][(t, "year")] = stream(seed, 200 + ord(t)).integers(
            1980, 2022, n[t], dtype=np.int64).astype(np.int32)
    return h


# ---------------------------------------------------------------- workloads

SCHOLARLY_STAR = {"P": ("A", "V", "T"), "A": ("P",), "V": ("P",), "T": ("P",)}
NEWS_STAR = {"R": ("E", "O", "L", "H"), "E": ("R",), "O": ("R",), "L": ("R",), "H": ("R",)}


def schema_walk(rng, star, length, start=None):
    """A random walk of `length` node types on a star schema."""
    hub = [t for t, nb in star.items() if len(nb) > 1][0]
    leaves = list(star[hub])
    if start is None:
        start = leaves[int(rng.integers(len(leaves)))] if rng.random() < 0.75 else hub
    walk = [start]
    while len(walk) < length:
        cur = walk[-1]
        walk.append(hub if cur != hub else leaves[int(rng.integers(len(leaves)))])
    return walk


def config1_query():
    """APTPA, unconstrained."""
    return {"types": list("APTPA"), "constraints": []}


def _year_on_every(types, t, lo, hi, prop="year"):
    return [{"pos": i, "prop": prop, "op": "range", "lo": lo, "hi": hi}
            for i, x in enumerate(types) if x == t]


def config2_queries(hin, seed: int = 2, n_anchor_a: int = 256, n_anchor_t: int = 16,
                    n_anchor_v: int = 16):
    """Twenty constrained queries: four each of APA, APVPA, APTPA, TPAPT and VPTPV,
    with year in [2010, 2020] on every P position. APVPA and APTPA are anchored on a
    seeded set of n_anchor_a authors, TPAPT on n_anchor_t topics and VPTPV on
    n_anchor_v venues (a first-node id-set constraint: the 'entity of interest' of the
    session workloads, Sec. 4.1.2), drawn uniformly among nodes with at least one edge.
    APA runs unanchored."""
    g = stream(seed, 500)
    deg_a = np.zeros(hin["types"]["A"], np.int64)
    deg_t = np.zeros(hin["types"]["T"], np.int64)
    deg_v = np.zeros(hin["types"]["V"], np.int64)
    for a, b, s, d in hin["relations"]:
        if (a, b) == ("P", "V"):
            deg_v += np.bincount(d, minlength=deg_v.size)
        if (a, b) == ("P", "A"):
            deg_a += np.bincount(d, minlength=deg_a.size)
        if (a, b) == ("P", "T"):
            deg_t += np.bincount(d, minlength=deg_t.size)
    live_a = np.nonzero(deg_a)[0]
    live_t = np.nonzero(deg_t)[0]
    live_v = np.nonzero(deg_v)[0]
    out = []
    for rep in range(4):
        for name in ("APA", "APVPA", "APTPA", "TPAPT", "VPTPV"):
            types = list(name)
            cons = _year_on_every(types, "P", 2010, 2020)
            if name in ("APVPA", "APTPA"):
                ids = np.sort(g.choice(live_a, size=min(n_anchor_a, live_a.size), replace=False))
                cons.append({"pos": 0, "prop": None, "op": "in", "set": ids.astype(np.uint32)})
            elif name == "TPAPT":
                ids = np.sort(g.choice(live_t, size=min(n_anchor_t, live_t.size), replace=False))
                cons.append({"pos": 0, "prop": None, "op": "in", "set": ids.astype(np.uint32)})
            elif name == "VPTPV":
                ids = np.sort(g.choice(live_v, size=min(n_anchor_v, live_v.size), replace=False))
                cons.append({"pos": 0, "prop": None, "op": "in", "set": ids.astype(np.uint32)})
            out.append({"types": types, "constraints": cons})
    return out


YEAR_RANGES = ((2000, 2021), (1990, 2010), (2010, 2020), (1980, 2000))


def batched_queries(seed: int = 3, n: int = 256, pool: int = 40, s: float = 1.1,
                    lengths=(3, 7), star=SCHOLARLY_STAR, prop=("P", "year"),
                    ranges=YEAR_RANGES, anchor_p: float = 0.0, n_anchors: int = 16,
                    counts=None):
    """n queries drawn Zipf(s) from a seeded pool of templates; a template is a
    schema walk of length in [lengths] plus, with probability 1/2, one year range
    (from a small set) on every position of the constrained type. With probability
    anchor_p a drawn query also fixes its first node to one of n_anchors seeded
    entities of that type (an id-equality constraint: the entity of interest of a
    session, Sec. 4.2); sub-chains away from the first position stay shared. counts
    gives the node count of each type (default: the 2,000-paper scholarly HIN)."""
    g = stream(seed, 600)
    templates = []
    for _ in range(pool):
        L = int(g.integers(lengths[0], lengths[1] + 1))
        types = schema_walk(g, star, L)
        cons = []
        if g.random() < 0.5:
            lo, hi = ranges[int(g.integers(len(ranges)))]
            cons = _year_on_every(types, prop[0], lo, hi, prop[1])
        templates.append({"types": types, "constraints": cons})
    pick = zipf_sampler(pool, s, stream(seed, 601))(stream(seed, 602), n)
    out = [templates[int(i)] for i in pick]
    if anchor_p > 0.0:
        ga = stream(seed, 603)
        counts = dict(counts or CONFIG1_COUNTS)
        anchors = {t: ga.choice(c, size=min(n_anchors, c), replace=False)
                   for t, c in counts.items()}
        for qi, q in enumerate(out):
            if ga.random() < anchor_p:
                t = q["types"][0]
                a = int(anchors[t][int(ga.integers(len(anchors[t])))])
                out[qi] = {"types": q["types"], "constraints": list(q["constraints"]) +
                           [{"pos": 0, "prop": None, "op": "eq", "lo": a}]}
    return out


def long_queries(seed: int = 5, n: int = 64):
    """n metapaths of length 7..9 on the scholarly schema that pass through V and T,
    e.g. APVPTPVPA."""
    g = stream(seed, 700)
    out = []
    while len(out) < n:
        L = int(g.integers(7, 10))
        types = schema_walk(g, SCHOLARLY_STAR, L)
        if "V" in types and "T" in types:
            out.append({"types": types, "constraints": []})
    return out


def random_queries(hin, seed, n, lengths=(2, 7), star=SCHOLARLY_STAR, p_cons=0.5):
    """Random constrained queries for parity tests: schema walks with a random mix of
    range constraints on any property the HIN has, id equality and id-set
    constraints at random positions."""
    g = stream(seed, 800)
    out = []
    for _ in range(n):
        L = int(g.integers(lengths[0], lengths[1] + 1))
        types = schema_walk(g, star, L)
        cons = []
        for i, t in enumerate(types):
            if g.random() >= p_cons:
                continue
            kind = int(g.integers(3))
            nt = hin["types"][t]
            if kind == 0 and (t, "year") in hin["props"]:
                lo = int(g.integers(1980, 2022))
                hi = int(g.integers(lo, 2023))
                cons.append({"pos": i, "prop": "year", "op": "range", "lo": lo, "hi": hi})
            elif kind == 1:
                cons.append({"pos": i, "prop": None, "op": "eq", "lo": int(g.integers(nt))})
            else:
                k = int(g.integers(1, max(2, nt // 2) + 1))
                ids = np.unique(g.integers(0, nt, size=k)).astype(np.uint32)
                cons.append({"pos": i, "prop": None, "op": "in", "set": ids})
        out.append({"types": types, "constraints": cons})
    return out


def serving_stream(hin, seed: int = 4, n: int = 100_000, n_templates: int = 500, s: float = 1.0,
                   restart_p: float = 0.08, rate_qps: float = 1000.0, star=NEWS_STAR,
                   hub="R", date_prop="date", days=730):
    """Session workload (Sec. 4.1.2): each session fixes an anchor entity (first-node
    equality) and a date window of U{1..30} days; with probability restart_p a new
    session starts, else the next query reuses the session's anchor and window with a
    new template drawn Zipf(s) over n_templates schema walks of length 3..7 that start
    at a non-hub type. Arrival times are a Poisson process of rate rate_qps.
    Returns (queries, arrival_seconds)."""
    g = stream(seed, 900)
    templates = []
    while len(templates) < n_templates:
        L = int(g.integers(3, 8))
        w = schema_walk(g, star, L)
        if w[0] != hub:
            templates.append(w)
    pick = zipf_sampler(n_templates, s, stream(seed, 901))
    tid = pick(stream(seed, 902), n)
    queries = []
    anchor = None
    for i in range(n):
        types = templates[int(tid[i])]
        if anchor is None or g.random() < restart_p:
            w = int(g.integers(1, 31))
            lo = int(g.integers(0, days - w + 1))
            anchor = {"win": (lo, lo + w - 1), "ids": {}}
        t0 = types[0]
        if t0 not in anchor["ids"]:
            anchor["ids"][t0] = int(g.integers(hin["types"][t0]))
        cons = [{"pos": 0, "prop": None, "op": "eq", "lo": anchor["ids"][t0]}]
        cons += _year_on_every(types, hub, anchor["win"][0], anchor["win"][1], date_prop)
        queries.append({"types": list(types), "constraints": cons})
    gaps = g.exponential(1.0 / rate_qps, n)
    return queries, np.cumsum(gaps)
