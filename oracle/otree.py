"""Overlap Tree for the oracle (test infrastructure only).

Sec. 3.3: a generalised suffix tree over the metapaths of the workload (one symbol per
node type), built by inserting, for every query, the whole metapath and each of its
proper suffixes (Sec. 3.3.2). A query-specific terminator ends every inserted string,
so each suffix ends at its own leaf (footnote in Sec. 3.3.1). Inserting a suffix walks
from the root along the longest matching path; a match that stops inside an edge
splits the edge with a new internal node; the suffix's remainder hangs from the last
node as a new leaf. Every node on the walked path counts one more occurrence, so a
node's frequency f is the number of leaves below it: the number of occurrences of its
string among all inserted queries (leaves have f = 1).

Sec. 3.3.4: every node carries a constraints index, a map from the canonical string of
the constraints on its positions to the entry (f, p, c, rho); the walk updates the entry
of the constraints the inserted suffix carries on those positions.

Sec. 3.3.3: with lambda = sum |m_i| leaves, a tree whose internal nodes all have at
least two children has at most 2*lambda - 1 nodes.
"""
from __future__ import annotations


class Entry:
    """(f, p, c, rho) of one sub-metapath under one constraint key."""

    __slots__ = ("f", "p", "c", "rho")

    def __init__(self):
        self.f = 0
        self.p = None     # cache entry key, or None
        self.c = None     # recorded cost of computing it
        self.rho = None   # recorded nnz of its result


class Node:
    __slots__ = ("parent", "label", "children", "f", "cidx", "depth")

    def __init__(self, parent, label, depth):
        self.parent = parent
        self.label = tuple(label)   # symbols on the edge into this node
        self.children = {}          # first symbol of the child's label -> child
        self.f = 0
        self.cidx = {}              # constraint key -> Entry
        self.depth = depth          # length of the node's string (terminator included)

    def is_leaf(self):
        return not self.children

    def string(self):
        parts = []
        n = self
        while n.parent is not None:
            parts.append(n.label)
            n = n.parent
        out = []
        for p in reversed(parts):
            out.extend(p)
        return tuple(out)


def is_terminator(x):
    return isinstance(x, tuple) and len(x) == 2 and x[0] == "$"


def constraint_key(cons_by_pos, start, length):
    """Canonical string of the constraints on positions start..start+length-1,
    renumbered from 0. cons_by_pos maps a position to a sorted tuple of constraint
    descriptions."""
    parts = []
    for i in range(start, start + length):
        if cons_by_pos.get(i):
            parts.append(f"{i - start}:" + "&".join(cons_by_pos[i]))
    return "|".join(parts)


class OverlapTree:
    def __init__(self):
        self.root = Node(None, (), 0)
        self.n_queries = 0
        self.n_leaves = 0

    def insert(self, types, cons_by_pos=None):
        """Insert a metapath (sequence of type symbols) with its per-position constraint
        descriptions; returns the query id used in its terminator."""
        cons_by_pos = cons_by_pos or {}
        qid = self.n_queries
        self.n_queries += 1
        s = tuple(types) + (("$", qid),)
        n = len(types)
        for k in range(n):
            self._insert_suffix(s[k:], k, n, cons_by_pos)
        return qid

    def _insert_suffix(self, suf, start, n, cons_by_pos):
        node, i = self.root, 0
        path = []
        while True:
            child = node.children.get(suf[i])
            if child is None:
                leaf = Node(node, suf[i:], node.depth + len(suf) - i)
                node.children[suf[i]] = leaf
                self.n_leaves += 1
                path.append(leaf)
                break
            lab = child.label
            j = 0
            while j < len(lab) and i + j < len(suf) and lab[j] == suf[i + j]:
                j += 1
            if j == len(lab):
                node, i = child, i + j
                path.append(child)
                continue
            # the match ends inside the edge into `child`: split it
            mid = Node(node, lab[:j], node.depth + j)
            node.children[suf[i]] = mid
            child.label = lab[j:]
            child.parent = mid
            mid.children[lab[j]] = child
            mid.f = child.f
            # the occurrences counted below `child` so far also pass through `mid`
            for k, e in child.cidx.items():
                mid.cidx.setdefault(restrict_key(k, mid.depth), Entry()).f += e.f
            self._move_entries(child, mid)
            leaf = Node(mid, suf[i + j:], mid.depth + len(suf) - i - j)
            mid.children[suf[i + j]] = leaf
            self.n_leaves += 1
            path += [mid, leaf]
            break
        for x in path:
            x.f += 1
            length = min(x.depth, n - start)   # positions of the metapath the node covers
            key = constraint_key(cons_by_pos, start, length)
            x.cidx.setdefault(key, Entry()).f += 1

    @staticmethod
    def _move_entries(child, mid):
        """A leaf's string minus its terminator may become an internal node's string when
        the same metapath arrives again; its constraint entries move there."""
        if len(child.label) == 1 and is_terminator(child.label[0]):
            for k, e in child.cidx.items():
                m = mid.cidx[k]
                m.p, m.c, m.rho = e.p, e.c, e.rho
                e.p = None

    # ---- look-ups

    def locate(self, s):
        """(node, exact) for a symbol string: the node at or just below the end of the
        match, and whether the string ends exactly at that node; (None, False) when s
        does not occur."""
        node, i = self.root, 0
        s = tuple(s)
        while i < len(s):
            child = node.children.get(s[i])
            if child is None:
                return None, False
            lab = child.label
            j = 0
            while j < len(lab) and i + j < len(s):
                if lab[j] != s[i + j]:
                    return None, False
                j += 1
            i += j
            if i == len(s):
                return child, j == len(lab)
            node = child
        return node, True

    def frequency(self, s, key=None):
        """Occurrences of sub-metapath s (with constraint key, if given)."""
        node, _ = self.locate(s)
        if node is None:
            return 0
        if key is None:
            return node.f
        # the constraint entries live on the node at or below the end of s; count the
        # occurrences whose constraints on s's positions match key
        return self._key_freq(node, len(s), key)

    def _key_freq(self, node, length, key):
        e = node.cidx.get(key) if node.depth == length or self._ends_in_terminator(node, length) else None
        if e is not None:
            return e.f
        # s ends inside the edge into node: every suffix below shares the same first
        # `length` positions, so count leaves below whose recorded key restricted to
        # `length` equals key
        return sum(1 for leaf_key in self._leaf_keys(node, length) if leaf_key == key)

    @staticmethod
    def _ends_in_terminator(node, length):
        return node.is_leaf() and node.depth - 1 == length

    def _leaf_keys(self, node, length):
        for leaf in self.leaves(node):
            for k, e in leaf.cidx.items():
                yield from [restrict_key(k, length)] * e.f

    def leaves(self, node=None):
        node = node or self.root
        stack = [node]
        while stack:
            x = stack.pop()
            if x.is_leaf():
                yield x
            else:
                stack.extend(x.children.values())

    def nodes(self):
        stack = [self.root]
        while stack:
            x = stack.pop()
            yield x
            stack.extend(x.children.values())


def restrict_key(key, length):
    """A constraint key restricted to the first `length` positions."""
    if not key:
        return key
    keep = [p for p in key.split("|") if int(p.split(":", 1)[0]) < length]
    return "|".join(keep)
