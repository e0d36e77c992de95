"""Shared helpers for the tests: random tiny acyclic queries and relations."""
from __future__ import annotations

import random
from typing import List, Tuple

import numpy as np


def random_tree_query(rng: random.Random, r: int, share_prob: float = 0.4):
    """A random connected acyclic query over r relations.  Relation k > 0 joins a random
    earlier relation; each endpoint is a fresh attribute or, with probability
    share_prob, an attribute that relation already has (so a component can span
    three or more relations, as {0, 1, 3} in Figure 3)."""
    attrs: List[int] = [0] * r
    edges: List[Tuple[int, int, int, int]] = []

    def pick(k: int) -> int:
        if attrs[k] > 0 and rng.random() < share_prob:
            return rng.randrange(attrs[k])
        attrs[k] += 1
        return attrs[k] - 1

    for k in range(1, r):
        par = rng.randrange(k)
        a_par = pick(par)
        a_k = pick(k)
        edges.append((par, a_par, k, a_k))
    return attrs, edges


def random_relations(rng: random.Random, attrs: List[int], n_max: int, domain: int, signed: bool = True):
    rels = []
    for a in attrs:
        n = rng.randint(1, n_max)
        cols = np.array([[rng.randrange(domain) for _ in range(n)] for _ in range(a)], dtype=np.int64)
        w = np.array([rng.choice([-2, -1, 1, 1, 2, 3]) for _ in range(n)], dtype=np.int64) if signed else None
        rels.append((cols, w))
    return rels
