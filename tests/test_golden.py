"""Figures the paper prints (tests/golden/paper_facts.json, each with its citation)."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_pairs_per_site():
    facts = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))
    d = facts["dets_per_site_5718"]
    # all source x sink combinations: one determinant per (i, j) pair (Sec. 4)
    assert d["terms"] ** 2 == d["value"]
    idx = np.indices((7, 5)).reshape(2, -1)
    assert idx.shape[1] == 7 * 5
