"""The seeded workload generators (host only): the batched workload's anchors are valid
node ids of the anchored type, the anchored share is near the requested one, the draws are
reproducible, and the full-size queries anchor every template but APA."""
import numpy as np

import gen


def test_batched_anchors_are_valid_and_reproducible():
    qs = gen.batched_queries(seed=3, n=256, pool=500, anchor_p=0.75)
    again = gen.batched_queries(seed=3, n=256, pool=500, anchor_p=0.75)
    assert qs == again
    counts = gen.CONFIG1_COUNTS
    anchored = 0
    for q in qs:
        eqs = [c for c in q["constraints"] if c["prop"] is None]
        if eqs:
            anchored += 1
            assert len(eqs) == 1 and eqs[0]["pos"] == 0 and eqs[0]["op"] == "eq"
            assert 0 <= eqs[0]["lo"] < counts[q["types"][0]]
    assert 0.65 < anchored / len(qs) < 0.85
    plain = gen.batched_queries(seed=3, n=256, pool=500)
    assert all(not any(c["prop"] is None for c in q["constraints"]) for q in plain)
    # anchoring only adds the first-node constraint: the template draw is unchanged
    for a, b in zip(qs, plain):
        assert a["types"] == b["types"]
        assert [c for c in a["constraints"] if c["prop"] is not None] == b["constraints"]


def test_full_size_queries_anchor_all_but_apa():
    h = gen.config2_hin(seed=2, scale=0.001)
    qs = gen.config2_queries(h, seed=2, n_anchor_a=8, n_anchor_t=4, n_anchor_v=4)
    assert len(qs) == 20
    for q in qs:
        name = "".join(q["types"])
        ids = [c for c in q["constraints"] if c["prop"] is None]
        years = [c for c in q["constraints"] if c["prop"] == "year"]
        assert len(years) == q["types"].count("P")
        assert all((c["lo"], c["hi"]) == (2010, 2020) for c in years)
        if name == "APA":
            assert not ids
        else:
            assert len(ids) == 1 and ids[0]["pos"] == 0 and ids[0]["op"] == "in"
            s = np.asarray(ids[0]["set"])
            assert s.size > 0 and s.max() < h["types"][q["types"][0]]
