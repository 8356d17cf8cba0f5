"""Pin of the oracle's Philox4x32-10 against the published known-answer vectors."""
import json
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers(orc):
    kat = json.load(open(os.path.join(GOLD, "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        out = orc.philox4x32_10(ctr, key)
        assert [int(x) for x in out] == [int(x, 16) for x in v["out"]]


def test_uniform_is_24_bit_and_roughly_uniform(orc):
    u = np.array([orc.philox_uniform(12345, p, 987654321) for p in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all((u * 2 ** 24) == np.floor(u * 2 ** 24))
    # Kolmogorov-Smirnov distance of 20000 uniforms: well below 0.02 (p ~ 1e-7)
    s = np.sort(u)
    ks = np.max(np.abs(s - (np.arange(1, s.size + 1) / s.size)))
    assert ks < 0.02
