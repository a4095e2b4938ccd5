"""Values printed in the paper: the spatial-hash constants of Section 4.1
(tests/golden/teschner_constants.txt) are the ones the GPU hash uses."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_teschner_constants_match_the_paper():
    golden = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "teschner_constants.txt")):
        if line.strip() and not line.startswith("#"):
            axis, c = line.split()
            golden[axis] = int(c)
    src = open(os.path.join(ROOT, "include", "hc_core.cuh")).read()
    body = src[src.index("teschner(unsigned long long key)"):]
    body = body[:body.index("\n}\n")]
    used = dict(re.findall(r"\((\w) \* (\d+)ull\)", body))
    assert {k: int(v) for k, v in used.items()} == golden
