"""The tuner's table writer (host logic, no GPU): the C table it writes
parses back to the chosen row-group sizes, and the committed table has the
writer's form."""

import os
import re

from paper_1104_3408_gb300 import tune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ENTRY = re.compile(r"\{(\d+), (\d+), (\d+), (\d+), 0, \{([\d, ]+)\}\},")


def _entries(text):
    return [(int(a), int(b), int(c), int(d), [int(x) for x in r.split(",")])
            for a, b, c, d, r in ENTRY.findall(text)]


def test_table_round_trip():
    res = [{"n_r": 33, "n_theta": 48, "L": 46, "n_fields": 50, "rows": [48, 96, 96, 48, 96]},
           {"n_r": 9, "n_theta": 12, "L": 10, "n_fields": 50, "rows": [48] * 5}]
    got = _entries(tune.table_text(res))
    assert got == [(33, 48, 46, 50, [48, 96, 96, 48, 96]), (9, 12, 10, 50, [48] * 5),
                   (0, 0, 0, 0, [0] * 5)]


def test_committed_table_lists_the_tuned_shapes():
    with open(os.path.join(ROOT, "paper_1104_3408_gb300", "csrc", "tile_table.h")) as fh:
        got = _entries(fh.read())
    assert got[-1][0] == 0  # end of table
    shapes = {(e[0], e[1], e[2], e[3]) for e in got[:-1]}
    assert shapes == {(n_r, nt, L, nf) for n_r, nt, L, nf, _ in tune.default_shapes()}
    for e in got[:-1]:
        n_r, nt, L = e[0], e[1], e[2]
        for rows, P in zip(e[4], tune.family_rows(n_r, nt, L)):
            # 48 up to 48 operator rows; either candidate above
            assert rows in ((48,) if P <= 48 else (48, 96))
