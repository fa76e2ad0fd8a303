"""The oracle against hand-worked cases stored under tests/golden/ (each file
states the passage it follows and how its values were worked out)."""
import os

import numpy as np

HERE = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name):
    with open(os.path.join(HERE, name)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if line:
                yield line


def _schedule_cases():
    cases, cur = [], None
    for line in _lines("schedules.txt"):
        key, _, rest = line.partition(" ")
        if key == "case":
            cur = {"name": rest.strip()}
            cases.append(cur)
        elif key in ("count", "target"):
            cur[key] = np.array([int(v) for v in rest.split()], dtype=np.int64)
        else:
            links = []
            for tok in rest.split():
                sd, amt = tok.split(":")
                s, d = sd.split(">")
                links.append((int(s), int(d), int(amt)))
            cur[key] = links
    return cases


def test_schedules_match_hand_worked_cases(orc):
    cases = _schedule_cases()
    assert len(cases) >= 4
    scheme = {"gs": orc.RPA_GS, "sgs": orc.RPA_SGS, "lgs": orc.RPA_LGS}
    for c in cases:
        for key, sch in scheme.items():
            s, d, a = orc.schedule(sch, c["count"], c["target"])
            got = list(zip(s.tolist(), d.tolist(), a.tolist()))
            assert got == c[key], (c["name"], key, got)


def test_systematic_matches_hand_worked_cases(orc):
    n = 0
    for line in _lines("systematic.txt"):
        _, body = line.split(" ", 1)
        q, u, anc = (part.split() for part in body.split("|"))
        q = np.array([int(v) for v in q], dtype=np.uint64)
        rc, got, off = orc.systematic(q, int(u[0]))
        assert rc == 0
        want = [int(v) for v in anc]
        assert got.tolist() == want, (q.tolist(), u, got.tolist())
        assert np.array_equal(off, np.bincount(want, minlength=len(q)))
        n += 1
    assert n >= 6
