"""Parser for the hand-derived golden walkthroughs under tests/golden/."""

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse(name):
    """Returns (b, steps); each step is a tuple whose first item names it."""
    b = None
    steps = []
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            t = line.split()
            if t[0] == "b":
                b = int(t[1])
            elif t[0] == "cleanup":
                steps.append(("cleanup",))
            elif t[0] == "op":
                kind, args = t[1], t[2:]
                keys, vals, dels = [], [], []
                for a in args:
                    if kind == "delete":
                        keys.append(int(a)); vals.append(0); dels.append(1)
                    elif kind == "insert":
                        k, v = a.split(":"); keys.append(int(k)); vals.append(int(v)); dels.append(0)
                    elif kind == "update":
                        if a.startswith("-"):
                            keys.append(int(a[1:])); vals.append(0); dels.append(1)
                        else:
                            k, v = a.lstrip("+").split(":"); keys.append(int(k)); vals.append(int(v)); dels.append(0)
                    else:
                        raise ValueError(kind)
                steps.append(("op", kind, np.array(keys, np.uint32), np.array(vals, np.uint32),
                              np.array(dels, np.uint8)))
            elif t[0] == "expect":
                what = t[1]
                if what == "r":
                    steps.append(("r", int(t[2])))
                elif what == "level":
                    i = int(t[2])
                    if t[3] == "empty":
                        steps.append(("level", i, None, None))
                    else:
                        vi = t.index("v")
                        kv = np.array([int(x) for x in t[4:vi]], np.uint32)
                        v = np.array([int(x) for x in t[vi + 1:]], np.uint32)
                        steps.append(("level", i, kv, v))
                elif what == "lookup":
                    q, val, found = [], [], []
                    for a in t[2:]:
                        k, r = a.split("=")
                        q.append(int(k))
                        found.append(0 if r == "none" else 1)
                        val.append(0 if r == "none" else int(r))
                    steps.append(("lookup", np.array(q, np.uint32), np.array(val, np.uint32),
                                  np.array(found, np.uint8)))
                elif what == "count":
                    steps.append(("count", int(t[2]), int(t[3]), int(t[4])))
                elif what == "range":
                    kv = [tuple(int(x) for x in a.split(":")) for a in t[4:]]
                    steps.append(("range", int(t[2]), int(t[3]), kv))
                else:
                    raise ValueError(what)
            else:
                raise ValueError(line)
    return b, steps


def levels_lookup(levels, q):
    """Lookup rule of §III-D on explicit level arrays listed newest first."""
    for kv, v in levels:
        if len(kv) == 0:
            continue
        i = int(np.searchsorted(kv >> 1, q, side="left"))
        if i < len(kv) and (int(kv[i]) >> 1) == q:
            return (1, int(v[i])) if (int(kv[i]) & 1) else (0, 0)
    return (0, 0)
