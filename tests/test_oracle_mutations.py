"""Planted mistakes in a copy of the oracle: every one must fail a pin.

The oracle is trusted because its pins (``tests/test_oracle.py``: the
hand-worked Fig. 1 walkthrough, one test per §III-A rule, brute force on
tiny logs, the building invariants of §III-B, closed forms, the cleanup
model of §IV-E) are fixed by the paper and the mathematics, not by the
oracle itself.  This file checks that those pins are strong enough: each
mutant below is a one-line slip of the kind a plausible mistake would make
(a dropped term, a wrong sign or index, a swapped operand, an off-by-one at
an inclusive bound), planted in a copy of the oracle, and the oracle tests
run against the copy in a child process must report a failed test.

The copy holds the oracle package, the oracle tests with their golden
fixtures and the seeded input generators; the repository's oracle is never
touched.  A child must fail a test (pytest exit status 1), not stop on a
collection or build error, and the unchanged copy must pass.
"""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CPP = "oracle/lsm_oracle.cpp"
PY = "oracle/__init__.py"
BRUTE = "oracle/brute.py"

# (name, file, text in the oracle, text planted instead); each text occurs
# exactly once in its file.
MUTANTS = [
    # §IV-A encoding and the batch sort (rule 4 reading: the last insert wins)
    ("status_bit_inverted", CPP,
     "return (key << 1) | (is_delete ? 0u : 1u);",
     "return (key << 1) | (is_delete ? 1u : 0u);"),
    ("batch_not_reversed", CPP,
     "  std::reverse(ops.begin(), ops.end());\n", ""),
    ("batch_sorted_by_key_only", CPP,
     "std::stable_sort(ops.begin(), ops.end(), kv_less);",
     "std::stable_sort(ops.begin(), ops.end(), key_less);"),
    ("pad_with_first_op", CPP,
     "const uint64_t j = i < n ? i : n - 1;",
     "const uint64_t j = i < n ? i : 0;"),
    ("tombstone_keeps_value", CPP,
     "del ? 0u : (vals ? vals[j] : 0u), t};",
     "vals ? vals[j] : 0u, t};"),
    # Fig. 2(a) / Fig. 3: the newer source first among equal keys
    ("level_before_buffer_on_ties", CPP,
     "std::merge(buffer.begin(), buffer.end(), s->level[i].begin(),\n"
     "               s->level[i].end(), merged.begin(), key_less);",
     "std::merge(s->level[i].begin(), s->level[i].end(), buffer.begin(),\n"
     "               buffer.end(), merged.begin(), key_less);"),
    ("merge_on_key_variable", CPP,
     "s->level[i].end(), merged.begin(), key_less);\n    buffer.swap(merged);",
     "s->level[i].end(), merged.begin(), kv_less);\n    buffer.swap(merged);"),
    ("levels_not_emptied", CPP,
     "    s->level[i].clear();\n    ++i;", "    ++i;"),
    # §III-F / §IV-E cleanup
    ("cleanup_without_head_test", CPP,
     "if (head && (all[i].kv & 1u)) live.push_back(all[i]);",
     "if (all[i].kv & 1u) live.push_back(all[i]);"),
    ("cleanup_older_level_first", CPP,
     "std::merge(all.begin(), all.end(), s->level[i].begin(), s->level[i].end(),",
     "std::merge(s->level[i].begin(), s->level[i].end(), all.begin(), all.end(),"),
    ("cleanup_r_off_by_one", CPP,
     "const uint64_t r_new = (n_live + s->b - 1) / s->b;",
     "const uint64_t r_new = (n_live + s->b) / s->b;"),
    ("cleanup_largest_level_first", CPP,
     "for (int i = 0; i < 64; ++i) {\n    if (!((r_new >> i) & 1u)) continue;",
     "for (int i = 63; i >= 0; --i) {\n    if (!((r_new >> i) & 1u)) continue;"),
    # §III-A rules in O1
    ("o1_deletes_not_erased", CPP,
     "  for (const auto& kv : deleted) o->m.erase(kv.first);\n", ""),
    ("o1_insert_beats_delete_in_batch", CPP,
     "    if (deleted.count(keys[i])) continue;\n", ""),
    ("o1_first_insert_wins", CPP,
     "    o->m[keys[i]] = vals ? vals[i] : 0u;",
     "    o->m.emplace(keys[i], vals ? vals[i] : 0u);"),
    # §I-B queries in O1 (inclusive bounds)
    ("o1_count_excludes_k2", CPP,
     "it != m.end() && it->first <= hi; ++it) ++c;",
     "it != m.end() && it->first < hi; ++it) ++c;"),
    ("o1_range_excludes_k1", CPP,
     "for (auto it = m.lower_bound(k1[i]); it != m.end() && it->first <= hi; ++it) {",
     "for (auto it = m.upper_bound(k1[i]); it != m.end() && it->first <= hi; ++it) {"),
    ("o1_predecessor_exclusive", CPP,
     "auto it = m.upper_bound(std::min(q[i], kMaxUserKey));",
     "auto it = m.lower_bound(std::min(q[i], kMaxUserKey));"),
    ("o1_successor_exclusive", CPP,
     "      auto it = m.lower_bound(q[i]);\n      if (it != m.end()) {",
     "      auto it = m.upper_bound(q[i]);\n      if (it != m.end()) {"),
    # O2 (offline last writer) and the single-level closed form
    ("o2_oldest_batch_first", CPP,
     "    if (x.batch != y.batch) return x.batch > y.batch;\n    return x.pos > y.pos;",
     "    if (x.batch != y.batch) return x.batch < y.batch;\n    return x.pos > y.pos;"),
    ("o2_first_insert_wins", CPP,
     "    return x.pos > y.pos;\n  });\n  uint64_t out = 0;",
     "    return x.pos < y.pos;\n  });\n  uint64_t out = 0;"),
    ("o2_delete_ignored", CPP,
     "      any_delete |= ops[j].del != 0;\n", ""),
    ("single_level_insert_before_tombstone", CPP,
     "if (x.del != y.del) return x.del > y.del;",
     "if (x.del != y.del) return x.del < y.del;"),
    ("single_level_pad_with_first_op", PY,
     "idx = np.minimum(np.arange(b), n - 1)",
     "idx = np.where(np.arange(b) < n, np.arange(b), 0)"),
    ("o2_count_excludes_k2", PY,
     'hi = np.searchsorted(self.keys, k2, side="right")',
     'hi = np.searchsorted(self.keys, k2, side="left")'),
    ("o2_lookup_ignores_key", PY,
     "hit = (i < len(self.keys)) & (self.keys[ic] == q)",
     "hit = (i < len(self.keys))"),
    # API-level splitting of a call into batches of b
    ("split_drops_last_chunk", PY,
     "for s in range(0, n, b):",
     "for s in range(0, n - n % b if n > b else n, b):"),
    # B (brute force from the log)
    ("brute_first_insert_wins", BRUTE,
     "            else:\n                value = v",
     "            elif value is None:\n                value = v"),
    ("brute_insert_beats_delete", BRUTE,
     "            if deleted:\n                return False, 0\n            return True, value",
     "            if value is None:\n                return False, 0\n            return True, value"),
    ("brute_range_excludes_k2", BRUTE,
     "            if k1 <= k <= k2:", "            if k1 <= k < k2:"),
    ("brute_oldest_batch_first", BRUTE,
     "    for batch in reversed(batches):", "    for batch in batches:"),
]


def make_copy(dst, mutant=None):
    """The oracle package, its tests and fixtures, and the input generators,
    copied to ``dst``; ``mutant`` (file, old, new) planted in the copy."""
    ignore = shutil.ignore_patterns("__pycache__", "*.pyc", "*.tmp.*")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ignore)
    os.makedirs(os.path.join(dst, "tests"))
    # the oracle tests and the helper modules beside them
    for f in os.listdir(os.path.join(ROOT, "tests")):
        if f.endswith(".py") and (f == "test_oracle.py" or not f.startswith("test_")):
            shutil.copy2(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    pkg = os.path.join(dst, "paper_1707_05354_gb300")
    os.makedirs(pkg)
    for f in ("__init__.py", "workload.py"):
        shutil.copy2(os.path.join(ROOT, "paper_1707_05354_gb300", f), os.path.join(pkg, f))
    if mutant is not None:
        rel, old, new = mutant
        path = os.path.join(dst, rel)
        with open(path) as fh:
            src = fh.read()
        assert src.count(old) == 1, "mutation site not unique in %s: %r" % (rel, old)
        with open(path, "w") as fh:
            fh.write(src.replace(old, new))
        # a planted C++ change must rebuild the copy's library
        if rel.endswith(".cpp"):
            lib = os.path.join(dst, "oracle", "liblsm_oracle.so")
            if os.path.exists(lib):
                os.remove(lib)


def run_oracle_tests(dst):
    env = dict(os.environ)
    env.pop("PYTHONPATH", None)
    env["PYTHONDONTWRITEBYTECODE"] = "1"
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", os.path.join("tests", "test_oracle.py")],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout[-3000:] + p.stderr[-2000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    jobs = {"unchanged": None}
    jobs.update({name: (rel, old, new) for name, rel, old, new in MUTANTS})
    dirs = {}
    for name, mut in jobs.items():
        d = str(tmp_path / name)
        os.makedirs(d)
        make_copy(d, mut)
        dirs[name] = d
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        res = dict(zip(jobs, ex.map(run_oracle_tests, [dirs[n] for n in jobs])))
    rc, out = res.pop("unchanged")
    assert rc == 0, "the unchanged copy must pass:\n" + out
    survivors = [n for n, (rc, _) in res.items() if rc == 0]
    assert not survivors, "planted mistakes no pin catches: %s" % survivors
    broken = {n: out for n, (rc, out) in res.items() if rc != 1}
    assert not broken, "mutants that did not build or collect:\n" + "\n".join(
        "%s:\n%s" % kv for kv in broken.items())


@pytest.mark.parametrize("name,rel,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutation_site_exists(name, rel, old, new):
    with open(os.path.join(ROOT, rel)) as fh:
        assert fh.read().count(old) == 1, name
