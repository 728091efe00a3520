"""Brute-force dictionary answers from the raw operation log (tiny inputs only).

TEST INFRASTRUCTURE ONLY: the product library never imports this module.

This is the plain definition of §I-B under the batch semantics of §III-A,
written without any data structure: to answer a query about key k, walk the
batches from the newest to the oldest and stop at the first batch that mentions
k.  Inside that batch a delete of k wins over any insert of k (rule 6);
otherwise the last insert of k in input order wins (rule 4, read as "last
wins").  A key no batch mentions is absent.  Pure Python loops, so only for
logs of a few thousand operations.

A batch is a list of (key, value, is_delete) triples in input order.
"""

MAX_USER_KEY = (1 << 31) - 2


def state_of(batches, key):
    """(found, value) for one key."""
    for batch in reversed(batches):
        mentioned = False
        deleted = False
        value = None
        for k, v, d in batch:
            if k != key:
                continue
            mentioned = True
            if d:
                deleted = True
            else:
                value = v
        if mentioned:
            if deleted:
                return False, 0
            return True, value
    return False, 0


def lookup(batches, queries):
    return [state_of(batches, q) for q in queries]


def range_query(batches, k1, k2):
    """Sorted list of live (key, value) with k1 <= key <= k2 (inclusive)."""
    k2 = min(k2, MAX_USER_KEY)
    if k1 > k2:
        return []
    keys = set()
    for batch in batches:
        for k, _, _ in batch:
            if k1 <= k <= k2:
                keys.add(k)
    out = []
    for k in sorted(keys):
        found, v = state_of(batches, k)
        if found:
            out.append((k, v))
    return out


def count(batches, k1, k2):
    return len(range_query(batches, k1, k2))


def count_by_enumeration(batches, k1, k2):
    """Count by testing every key in [k1, k2] one by one (small widths only)."""
    k2 = min(k2, MAX_USER_KEY)
    return sum(1 for k in range(k1, k2 + 1) if state_of(batches, k)[0])


def neighbor(batches, q, successor=True):
    """(key, value) of the live key nearest to q on one side (inclusive), or
    None: every key the log mentions on that side, tested one by one."""
    keys = set()
    for batch in batches:
        for k, _, _ in batch:
            if (k >= q) if successor else (k <= min(q, MAX_USER_KEY)):
                keys.add(k)
    for k in (sorted(keys) if successor else sorted(keys, reverse=True)):
        found, v = state_of(batches, k)
        if found:
            return k, v
    return None
