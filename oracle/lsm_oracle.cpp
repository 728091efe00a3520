// CPU oracle for the GPU LSM dictionary (Ashkiani et al., "GPU LSM: A Dynamic
// Dictionary Data Structure for the GPU", arXiv 1707.05354).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
// calls this file; only the tests, the smoke check and the benchmark's CPU
// baseline do.  It shares no code, header, table or helper with the CUDA path.
//
// Three independent models live here, each written plainly and slowly:
//
//   O1  ordered map (std::map).  The dictionary of §I-B, updated batch by batch
//       under the batch semantics of §III-A.  This is the plain definition of
//       what every query must return; it is also the timed CPU baseline.
//   O2  offline last-writer oracle.  Sorts the whole operation log once and
//       keeps, per key, the outcome of the latest batch that touched it.  Same
//       answers as O1 (checked in the tests), built for inputs where O1 would
//       need many GB of map nodes.
//   S   structural model.  Replays the insertion algorithm of Fig. 2(a) and
//       Fig. 3 with std::stable_sort / std::merge on explicit per-level arrays,
//       so that the GPU's level contents can be compared bit for bit, and the
//       cleanup of §III-F / §IV-E on those arrays.
//
// Readings of the paper used here (each also listed in the design notes):
//   * key variable = (original key << 1) | status, status 1 = regular,
//     0 = tombstone (§IV-A).
//   * user keys are < 2^31 - 1; the key 2^31 - 1 is reserved for the cleanup
//     placebos, which are tombstones (§IV-E footnote; the printed 2^32 - 1
//     would carry status 1 and be visible).
//   * several inserts of one key in one batch: the last in input order wins
//     (§III-A rule 4 allows any choice; this one matches applying the ops to a
//     map in order).  A delete beats every insert of its key in the same batch
//     (rule 6).
//   * a short batch of n < b ops is padded with b - n copies of op n-1 (§IV-A).
//   * a tombstone's value is 0.
//   * count/range bounds are inclusive (§I-B); k1 > k2 gives an empty answer;
//     k2 >= 2^31 - 1 is clamped to 2^31 - 2.
//   * lookup of a tombstoned key reports "not found" (§III-D, §IV-B).
//   * cleanup: r' = ceil(n'/b), placebos fill the tail of the largest level,
//     live elements fill the set bits of r' in ascending level order (§IV-E).

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

namespace {

constexpr uint32_t kMaxUserKey = 0x7FFFFFFEu;   // 2^31 - 2, largest usable key
constexpr uint32_t kPlaceboKv = 0xFFFFFFFEu;    // key 2^31 - 1, tombstone

uint32_t key_variable(uint32_t key, bool is_delete) {
  // §IV-A: the original key shifted once, status bit in the LSB.
  return (key << 1) | (is_delete ? 0u : 1u);
}

// ---------------------------------------------------------------- O1 ------
struct O1 {
  std::map<uint32_t, uint32_t> m;
};

// One batch under §III-A: rules 5 and 6 first (every key deleted anywhere in
// the batch is gone, whatever else the batch does with it), then rule 3/4 for
// the remaining inserts, in input order so that the last one wins.
void o1_apply(O1* o, const uint32_t* keys, const uint32_t* vals,
              const uint8_t* is_del, uint64_t n) {
  std::map<uint32_t, bool> deleted;
  for (uint64_t i = 0; i < n; ++i)
    if (is_del[i]) deleted[keys[i]] = true;
  for (const auto& kv : deleted) o->m.erase(kv.first);
  for (uint64_t i = 0; i < n; ++i) {
    if (is_del[i]) continue;
    if (deleted.count(keys[i])) continue;
    o->m[keys[i]] = vals ? vals[i] : 0u;
  }
}

// ---------------------------------------------------------------- S -------
struct Elem {
  uint32_t kv;
  uint32_t v;
  uint32_t batch;   // batch number, kept only to check the building invariants
};

struct S {
  uint32_t b = 0;
  uint64_t r = 0;                         // number of resident batches
  std::vector<std::vector<Elem>> level;   // level[i] empty or of size b * 2^i
  uint32_t next_batch = 0;
};

bool key_less(const Elem& x, const Elem& y) { return (x.kv >> 1) < (y.kv >> 1); }
bool kv_less(const Elem& x, const Elem& y) { return x.kv < y.kv; }

// Fig. 2(a) / Fig. 3: sort the batch on the whole key variable, then merge it
// with every full level from the smallest up, ignoring the status bit, the
// buffer (newer) first among equal keys; the result lands in the first empty
// level.  The batch is sorted stably from the reversed input so that the last
// of several equal key variables comes first (rule 4 reading above).
void s_apply(S* s, const uint32_t* keys, const uint32_t* vals,
             const uint8_t* is_del, uint64_t n) {
  const uint32_t b = s->b;
  const uint32_t t = s->next_batch++;
  std::vector<Elem> ops(b);
  for (uint64_t i = 0; i < b; ++i) {
    const uint64_t j = i < n ? i : n - 1;   // pad with copies of op n-1
    const bool del = is_del[j] != 0;
    ops[i] = Elem{key_variable(keys[j], del), del ? 0u : (vals ? vals[j] : 0u), t};
  }
  std::reverse(ops.begin(), ops.end());
  std::stable_sort(ops.begin(), ops.end(), kv_less);

  std::vector<Elem> buffer = ops;
  size_t i = 0;
  while (i < s->level.size() && !s->level[i].empty()) {
    std::vector<Elem> merged(buffer.size() + s->level[i].size());
    // std::merge keeps elements of the first range ahead of equivalent ones
    // of the second range: the buffer holds the newer elements.
    std::merge(buffer.begin(), buffer.end(), s->level[i].begin(),
               s->level[i].end(), merged.begin(), key_less);
    buffer.swap(merged);
    s->level[i].clear();
    ++i;
  }
  if (i == s->level.size()) s->level.emplace_back();
  s->level[i] = buffer;
  s->r += 1;
}

// §III-F / §IV-E cleanup on the level arrays: merge all levels from the
// smallest (newest) to the largest, keep only the first element of each key
// and only if it is regular, pad with placebos to a multiple of b and slice the
// sorted result into the levels of r' = ceil(n'/b), smaller keys to smaller
// levels.
void s_cleanup(S* s) {
  std::vector<Elem> all;
  for (size_t i = 0; i < s->level.size(); ++i) {
    if (s->level[i].empty()) continue;
    std::vector<Elem> merged(all.size() + s->level[i].size());
    std::merge(all.begin(), all.end(), s->level[i].begin(), s->level[i].end(),
               merged.begin(), key_less);
    all.swap(merged);
  }
  std::vector<Elem> live;
  for (size_t i = 0; i < all.size(); ++i) {
    const bool head = (i == 0) || ((all[i - 1].kv >> 1) != (all[i].kv >> 1));
    if (head && (all[i].kv & 1u)) live.push_back(all[i]);
  }
  const uint64_t n_live = live.size();
  const uint64_t r_new = (n_live + s->b - 1) / s->b;
  while (live.size() < r_new * s->b) live.push_back(Elem{kPlaceboKv, 0u, 0xFFFFFFFFu});
  s->level.assign(64, std::vector<Elem>());
  uint64_t pos = 0;
  for (int i = 0; i < 64; ++i) {
    if (!((r_new >> i) & 1u)) continue;
    const uint64_t size = uint64_t(s->b) << i;
    s->level[i].assign(live.begin() + pos, live.begin() + pos + size);
    pos += size;
  }
  while (!s->level.empty() && s->level.back().empty()) s->level.pop_back();
  s->r = r_new;
}

// ---------------------------------------------------------------- O2 ------
struct Op {
  uint32_t key;
  uint32_t batch;
  uint32_t pos;
  uint32_t val;
  uint8_t del;
};

}  // namespace

extern "C" {

// ---- O1 ------------------------------------------------------------------
void* o1_new() { return new O1(); }
void o1_free(void* h) { delete static_cast<O1*>(h); }

// Applies one batch (any n >= 1; the batch is not split).
void o1_apply_batch(void* h, const uint32_t* keys, const uint32_t* vals,
                    const uint8_t* is_del, uint64_t n) {
  o1_apply(static_cast<O1*>(h), keys, vals, is_del, n);
}

uint64_t o1_size(void* h) { return static_cast<O1*>(h)->m.size(); }

// Writes the live pairs in ascending key order.
void o1_dump(void* h, uint32_t* keys, uint32_t* vals) {
  uint64_t i = 0;
  for (const auto& kv : static_cast<O1*>(h)->m) {
    keys[i] = kv.first;
    vals[i] = kv.second;
    ++i;
  }
}

// §I-B lookup: the value of k, or "not found" (found = 0, value 0).
void o1_lookup(void* h, const uint32_t* q, uint64_t nq, uint32_t* val,
               uint8_t* found) {
  const auto& m = static_cast<O1*>(h)->m;
  for (uint64_t i = 0; i < nq; ++i) {
    auto it = m.find(q[i]);
    found[i] = it != m.end();
    val[i] = it != m.end() ? it->second : 0u;
  }
}

// §I-B count: number of live keys k with k1 <= k <= k2.
void o1_count(void* h, const uint32_t* k1, const uint32_t* k2, uint64_t nq,
              uint32_t* count) {
  const auto& m = static_cast<O1*>(h)->m;
  for (uint64_t i = 0; i < nq; ++i) {
    const uint32_t hi = std::min(k2[i], kMaxUserKey);
    uint32_t c = 0;
    if (k1[i] <= hi)
      for (auto it = m.lower_bound(k1[i]); it != m.end() && it->first <= hi; ++it) ++c;
    count[i] = c;
  }
}

// Order-based neighbour queries that §II-A's footnote names beside the
// three retrievals (successor and predecessor of a key), read inclusively:
// successor(q) = the live pair with the smallest key >= q, predecessor(q) =
// the one with the largest key <= q (keys above 2^31 - 2 are never live).
// found[i] = 0 and key = value = 0 when there is none.
void o1_neighbor(void* h, const uint32_t* q, uint64_t nq, int successor, uint32_t* key, uint32_t* val,
                 uint8_t* found) {
  const auto& m = static_cast<O1*>(h)->m;
  for (uint64_t i = 0; i < nq; ++i) {
    key[i] = val[i] = 0;
    found[i] = 0;
    if (successor) {
      auto it = m.lower_bound(q[i]);
      if (it != m.end()) {
        key[i] = it->first;
        val[i] = it->second;
        found[i] = 1;
      }
    } else {
      auto it = m.upper_bound(std::min(q[i], kMaxUserKey));
      if (it != m.begin()) {
        --it;
        key[i] = it->first;
        val[i] = it->second;
        found[i] = 1;
      }
    }
  }
}

// §I-B range, as CSR: offsets[nq + 1] (first call with keys == nullptr only
// fills offsets), then keys/vals of each query in ascending key order.
void o1_range(void* h, const uint32_t* k1, const uint32_t* k2, uint64_t nq,
              uint64_t* offsets, uint32_t* keys, uint32_t* vals) {
  const auto& m = static_cast<O1*>(h)->m;
  uint64_t total = 0;
  for (uint64_t i = 0; i < nq; ++i) {
    offsets[i] = total;
    const uint32_t hi = std::min(k2[i], kMaxUserKey);
    if (k1[i] > hi) continue;
    for (auto it = m.lower_bound(k1[i]); it != m.end() && it->first <= hi; ++it) {
      if (keys) {
        keys[total] = it->first;
        vals[total] = it->second;
      }
      ++total;
    }
  }
  offsets[nq] = total;
}

// ---- S -------------------------------------------------------------------
void* s_new(uint32_t b) {
  S* s = new S();
  s->b = b;
  return s;
}
void s_free(void* h) { delete static_cast<S*>(h); }

// One batch of n <= b ops (n >= 1).
void s_apply_batch(void* h, const uint32_t* keys, const uint32_t* vals,
                   const uint8_t* is_del, uint64_t n) {
  s_apply(static_cast<S*>(h), keys, vals, is_del, n);
}

void s_cleanup_all(void* h) { s_cleanup(static_cast<S*>(h)); }

uint64_t s_r(void* h) { return static_cast<S*>(h)->r; }

// Size of level i (0 when empty or beyond the last level).
uint64_t s_level_size(void* h, int i) {
  S* s = static_cast<S*>(h);
  return i < int(s->level.size()) ? s->level[i].size() : 0;
}

// Copies level i: key variables, values and the batch number of each element.
void s_level(void* h, int i, uint32_t* kv, uint32_t* v, uint32_t* batch) {
  S* s = static_cast<S*>(h);
  const auto& lv = s->level[i];
  for (size_t j = 0; j < lv.size(); ++j) {
    kv[j] = lv[j].kv;
    v[j] = lv[j].v;
    if (batch) batch[j] = lv[j].batch;
  }
}

// ---- O2 ------------------------------------------------------------------
// Offline: given the whole log as (key, value, is_delete, batch number) in
// input order, write the sorted live dictionary and return its size.
// Per key, the latest batch touching it decides (§III-A rule 3); inside that
// batch a delete wins (rule 6), otherwise the last insert in input order
// (rule 4 reading).
uint64_t o2_build(const uint32_t* keys, const uint32_t* vals,
                  const uint8_t* is_del, const uint32_t* batch, uint64_t n,
                  uint32_t* out_keys, uint32_t* out_vals) {
  std::vector<Op> ops(n);
  for (uint64_t i = 0; i < n; ++i)
    ops[i] = Op{keys[i], batch[i], uint32_t(i), vals ? vals[i] : 0u, is_del[i]};
  std::sort(ops.begin(), ops.end(), [](const Op& x, const Op& y) {
    if (x.key != y.key) return x.key < y.key;
    if (x.batch != y.batch) return x.batch > y.batch;
    return x.pos > y.pos;
  });
  uint64_t out = 0;
  for (uint64_t i = 0; i < n;) {
    uint64_t j = i;
    bool any_delete = false;
    while (j < n && ops[j].key == ops[i].key && ops[j].batch == ops[i].batch) {
      any_delete |= ops[j].del != 0;
      ++j;
    }
    if (!any_delete) {           // ops[i] is the last insert of the latest batch
      out_keys[out] = ops[i].key;
      out_vals[out] = ops[i].val;
      ++out;
    }
    while (j < n && ops[j].key == ops[i].key) ++j;
    i = j;
  }
  return out;
}

// Closed form of a single full level.  When r is a power of two, every
// resident batch sits in level log2(r), and Fig. 2(a) / Fig. 3 make its order
//   key ascending; newer batch first (§III-B); inside a batch the stable sort
//   of the reversed input on the key variable (tombstone first, then the
//   later op first).
// Input: the padded ops of every batch in arrival order (batch number per op),
// output: the level's key variables and values.
void o2_single_level(const uint32_t* keys, const uint32_t* vals, const uint8_t* is_del,
                     const uint32_t* batch, uint64_t n, uint32_t* out_kv, uint32_t* out_v) {
  std::vector<Op> ops(n);
  for (uint64_t i = 0; i < n; ++i)
    ops[i] = Op{keys[i], batch[i], uint32_t(i), vals ? vals[i] : 0u, is_del[i]};
  std::sort(ops.begin(), ops.end(), [](const Op& x, const Op& y) {
    if (x.key != y.key) return x.key < y.key;
    if (x.batch != y.batch) return x.batch > y.batch;
    if (x.del != y.del) return x.del > y.del;
    return x.pos > y.pos;
  });
  for (uint64_t i = 0; i < n; ++i) {
    out_kv[i] = key_variable(ops[i].key, ops[i].del != 0);
    out_v[i] = ops[i].del ? 0u : ops[i].val;
  }
}

}  // extern "C"
