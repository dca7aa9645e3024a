// CPU oracle for the column-oriented Datalog fixpoint.
//
// TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU
// baseline leg of the bench load this library; the product path never does.
// It shares no code, header, table or helper with the GPU library.
//
// What it computes: the least fixpoint of positive Horn rules
// H <- B1, ..., Bn over the loaded facts (Section 2, "Datalog and RDF"),
// reached by rounds in which every rule is applied once (Section 3,
// "Schedule multiple rules per iteration"):
//   * semi-naive (Section 3, "Continuous Memory Layout": full / delta / new):
//       round 1 applies every rule to the loaded facts;
//       round r > 1 applies, for every rule and every body atom i whose
//       relation is derived by some rule (an IDB atom), the variant in which
//       atom i reads delta_{r-1}, the IDB atoms before i read
//       full_{r-1} - delta_{r-1}, and the IDB atoms after i read full_{r-1};
//       atoms over input-only (EDB) relations always read the full relation;
//       new_R is the union of the heads, delta_R = new_R - full_R
//       (the difference operator of Section 4, "Union and Deduplication"),
//       full_R = full_R U delta_R;
//   * naive: every round applies every rule to full_{r-1}.
// The loop stops after the first round in which every delta is empty.
// "iterations" counts the rounds that produced a non-empty delta.
//
// Relations are std::set of fixed-width tuples (unused trailing positions are
// zero), which orders them lexicographically by unsigned column value.
// Joins are left-to-right nested loops; every atom after the first is looked
// up through a std::map keyed on the positions bound when it is reached.

#include <array>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

namespace {

constexpr int kMaxArity = 8;
using Tuple = std::array<uint32_t, kMaxArity>;
using Rel = std::set<Tuple>;

struct Term {
  bool is_const;
  uint32_t v;  // constant value, or variable id
};
struct Atom {
  int rel;
  std::vector<Term> t;
};
struct Rule {
  Atom head;
  std::vector<Atom> body;
  std::vector<std::pair<uint32_t, uint32_t>> neq;  // variable ids that must differ
};

struct Oracle {
  std::vector<uint32_t> arity;
  std::vector<Rel> full;
  std::vector<Rule> rules;
  std::vector<std::vector<uint64_t>> delta_sizes;  // [relation][round]
  uint64_t rounds = 0;
  uint64_t iterations = 0;
  bool ran = false;
};

bool is_idb(const Oracle& o, int rel) {
  for (const Rule& r : o.rules)
    if (r.head.rel == rel) return true;
  return false;
}

// Applies one rule with body atom i reading *src[i]; inserts heads into out.
void eval_rule(const Rule& r, const std::vector<const Rel*>& src, Rel& out) {
  const size_t nb = r.body.size();
  uint32_t max_var = 0;
  for (const Atom& a : r.body)
    for (const Term& t : a.t)
      if (!t.is_const && t.v > max_var) max_var = t.v;
  // positions of atom i that are fixed when it is reached
  std::vector<std::vector<int>> key_pos(nb);
  std::vector<bool> seen(max_var + 1, false);
  for (size_t i = 0; i < nb; ++i) {
    const Atom& a = r.body[i];
    for (size_t k = 0; k < a.t.size(); ++k)
      if (a.t[k].is_const || seen[a.t[k].v]) key_pos[i].push_back(static_cast<int>(k));
    for (const Term& t : a.t)
      if (!t.is_const) seen[t.v] = true;
  }
  std::vector<std::map<std::vector<uint32_t>, std::vector<const Tuple*>>> index(nb);
  for (size_t i = 1; i < nb; ++i)
    for (const Tuple& t : *src[i]) {
      std::vector<uint32_t> key;
      for (int k : key_pos[i]) key.push_back(t[k]);
      index[i][key].push_back(&t);
    }
  std::vector<int64_t> env(max_var + 1, -1);

  // depth-first enumeration of bindings
  struct Frame {
    static void go(const Rule& r, const std::vector<const Rel*>& src,
                   const std::vector<std::vector<int>>& key_pos,
                   const std::vector<std::map<std::vector<uint32_t>, std::vector<const Tuple*>>>& index,
                   std::vector<int64_t>& env, size_t i, Rel& out) {
      if (i == r.body.size()) {
        for (const auto& ne : r.neq)
          if (env[ne.first] == env[ne.second]) return;
        Tuple h{};
        for (size_t k = 0; k < r.head.t.size(); ++k) {
          const Term& t = r.head.t[k];
          h[k] = t.is_const ? t.v : static_cast<uint32_t>(env[t.v]);
        }
        out.insert(h);
        return;
      }
      const Atom& a = r.body[i];
      auto try_tuple = [&](const Tuple& t) {
        std::vector<uint32_t> bound_here;
        bool ok = true;
        for (size_t k = 0; k < a.t.size() && ok; ++k) {
          const Term& term = a.t[k];
          if (term.is_const) {
            ok = t[k] == term.v;
          } else if (env[term.v] >= 0) {
            ok = static_cast<uint32_t>(env[term.v]) == t[k];
          } else {
            env[term.v] = t[k];
            bound_here.push_back(term.v);
          }
        }
        if (ok) go(r, src, key_pos, index, env, i + 1, out);
        for (uint32_t v : bound_here) env[v] = -1;
      };
      if (i == 0) {
        for (const Tuple& t : *src[0]) try_tuple(t);
      } else {
        std::vector<uint32_t> key;
        for (int k : key_pos[i]) {
          const Term& term = a.t[k];
          key.push_back(term.is_const ? term.v : static_cast<uint32_t>(env[term.v]));
        }
        auto it = index[i].find(key);
        if (it == index[i].end()) return;
        for (const Tuple* t : it->second) try_tuple(*t);
      }
    }
  };
  Frame::go(r, src, key_pos, index, env, 0, out);
}

Rel set_minus(const Rel& a, const Rel& b) {
  Rel d;
  for (const Tuple& t : a)
    if (!b.count(t)) d.insert(t);
  return d;
}

int64_t run(Oracle& o, bool naive, uint64_t max_iters) {
  const size_t nr = o.arity.size();
  std::vector<bool> idb(nr);
  for (size_t r = 0; r < nr; ++r) idb[r] = is_idb(o, static_cast<int>(r));
  o.delta_sizes.assign(nr, {});
  std::vector<Rel> delta(nr);
  o.rounds = 0;
  o.iterations = 0;
  for (uint64_t round = 1;; ++round) {
    if (round > max_iters + 1) return -5;
    std::vector<Rel> fresh(nr);
    for (const Rule& rule : o.rules) {
      const size_t nb = rule.body.size();
      std::vector<const Rel*> src(nb);
      if (naive || round == 1) {
        for (size_t j = 0; j < nb; ++j) src[j] = &o.full[rule.body[j].rel];
        eval_rule(rule, src, fresh[rule.head.rel]);
        continue;
      }
      bool has_idb_atom = false;
      for (size_t i = 0; i < nb; ++i) {
        if (!idb[rule.body[i].rel]) continue;
        has_idb_atom = true;
        std::vector<Rel> olds;  // full - delta for IDB atoms before i
        olds.reserve(nb);
        for (size_t j = 0; j < nb; ++j) {
          const int rel = rule.body[j].rel;
          if (j == i) {
            src[j] = &delta[rel];
          } else if (idb[rel] && j < i) {
            olds.push_back(set_minus(o.full[rel], delta[rel]));
            src[j] = &olds.back();
          } else {
            src[j] = &o.full[rel];
          }
        }
        eval_rule(rule, src, fresh[rule.head.rel]);
      }
      (void)has_idb_atom;  // EDB-only rules add nothing after round 1
    }
    bool any = false;
    for (size_t r = 0; r < nr; ++r) {
      delta[r] = set_minus(fresh[r], o.full[r]);
      for (const Tuple& t : delta[r]) o.full[r].insert(t);
      o.delta_sizes[r].push_back(delta[r].size());
      if (!delta[r].empty()) any = true;
    }
    o.rounds = round;
    if (!any) break;
    o.iterations = round;
  }
  o.ran = true;
  return static_cast<int64_t>(o.iterations);
}

}  // namespace

extern "C" {

void* orc_new(void) { return new Oracle(); }
void orc_free(void* h) { delete static_cast<Oracle*>(h); }

int orc_add_relation(void* h, uint32_t arity) {
  Oracle& o = *static_cast<Oracle*>(h);
  if (arity < 1 || arity > kMaxArity) return -1;
  o.arity.push_back(arity);
  o.full.emplace_back();
  return static_cast<int>(o.arity.size() - 1);
}

// rows: n tuples, row-major, arity values each.
int orc_load(void* h, int rel, const uint32_t* rows, uint64_t n) {
  Oracle& o = *static_cast<Oracle*>(h);
  if (rel < 0 || rel >= static_cast<int>(o.arity.size())) return -1;
  const uint32_t a = o.arity[rel];
  for (uint64_t i = 0; i < n; ++i) {
    Tuple t{};
    for (uint32_t k = 0; k < a; ++k) t[k] = rows[i * a + k];
    o.full[rel].insert(t);
  }
  return 0;
}

// Flat rule encoding:
//   head_rel, head_arity, (is_const, value) * head_arity,
//   nbody, [rel, arity, (is_const, value) * arity] * nbody,
//   nneq, (var_a, var_b) * nneq
int orc_add_rule(void* h, const int64_t* s, uint32_t len) {
  Oracle& o = *static_cast<Oracle*>(h);
  uint32_t p = 0;
  auto next = [&](int64_t& v) {
    if (p >= len) return false;
    v = s[p++];
    return true;
  };
  auto read_atom = [&](Atom& a) {
    int64_t rel, ar;
    if (!next(rel) || !next(ar)) return false;
    if (rel < 0 || rel >= static_cast<int64_t>(o.arity.size()) || ar != o.arity[rel]) return false;
    a.rel = static_cast<int>(rel);
    for (int64_t k = 0; k < ar; ++k) {
      int64_t c, v;
      if (!next(c) || !next(v)) return false;
      a.t.push_back(Term{c != 0, static_cast<uint32_t>(v)});
    }
    return true;
  };
  Rule r;
  if (!read_atom(r.head)) return -1;
  int64_t nb, nn;
  if (!next(nb) || nb < 1) return -1;
  for (int64_t i = 0; i < nb; ++i) {
    Atom a;
    if (!read_atom(a)) return -1;
    r.body.push_back(a);
  }
  if (!next(nn)) return -1;
  for (int64_t i = 0; i < nn; ++i) {
    int64_t x, y;
    if (!next(x) || !next(y)) return -1;
    r.neq.emplace_back(static_cast<uint32_t>(x), static_cast<uint32_t>(y));
  }
  o.rules.push_back(r);
  return 0;
}

int64_t orc_run(void* h, int naive, uint64_t max_iters) {
  return run(*static_cast<Oracle*>(h), naive != 0, max_iters);
}

uint64_t orc_size(void* h, int rel) { return static_cast<Oracle*>(h)->full.at(rel).size(); }

int orc_export(void* h, int rel, uint32_t* rows) {
  Oracle& o = *static_cast<Oracle*>(h);
  const uint32_t a = o.arity.at(rel);
  uint64_t i = 0;
  for (const Tuple& t : o.full[rel]) {
    for (uint32_t k = 0; k < a; ++k) rows[i * a + k] = t[k];
    ++i;
  }
  return 0;
}

uint64_t orc_rounds(void* h) { return static_cast<Oracle*>(h)->rounds; }

int orc_delta_sizes(void* h, int rel, uint64_t* out, uint64_t cap) {
  Oracle& o = *static_cast<Oracle*>(h);
  const auto& d = o.delta_sizes.at(rel);
  for (uint64_t i = 0; i < d.size() && i < cap; ++i) out[i] = d[i];
  return static_cast<int>(d.size());
}

}  // extern "C"
