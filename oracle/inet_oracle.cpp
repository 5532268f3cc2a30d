// inet_oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, sequential evaluator of the lightweight interaction calculus
// (Sec. 2.2).  It exists to check the CUDA evaluator: only tests, the smoke
// check and the CPU-baseline leg of the benchmark may build or run it.  It
// shares no code, header or table with the CUDA path and has its own parser.
//
// What it computes (Sec. 2.2, "Communication", "Substitution", "Collect",
// "Interaction"; Theorem 1):
//   * a configuration < t.. | Delta > is held literally, as interface terms
//     and a multiset of equations whose sides are term trees;
//   * ->int and ->com are applied until neither applies (Theorem 1 says these
//     two rules alone reach the normal form with respect to active pairs);
//   * then ->col and ->sub are applied exhaustively (they never create an
//     active pair, so they are pushed to the end, as the paper argues after
//     Theorem 1);
//   * the result is the interface rendered with canonical names, the number
//     of ->int steps (total and per rule), and the number of live agents.
//
// Schedules: "lifo" (default), "fifo", "random" (seeded), and "rounds":
// every active pair present at the start of a round is reduced, then ->com
// runs to a fixpoint; the size of each round is recorded.  By uniform
// confluence (Sec. 2.1, Proposition on uniform confluence) every schedule
// gives the same result and the same number of interactions.  "--eager"
// interleaves ->col/->sub after every step instead of deferring them, to
// check Theorem 1's claim that deferring them changes nothing.
//
// Parity pins for every function here live in tests/ (closed forms, the
// paper's worked examples, brute force over reduction orders).
//
// Usage: inet_oracle RULES_FILE NETS_FILE [--mode lifo|fifo|random|rounds]
//        [--seed S] [--eager] [--threads T] [--max-interactions N]
//        [--max-result-chars N] [--quiet]
// Output: one JSON object per net, one per line, in input order.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <random>
#include <stdexcept>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

constexpr int kMaxArity = 8;

// ---------------------------------------------------------------------------
// Terms (Sec. 2.2, "Terms"): t = x | alpha(t1, ..., tn).

struct Term {
  int sym = -1;          // agent symbol index, or -1 for a name
  int64_t name = -1;     // name id when sym == -1
  Term* arg[kMaxArity] = {};
};

struct Symbols {
  std::vector<std::string> names;
  std::vector<int> arity;
  std::map<std::string, int> index;
  int get(const std::string& s, int ar) {
    auto it = index.find(s);
    if (it == index.end()) {
      int id = (int)names.size();
      names.push_back(s);
      arity.push_back(ar);
      index[s] = id;
      return id;
    }
    if (arity[it->second] != ar)
      throw std::runtime_error("PARSE: symbol " + s + " used with two arities");
    return it->second;
  }
};

// ---------------------------------------------------------------------------
// Parser for the text syntax.  Upper-case initial = agent symbol, lower-case
// initial = name (Sec. 3.3 distinguishes agents and variables by case).  A
// term is parsed into a syntax tree of strings first (iteratively, numerals
// can be millions deep).

struct PNode {           // parsed term: symbol or name with children indexes
  std::string id;
  bool is_name = false;
  std::vector<int> kids;
};

struct Lexer {
  const std::string& s;
  size_t i = 0;
  explicit Lexer(const std::string& src) : s(src) {}
  void skip() {
    for (;;) {
      while (i < s.size() && (s[i] == ' ' || s[i] == '\t' || s[i] == '\n' || s[i] == '\r')) i++;
      if (i < s.size() && s[i] == '#') {
        while (i < s.size() && s[i] != '\n') i++;
        continue;
      }
      return;
    }
  }
  bool eof() { skip(); return i >= s.size(); }
  char peek() { skip(); return i < s.size() ? s[i] : '\0'; }
  bool accept(const char* tok) {
    skip();
    size_t n = strlen(tok);
    if (s.compare(i, n, tok) == 0) { i += n; return true; }
    return false;
  }
  void expect(const char* tok) {
    if (!accept(tok)) throw std::runtime_error(std::string("PARSE: expected '") + tok + "' at offset " + std::to_string(i));
  }
  std::string ident() {
    skip();
    size_t b = i;
    if (i < s.size() && isalpha((unsigned char)s[i])) {
      i++;
      while (i < s.size() && (isalnum((unsigned char)s[i]) || s[i] == '_' || s[i] == '\'')) i++;
    }
    if (b == i) throw std::runtime_error("PARSE: expected identifier at offset " + std::to_string(i));
    return s.substr(b, i - b);
  }
};

// Parse one term into pool; returns the root index.  Iterative.
int parse_term(Lexer& lx, std::vector<PNode>& pool) {
  struct Frame { int node; };
  std::vector<Frame> stack;
  int root = -1;
  for (;;) {
    std::string id = lx.ident();
    int me = (int)pool.size();
    pool.push_back(PNode{});
    pool[me].id = id;
    pool[me].is_name = islower((unsigned char)id[0]) != 0;
    if (!stack.empty()) pool[stack.back().node].kids.push_back(me);
    else root = me;
    if (!pool[me].is_name && lx.accept("(")) {
      if (lx.accept(")")) {
        // S() == S with no arguments
      } else {
        stack.push_back({me});
        continue;  // parse first child
      }
    }
    // finished a term: close parents while possible
    for (;;) {
      if (stack.empty()) return root;
      if (lx.accept(",")) break;  // next sibling
      lx.expect(")");
      stack.pop_back();
    }
  }
}

// ---------------------------------------------------------------------------
// Rules (Sec. 2.2, "Interaction Rules"): alpha(x..) = beta(y..) -> Theta.

struct RTerm {           // rule template term
  int sym = -1;          // -1 = name
  int var = -1;          // rule-local name index
  std::vector<RTerm> kids;
};

struct Rule {
  int a = -1, b = -1;             // LHS symbols
  std::vector<int> a_vars, b_vars; // rule-local name index of each LHS port
  std::vector<std::pair<RTerm, RTerm>> rhs;
  int nvars = 0;                   // rule-local names (LHS and bound)
  std::vector<bool> is_lhs;        // per rule-local name
  int rhs_agents = 0;
};

struct RuleSet {
  Symbols sym;
  std::vector<Rule> rules;
  // (alpha, beta) -> rule index * 2 + flipped
  std::map<std::pair<int, int>, int> table;
};

RTerm to_rterm(const std::vector<PNode>& pool, int n, Symbols& sym,
               std::map<std::string, int>& vars, std::vector<int>& occ) {
  RTerm t;
  const PNode& p = pool[n];
  if (p.is_name) {
    auto it = vars.find(p.id);
    int v;
    if (it == vars.end()) { v = (int)vars.size(); vars[p.id] = v; occ.push_back(0); }
    else v = it->second;
    occ[v]++;
    t.var = v;
    return t;
  }
  t.sym = sym.get(p.id, (int)p.kids.size());
  for (int k : p.kids) t.kids.push_back(to_rterm(pool, k, sym, vars, occ));
  return t;
}

int count_agents(const RTerm& t) {
  if (t.sym < 0) return 0;
  int c = 1;
  for (auto& k : t.kids) c += count_agents(k);
  return c;
}

RuleSet parse_rules(const std::string& text) {
  RuleSet rs;
  Lexer lx(text);
  while (!lx.eof()) {
    std::vector<PNode> pool;
    int l = parse_term(lx, pool);
    lx.expect("=");
    int r = parse_term(lx, pool);
    lx.expect("->");
    if (pool[l].is_name || pool[r].is_name) throw std::runtime_error("PARSE: rule LHS must be two agents");
    Rule rule;
    std::map<std::string, int> vars;
    std::vector<int> occ;
    auto lhs_side = [&](int n, std::vector<int>& out) {
      for (int k : pool[n].kids) {
        if (!pool[k].is_name) throw std::runtime_error("PARSE: rule LHS ports must be names");
        if (vars.count(pool[k].id)) throw std::runtime_error("LINEARITY: LHS name repeated: " + pool[k].id);
        int v = (int)vars.size();
        vars[pool[k].id] = v;
        occ.push_back(0);
        out.push_back(v);
      }
    };
    rule.a = rs.sym.get(pool[l].id, (int)pool[l].kids.size());
    rule.b = rs.sym.get(pool[r].id, (int)pool[r].kids.size());
    lhs_side(l, rule.a_vars);
    lhs_side(r, rule.b_vars);
    int nlhs = (int)vars.size();
    if (!lx.accept(";")) {
      for (;;) {
        int x = parse_term(lx, pool);
        lx.expect("=");
        int y = parse_term(lx, pool);
        RTerm tx = to_rterm(pool, x, rs.sym, vars, occ);
        RTerm ty = to_rterm(pool, y, rs.sym, vars, occ);
        rule.rhs.emplace_back(std::move(tx), std::move(ty));
        if (lx.accept(";")) break;
        lx.expect(",");
      }
    }
    rule.nvars = (int)vars.size();
    rule.is_lhs.assign(rule.nvars, false);
    for (int v = 0; v < nlhs; v++) rule.is_lhs[v] = true;
    // Linearity (Sec. 2.2: names occur at most twice; a LHS name is bound by
    // the LHS, so it occurs exactly once in Theta; every other name of Theta
    // is bound inside Theta and occurs exactly twice there).
    for (auto& kv : vars) {
      int v = kv.second;
      int want = rule.is_lhs[v] ? 1 : 2;
      if (occ[v] != want)
        throw std::runtime_error("LINEARITY: name " + kv.first + " occurs " + std::to_string(occ[v]) +
                                 " times in the rule right-hand side, expected " + std::to_string(want));
    }
    for (auto& e : rule.rhs) rule.rhs_agents += count_agents(e.first) + count_agents(e.second);
    if (rule.a == rule.b) throw std::runtime_error("PARSE: rules between two agents of one symbol are not supported");
    int idx = (int)rs.rules.size();
    auto key = std::make_pair(rule.a, rule.b);
    if (rs.table.count(key) || rs.table.count({rule.b, rule.a}))
      throw std::runtime_error("PARSE: two rules for one active pair");
    rs.table[key] = idx * 2;
    rs.table[{rule.b, rule.a}] = idx * 2 + 1;
    rs.rules.push_back(std::move(rule));
  }
  return rs;
}

// ---------------------------------------------------------------------------
// A configuration < t.. | Delta > and the four reduction rules.

struct Result {
  std::string status = "ok";
  std::string text;              // canonical interface
  bool text_truncated = false;
  long long nat = -1;            // value when the interface is one numeral S^k(Z)
  uint64_t interactions = 0;
  std::vector<uint64_t> per_rule;
  long long live = 0, peak_live = 0;
  long long residual_eqs = 0, residual_agents = 0;
  std::vector<long long> rounds;       // active pairs per round ("rounds" mode)
  std::vector<long long> live_rounds;  // live agents after each round
  double seconds = 0;
};

struct Config {
  const RuleSet& rs;
  std::vector<Term*> iface;                    // interface t..
  struct Eq { Term* l; Term* r; bool alive; };
  std::vector<Eq> eqs;                         // Delta
  std::vector<int> free_eqs;
  // Top-level occurrences of each name: the (at most two) equations in which
  // it is a side.  Names are small integers; ids of names that have vanished
  // are reused for fresh names (the choice of fresh names is immaterial).
  std::vector<std::pair<int, int>> top;
  std::vector<int64_t> free_names;
  int64_t next_name = 0;
  std::vector<int> active;                     // equations alpha(..) = beta(..)
  std::vector<int64_t> com_work;               // names with two top-level equations
  std::vector<Term*> term_pool;                // recycled term nodes
  std::deque<Term> storage;
  long long live = 0, peak_live = 0;
  uint64_t interactions = 0;
  std::vector<uint64_t> per_rule;
  std::string mode = "lifo";
  std::mt19937_64 rng;
  bool eager = false;
  uint64_t max_interactions = ~0ull;

  explicit Config(const RuleSet& r) : rs(r), per_rule(r.rules.size(), 0) {}

  Term* new_term() {
    if (!term_pool.empty()) { Term* t = term_pool.back(); term_pool.pop_back(); *t = Term{}; return t; }
    storage.emplace_back();
    return &storage.back();
  }
  void free_term(Term* t) { term_pool.push_back(t); }
  int64_t fresh_name() {
    int64_t n;
    if (!free_names.empty()) { n = free_names.back(); free_names.pop_back(); }
    else n = next_name++;
    if ((size_t)n >= top.size()) top.resize((size_t)n + 1, {-1, -1});
    top[(size_t)n] = {-1, -1};
    return n;
  }
  static bool is_name(const Term* t) { return t->sym < 0; }

  void register_top(int64_t x, int e) {
    auto& slot = top[(size_t)x];
    if (slot.first < 0) slot.first = e;
    else if (slot.second < 0) { slot.second = e; com_work.push_back(x); }
    else throw std::runtime_error("LINEARITY: name occurs more than twice");
  }
  void unregister_top(int64_t x, int e) {
    auto& slot = top[(size_t)x];
    if (slot.first == e) { slot.first = slot.second; slot.second = -1; }
    else if (slot.second == e) slot.second = -1;
  }

  // Adds t = u to Delta.
  void add_eq(Term* l, Term* r) {
    int e;
    if (!free_eqs.empty()) { e = free_eqs.back(); free_eqs.pop_back(); eqs[(size_t)e] = {l, r, true}; }
    else { e = (int)eqs.size(); eqs.push_back({l, r, true}); }
    if (!is_name(l) && !is_name(r)) { active.push_back(e); return; }
    if (is_name(l)) register_top(l->name, e);
    if (is_name(r)) register_top(r->name, e);
  }
  void kill_eq(int e) {
    eqs[(size_t)e].alive = false;
    free_eqs.push_back(e);
  }

  // ->com (Sec. 2.2): < t | x = t, x = u, Delta > -> < t | t = u, Delta >.
  bool com(int64_t x) {
    auto slot = top[(size_t)x];
    int e1 = slot.first, e2 = slot.second;
    if (e1 < 0 || e2 < 0 || e1 == e2) return false;  // e1 == e2: x = x, a vicious circle
    auto other = [&](int e) -> Term* {
      Eq& q = eqs[(size_t)e];
      if (is_name(q.l) && q.l->name == x) return q.r;
      return q.l;
    };
    auto name_leaf = [&](int e) -> Term* {
      Eq& q = eqs[(size_t)e];
      if (is_name(q.l) && q.l->name == x) return q.l;
      return q.r;
    };
    Term* t = other(e1);
    Term* u = other(e2);
    Term* x1 = name_leaf(e1);
    Term* x2 = name_leaf(e2);
    if (is_name(t)) unregister_top(t->name, e1);
    if (is_name(u)) unregister_top(u->name, e2);
    top[(size_t)x] = {-1, -1};
    kill_eq(e1);
    kill_eq(e2);
    free_term(x1);
    free_term(x2);
    free_names.push_back(x);
    add_eq(t, u);
    return true;
  }

  // ->int (Sec. 2.2): replace alpha(t1..) = beta(t2..) by Theta', where the
  // bound names of Theta are renamed to fresh names and the LHS names are
  // replaced by the actual subterms t1.., t2...
  void interact(int e) {
    Term* l = eqs[(size_t)e].l;
    Term* r = eqs[(size_t)e].r;
    kill_eq(e);
    auto it = rs.table.find({l->sym, r->sym});
    if (it == rs.table.end())
      throw std::runtime_error("NO_RULE: no rule for " + rs.sym.names[(size_t)l->sym] + " = " +
                               rs.sym.names[(size_t)r->sym]);
    int ridx = it->second / 2;
    if (it->second & 1) std::swap(l, r);
    const Rule& rule = rs.rules[(size_t)ridx];
    std::vector<Term*> bind((size_t)rule.nvars, nullptr);   // LHS names -> subterms
    std::vector<int64_t> fresh((size_t)rule.nvars, -1);     // bound names -> fresh names
    for (size_t i = 0; i < rule.a_vars.size(); i++)
      bind[(size_t)rule.a_vars[i]] = l->arg[i];
    for (size_t i = 0; i < rule.b_vars.size(); i++) bind[(size_t)rule.b_vars[i]] = r->arg[i];
    for (int v = 0; v < rule.nvars; v++)
      if (!rule.is_lhs[(size_t)v]) fresh[(size_t)v] = fresh_name();
    std::vector<std::pair<Term*, Term*>> out;
    for (const auto& q : rule.rhs) out.emplace_back(inst(q.first, bind, fresh), inst(q.second, bind, fresh));
    free_term(l);
    free_term(r);
    live += rule.rhs_agents - 2;
    peak_live = std::max(peak_live, live);
    interactions++;
    per_rule[(size_t)ridx]++;
    for (auto& q : out) add_eq(q.first, q.second);
  }
  Term* inst(const RTerm& t, std::vector<Term*>& bind, const std::vector<int64_t>& fresh) {
    if (t.sym < 0) {
      if (bind[(size_t)t.var]) { Term* s = bind[(size_t)t.var]; bind[(size_t)t.var] = nullptr; return s; }
      Term* n = new_term();
      n->name = fresh[(size_t)t.var];
      return n;
    }
    Term* n = new_term();
    n->sym = t.sym;
    for (size_t k = 0; k < t.kids.size(); k++) n->arg[k] = inst(t.kids[k], bind, fresh);
    return n;
  }

  bool com_fixpoint() {
    bool any = false;
    while (!com_work.empty()) {
      int64_t x = com_work.back();
      com_work.pop_back();
      if (com(x)) any = true;
    }
    return any;
  }

  int pick_active() {
    size_t k;
    if (mode == "fifo") k = 0;
    else if (mode == "random") k = (size_t)(rng() % active.size());
    else k = active.size() - 1;
    int e = active[k];
    if (mode == "fifo") active.erase(active.begin());
    else { active[k] = active.back(); active.pop_back(); }
    return e;
  }

  void check_limit() {
    if (interactions >= max_interactions) throw std::runtime_error("STEP_LIMIT: interaction limit reached");
  }

  // Reduce with ->int and ->com until neither applies.
  void reduce(Result& res) {
    com_fixpoint();
    if (eager) collect_and_substitute();
    if (mode == "rounds") {
      while (!active.empty()) {
        std::vector<int> round;
        round.swap(active);
        res.rounds.push_back((long long)round.size());
        for (int e : round) { check_limit(); interact(e); }
        com_fixpoint();
        if (eager) collect_and_substitute();
        res.live_rounds.push_back(live);
      }
      return;
    }
    while (!active.empty() || !com_work.empty()) {
      if (!com_work.empty()) {
        int64_t x = com_work.back();
        com_work.pop_back();
        com(x);
      } else {
        check_limit();
        interact(pick_active());
      }
      if (eager) collect_and_substitute();
    }
  }

  // ->col and ->sub applied until neither applies (Sec. 2.2; Theorem 1 lets
  // them wait until the end).  col: an equation x = t with x in the interface
  // puts t in place of x there.  sub: an equation x = t with x inside a
  // non-variable side u of another equation puts t in place of x in u.
  // Implemented as a walk: every name leaf reached inside the interface (col)
  // or inside an agent of another equation (sub) whose name is a top-level
  // side of a live equation is replaced by that equation's other side, and
  // the equation is removed.
  void collect_and_substitute() {
    // leaf slot -> replace *slot by the other side of the defining equation
    auto try_replace = [&](Term** slot, int self_eq) -> bool {
      Term* leaf = *slot;
      if (!is_name(leaf)) return false;
      int64_t x = leaf->name;
      auto s = top[(size_t)x];
      int e = s.first >= 0 && s.first != self_eq ? s.first : (s.second >= 0 && s.second != self_eq ? s.second : -1);
      if (e < 0) return false;
      Eq& q = eqs[(size_t)e];
      if (!q.alive) return false;
      bool xl = is_name(q.l) && q.l->name == x;
      bool xr = is_name(q.r) && q.r->name == x;
      if (xl && xr) return false;  // x = x
      Term* t = xl ? q.r : q.l;
      Term* xleaf = xl ? q.l : q.r;
      if (is_name(t)) {
        unregister_top(t->name, e);
      }
      top[(size_t)x] = {-1, -1};
      kill_eq(e);
      free_term(xleaf);
      free_term(leaf);
      free_names.push_back(x);
      *slot = t;
      // t may now be a name that is a top-level side elsewhere: nothing to
      // register, since it now sits at a nested or interface position.
      return true;
    };
    // Walk from the interface (col), then from every other equation (sub).
    std::vector<Term**> stack;
    for (size_t i = 0; i < iface.size(); i++) stack.push_back(&iface[i]);
    auto drain = [&](int self_eq) {
      while (!stack.empty()) {
        Term** slot = stack.back();
        stack.pop_back();
        if (try_replace(slot, self_eq)) { stack.push_back(slot); continue; }
        Term* t = *slot;
        if (is_name(t)) continue;
        for (int k = 0; k < rs.sym.arity[(size_t)t->sym]; k++) stack.push_back(&t->arg[k]);
      }
    };
    drain(-1);
    bool changed = true;
    while (changed) {
      changed = false;
      for (size_t e = 0; e < eqs.size(); e++) {
        if (!eqs[e].alive) continue;
        // sub replaces a name nested inside an agent of this equation
        Eq& q = eqs[e];
        for (Term* side : {q.l, q.r}) {
          if (is_name(side)) continue;
          for (int k = 0; k < rs.sym.arity[(size_t)side->sym]; k++) stack.push_back(&side->arg[k]);
        }
        size_t before = free_eqs.size();
        drain((int)e);
        if (free_eqs.size() != before) changed = true;
      }
    }
  }

  // Canonical rendering: interface terms left to right, names renamed x0,
  // x1, .. in order of first occurrence.
  void render(Result& res, size_t max_chars) {
    std::unordered_map<int64_t, long long> canon;
    std::string out;
    bool trunc = false;
    std::vector<std::pair<Term*, int>> stack;  // (term, state) state -1 = close paren marker
    for (size_t i = 0; i < iface.size(); i++) {
      if (i) out += ", ";
      stack.push_back({iface[i], 0});
      while (!stack.empty()) {
        auto [t, st] = stack.back();
        stack.pop_back();
        if (out.size() > max_chars) { trunc = true; stack.clear(); break; }
        if (st == 1) { out += ")"; continue; }
        if (st == 2) { out += ", "; continue; }
        if (is_name(t)) {
          auto it = canon.find(t->name);
          long long c;
          if (it == canon.end()) { c = (long long)canon.size(); canon[t->name] = c; }
          else c = it->second;
          out += "x" + std::to_string(c);
          continue;
        }
        out += rs.sym.names[(size_t)t->sym];
        int ar = rs.sym.arity[(size_t)t->sym];
        if (ar == 0) continue;
        out += "(";
        stack.push_back({nullptr, 1});
        for (int k = ar - 1; k >= 0; k--) {
          stack.push_back({t->arg[k], 0});
          if (k) stack.push_back({nullptr, 2});
        }
      }
      if (trunc) break;
    }
    res.text = out;
    res.text_truncated = trunc;
    // numeral value: S^k(Z)
    res.nat = -1;
    if (iface.size() == 1) {
      long long k = 0;
      Term* t = iface[0];
      int S = -1, Z = -1;
      auto is = rs.sym.index.find("S");
      auto iz = rs.sym.index.find("Z");
      if (is != rs.sym.index.end()) S = is->second;
      if (iz != rs.sym.index.end()) Z = iz->second;
      while (!is_name(t) && t->sym == S && S >= 0) { k++; t = t->arg[0]; }
      if (!is_name(t) && t->sym == Z && Z >= 0) res.nat = k;
    }
  }

  long long count_residual_agents() {
    long long n = 0;
    std::vector<Term*> st;
    for (auto& q : eqs) {
      if (!q.alive) continue;
      st.push_back(q.l);
      st.push_back(q.r);
    }
    while (!st.empty()) {
      Term* t = st.back();
      st.pop_back();
      if (is_name(t)) continue;
      n++;
      for (int k = 0; k < rs.sym.arity[(size_t)t->sym]; k++) st.push_back(t->arg[k]);
    }
    return n;
  }
};

// Builds the configuration from parsed text and checks that every name occurs
// at most twice (Sec. 2.2, "Configurations").
void load_net(Config& c, const std::vector<PNode>& pool, const std::vector<int>& iface_roots,
              const std::vector<std::pair<int, int>>& eq_roots, const Symbols& sym) {
  std::map<std::string, int64_t> names;
  std::map<std::string, int> occ;
  long long agents = 0;
  auto build = [&](int root) -> Term* {
    // iterative construction
    Term* out = nullptr;
    std::vector<std::pair<int, Term**>> st;
    st.push_back({root, &out});
    while (!st.empty()) {
      auto [n, slot] = st.back();
      st.pop_back();
      const PNode& p = pool[(size_t)n];
      Term* t = c.new_term();
      *slot = t;
      if (p.is_name) {
        auto it = names.find(p.id);
        if (it == names.end()) {
          int64_t x = c.fresh_name();
          names[p.id] = x;
          t->name = x;
        } else t->name = it->second;
        if (++occ[p.id] > 2) throw std::runtime_error("LINEARITY: name " + p.id + " occurs more than twice");
        continue;
      }
      auto si = sym.index.find(p.id);
      if (si == sym.index.end()) throw std::runtime_error("PARSE: unknown agent symbol " + p.id);
      if (sym.arity[(size_t)si->second] != (int)p.kids.size())
        throw std::runtime_error("PARSE: wrong arity for " + p.id);
      if (p.kids.size() > (size_t)kMaxArity) throw std::runtime_error("PARSE: arity too large");
      t->sym = si->second;
      agents++;
      for (size_t k = 0; k < p.kids.size(); k++) st.push_back({p.kids[k], &t->arg[k]});
    }
    return out;
  };
  for (int r : iface_roots) c.iface.push_back(build(r));
  std::vector<std::pair<Term*, Term*>> eqs;
  for (auto& q : eq_roots) eqs.emplace_back(build(q.first), build(q.second));
  c.live = c.peak_live = agents;
  for (auto& q : eqs) c.add_eq(q.first, q.second);
}

struct NetText {
  std::vector<PNode> pool;
  std::vector<int> iface;
  std::vector<std::pair<int, int>> eqs;
};

std::vector<NetText> parse_nets(const std::string& text) {
  std::vector<NetText> out;
  Lexer lx(text);
  while (!lx.eof()) {
    NetText n;
    lx.expect("<");
    if (!lx.accept("|")) {
      for (;;) {
        n.iface.push_back(parse_term(lx, n.pool));
        if (lx.accept("|")) break;
        lx.expect(",");
      }
    }
    if (!lx.accept(">")) {
      for (;;) {
        int a = parse_term(lx, n.pool);
        lx.expect("=");
        int b = parse_term(lx, n.pool);
        n.eqs.emplace_back(a, b);
        if (lx.accept(">")) break;
        lx.expect(",");
      }
    }
    out.push_back(std::move(n));
  }
  return out;
}

struct Options {
  std::string mode = "lifo";
  uint64_t seed = 1;
  bool eager = false;
  int threads = 1;
  uint64_t max_interactions = ~0ull;
  size_t max_chars = (size_t)1 << 20;
  bool quiet = false;
};

Result run_one(const RuleSet& rs, const NetText& nt, const Options& o, uint64_t seed) {
  Result res;
  auto t0 = std::chrono::steady_clock::now();
  Config c(rs);
  c.mode = o.mode;
  c.rng.seed(seed);
  c.eager = o.eager;
  c.max_interactions = o.max_interactions;
  try {
    load_net(c, nt.pool, nt.iface, nt.eqs, rs.sym);  // nets use the rule set's symbols
    c.reduce(res);
    c.collect_and_substitute();
    c.render(res, o.max_chars);
  } catch (const std::exception& ex) {
    std::string m = ex.what();
    size_t colon = m.find(':');
    res.status = colon == std::string::npos ? "ERROR" : m.substr(0, colon);
    res.text = m;
  }
  res.interactions = c.interactions;
  res.per_rule = c.per_rule;
  res.live = c.live;
  res.peak_live = c.peak_live;
  if (res.status == "ok") {
    long long ne = 0;
    for (auto& q : c.eqs) ne += q.alive ? 1 : 0;
    res.residual_eqs = ne;
    res.residual_agents = c.count_residual_agents();
  }
  res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return res;
}

std::string json_escape(const std::string& s) {
  std::string o;
  for (char ch : s) {
    if (ch == '"' || ch == '\\') { o += '\\'; o += ch; }
    else if (ch == '\n') o += "\\n";
    else o += ch;
  }
  return o;
}

void print_result(size_t idx, const Result& r, bool quiet) {
  std::string s = "{\"net\": " + std::to_string(idx) + ", \"status\": \"" + r.status + "\"";
  if (!quiet || r.status != "ok") s += ", \"result\": \"" + json_escape(r.text) + "\"";
  s += ", \"truncated\": " + std::string(r.text_truncated ? "true" : "false");
  s += ", \"nat\": " + (r.nat >= 0 ? std::to_string(r.nat) : std::string("null"));
  s += ", \"interactions\": " + std::to_string(r.interactions);
  s += ", \"per_rule\": [";
  for (size_t i = 0; i < r.per_rule.size(); i++) s += (i ? ", " : "") + std::to_string(r.per_rule[i]);
  s += "], \"live\": " + std::to_string(r.live) + ", \"peak_live\": " + std::to_string(r.peak_live);
  s += ", \"residual_eqs\": " + std::to_string(r.residual_eqs) +
       ", \"residual_agents\": " + std::to_string(r.residual_agents);
  if (!r.rounds.empty() || !r.live_rounds.empty()) {
    s += ", \"rounds\": [";
    for (size_t i = 0; i < r.rounds.size(); i++) s += (i ? ", " : "") + std::to_string(r.rounds[i]);
    s += "], \"live_rounds\": [";
    for (size_t i = 0; i < r.live_rounds.size(); i++) s += (i ? ", " : "") + std::to_string(r.live_rounds[i]);
    s += "]";
  }
  char buf[64];
  snprintf(buf, sizeof buf, "%.6f", r.seconds);
  s += ", \"seconds\": " + std::string(buf) + "}";
  printf("%s\n", s.c_str());
}

std::string read_file(const char* path) {
  FILE* f = strcmp(path, "-") == 0 ? stdin : fopen(path, "rb");
  if (!f) throw std::runtime_error(std::string("cannot open ") + path);
  std::string s;
  char buf[1 << 16];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, n);
  if (f != stdin) fclose(f);
  return s;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 3) {
    fprintf(stderr, "usage: %s RULES NETS [--mode lifo|fifo|random|rounds] [--seed S] [--eager] "
                    "[--threads T] [--max-interactions N] [--max-result-chars N] [--quiet]\n", argv[0]);
    return 2;
  }
  Options o;
  for (int i = 3; i < argc; i++) {
    std::string a = argv[i];
    auto next = [&]() -> std::string {
      if (i + 1 >= argc) { fprintf(stderr, "missing value for %s\n", a.c_str()); exit(2); }
      return argv[++i];
    };
    if (a == "--mode") o.mode = next();
    else if (a == "--seed") o.seed = strtoull(next().c_str(), nullptr, 10);
    else if (a == "--eager") o.eager = true;
    else if (a == "--threads") o.threads = std::max(1, atoi(next().c_str()));
    else if (a == "--max-interactions") o.max_interactions = strtoull(next().c_str(), nullptr, 10);
    else if (a == "--max-result-chars") o.max_chars = (size_t)strtoull(next().c_str(), nullptr, 10);
    else if (a == "--quiet") o.quiet = true;
    else { fprintf(stderr, "unknown option %s\n", a.c_str()); return 2; }
  }
  if (o.mode != "lifo" && o.mode != "fifo" && o.mode != "random" && o.mode != "rounds") {
    fprintf(stderr, "bad mode %s\n", o.mode.c_str());
    return 2;
  }
  RuleSet rs;
  std::vector<NetText> nets;
  try {
    rs = parse_rules(read_file(argv[1]));
  } catch (const std::exception& ex) {
    std::string m = ex.what();
    size_t colon = m.find(':');
    printf("{\"rules\": \"%s\", \"message\": \"%s\"}\n",
           colon == std::string::npos ? "ERROR" : m.substr(0, colon).c_str(), json_escape(m).c_str());
    return 1;
  }
  try {
    nets = parse_nets(read_file(argv[2]));
  } catch (const std::exception& ex) {
    std::string m = ex.what();
    printf("{\"nets\": \"PARSE\", \"message\": \"%s\"}\n", json_escape(m).c_str());
    return 1;
  }
  std::vector<Result> results(nets.size());
  auto t0 = std::chrono::steady_clock::now();
  std::atomic<size_t> next{0};
  auto worker = [&]() {
    for (;;) {
      size_t i = next.fetch_add(1);
      if (i >= nets.size()) return;
      results[i] = run_one(rs, nets[i], o, o.seed + i);
    }
  };
  int nt = std::min<int>(o.threads, (int)std::max<size_t>(1, nets.size()));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; t++) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  uint64_t total = 0;
  for (size_t i = 0; i < results.size(); i++) {
    print_result(i, results[i], o.quiet);
    total += results[i].interactions;
  }
  fprintf(stderr, "{\"nets\": %zu, \"interactions\": %llu, \"seconds\": %.6f, \"threads\": %d}\n",
          nets.size(), (unsigned long long)total, secs, nt);
  return 0;
}
