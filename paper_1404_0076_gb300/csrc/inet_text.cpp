// Host side of the evaluator: tokenizer and parser of the text syntax, the
// rule compiler (Theta -> instantiation template), the net flattener and the
// readback walk.
#include "inet_text.h"

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cctype>
#include <cstring>
#include <string_view>
#include <unordered_map>

#include "host_pool.h"
#include "inet.h"

namespace inet {
namespace {

// ---------------------------------------------------------------------------
// Tokens: identifiers and the punctuation ( ) , = | < > ; and the arrow "->".

struct Tok {
  char kind;       // 'i' identifier, 'A' arrow, else the punctuation character
  uint32_t at, len;
};

bool tokenize(const std::string& s, std::vector<Tok>& toks, std::string& err) {
  size_t i = 0, n = s.size();
  while (i < n) {
    char c = s[i];
    if (c == '#') {
      while (i < n && s[i] != '\n') i++;
    } else if (isspace((unsigned char)c)) {
      i++;
    } else if (isalpha((unsigned char)c)) {
      size_t b = i++;
      while (i < n && (isalnum((unsigned char)s[i]) || s[i] == '_' || s[i] == '\'')) i++;
      toks.push_back({'i', (uint32_t)b, (uint32_t)(i - b)});
    } else if (c == '-' && i + 1 < n && s[i + 1] == '>') {
      toks.push_back({'A', (uint32_t)i, 2});
      i += 2;
    } else if (strchr("(),=|<>;", c)) {
      toks.push_back({c, (uint32_t)i, 1});
      i++;
    } else {
      err = "unexpected character '" + std::string(1, c) + "' at offset " + std::to_string(i);
      return false;
    }
  }
  return true;
}

// Syntax tree of one term, children as sibling lists.
struct Syn {
  uint32_t tok;
  bool name;
  int first = -1, last = -1, next = -1, nkids = 0;
};

struct Reader {
  const std::string& s;
  const std::vector<Tok>& t;
  size_t p = 0;
  std::string err;
  Reader(const std::string& src, const std::vector<Tok>& toks) : s(src), t(toks) {}
  bool at(char k) const { return p < t.size() && t[p].kind == k; }
  bool take(char k) {
    if (at(k)) { p++; return true; }
    return false;
  }
  bool need(char k, const char* what) {
    if (take(k)) return true;
    if (err.empty())
      err = std::string("expected ") + what + (p < t.size() ? " at offset " + std::to_string(t[p].at) : " at end");
    return false;
  }
  std::string text(uint32_t tok) const { return s.substr(t[tok].at, t[tok].len); }

  // Parses one term into `syn`; returns its index or -1.
  int term(std::vector<Syn>& syn) {
    std::vector<int> open;
    int root = -1;
    for (;;) {
      if (!at('i')) { need('i', "a term"); return -1; }
      int me = (int)syn.size();
      Syn node;
      node.tok = (uint32_t)p;
      node.name = islower((unsigned char)s[t[p].at]) != 0;
      syn.push_back(node);
      p++;
      if (open.empty()) root = me;
      else {
        Syn& par = syn[(size_t)open.back()];
        if (par.last < 0) par.first = me; else syn[(size_t)par.last].next = me;
        par.last = me;
        par.nkids++;
      }
      if (!syn[(size_t)me].name && take('(')) {
        if (!take(')')) { open.push_back(me); continue; }
      }
      for (;;) {
        if (open.empty()) return root;
        if (take(',')) break;
        if (!need(')', "')' or ','")) return -1;
        open.pop_back();
      }
    }
  }
};

std::vector<int> kids_of(const std::vector<Syn>& syn, int n) {
  std::vector<int> k;
  for (int c = syn[(size_t)n].first; c >= 0; c = syn[(size_t)c].next) k.push_back(c);
  return k;
}

// ---------------------------------------------------------------------------
// Rule compiler.  Theta is turned into a graph whose terminals are the ports
// of the new agents and the LHS names (the auxiliary ports of alpha and beta,
// i.e. the actual arguments t1.., t2.. of ->int); nesting, equations and
// names are edges through non-terminal nodes.  Contracting every path gives
// the wires of the right-hand side net:
//   P(j)-P(k)  a new active pair            -> link (NEW j, NEW k)
//   P(j)-X(k,p) principal into aux port      -> src[k][p] = NEW j  (->sub)
//   X(j,p)-X(k,q) two auxiliary ports        -> a fresh name slot v
//   X(j,p)-E(e) aux port to an argument      -> src[j][p] = EXT e (->sub)
//   P(j)-E(e), E(e)-E(f) equations with arguments -> link
struct RuleGraph {
  // node ids: terminals first: E(e) = e (0..5), then P/X of agent j at
  // 6 + 4j + port; non-terminal name occurrences after all terminals.
  std::vector<std::vector<int>> adj;
  int add() { adj.emplace_back(); return (int)adj.size() - 1; }
  void edge(int a, int b) { adj[(size_t)a].push_back(b); adj[(size_t)b].push_back(a); }
};

int compile_one(const std::string& src, const std::vector<Tok>& toks, Reader& rd,
                CompiledRules& out, std::string& err) {
  std::vector<Syn> syn;
  int la = rd.term(syn);
  if (la < 0 || !rd.need('=', "'='")) { err = rd.err; return INET_ERR_PARSE; }
  int lb = rd.term(syn);
  if (lb < 0 || !rd.need('A', "'->'")) { err = rd.err; return INET_ERR_PARSE; }
  std::vector<std::pair<int, int>> eqs;
  if (!rd.take(';')) {
    for (;;) {
      int x = rd.term(syn);
      if (x < 0 || !rd.need('=', "'='")) { err = rd.err; return INET_ERR_PARSE; }
      int y = rd.term(syn);
      if (y < 0) { err = rd.err; return INET_ERR_PARSE; }
      eqs.emplace_back(x, y);
      if (rd.take(';')) break;
      if (!rd.need(',', "',' or ';'")) { err = rd.err; return INET_ERR_PARSE; }
    }
  }
  (void)toks;
  auto label = [&](int n, int* lab_out) -> int {
    std::string id = rd.text(syn[(size_t)n].tok);
    int ar = syn[(size_t)n].nkids;
    if (ar > kMaxArity) { err = "symbol " + id + " has arity " + std::to_string(ar) + " > 3"; return INET_ERR_PARSE; }
    auto it = out.index.find(id);
    if (it == out.index.end()) {
      if (out.labels.size() >= kMaxLabels) { err = "more than 64 agent symbols"; return INET_ERR_PARSE; }
      int l = (int)out.labels.size();
      out.labels.push_back(id);
      out.arity.push_back(ar);
      out.index[id] = l;
      *lab_out = l;
      return 0;
    }
    if (out.arity[(size_t)it->second] != ar) { err = "symbol " + id + " used with two arities"; return INET_ERR_PARSE; }
    *lab_out = it->second;
    return 0;
  };
  if (syn[(size_t)la].name || syn[(size_t)lb].name) { err = "a rule's left-hand side is two agents"; return INET_ERR_PARSE; }
  int a, b, rc;
  if ((rc = label(la, &a)) || (rc = label(lb, &b))) return rc;
  if (a == b) { err = "rules between two agents of one symbol are not supported"; return INET_ERR_PARSE; }
  // LHS names -> external endpoints
  std::unordered_map<std::string, int> lhs;
  int side = 0;
  for (int root : {la, lb}) {
    int port = 0;
    for (int k : kids_of(syn, root)) {
      if (!syn[(size_t)k].name) { err = "a rule's left-hand side ports must be names"; return INET_ERR_PARSE; }
      std::string id = rd.text(syn[(size_t)k].tok);
      if (lhs.count(id)) { err = "name " + id + " repeated in a rule's left-hand side"; return INET_ERR_LINEARITY; }
      lhs[id] = side * 3 + port++;
    }
    side++;
  }
  // agents of Theta in pre-order
  RuleGraph g;
  for (int e = 0; e < 6; e++) g.add();
  std::vector<int> agent_of_syn(syn.size(), -1);
  std::vector<int> labs;
  for (auto& q : eqs) {
    for (int root : {q.first, q.second}) {
      std::vector<int> st{root};
      while (!st.empty()) {
        int n = st.back();
        st.pop_back();
        if (syn[(size_t)n].name) continue;
        int l;
        if ((rc = label(n, &l))) return rc;
        agent_of_syn[(size_t)n] = (int)labs.size();
        labs.push_back(l);
        std::vector<int> k = kids_of(syn, n);
        for (auto it = k.rbegin(); it != k.rend(); ++it) st.push_back(*it);
      }
    }
  }
  if ((int)labs.size() > kMaxNew) { err = "rule right-hand side has more than 8 agents"; return INET_ERR_PARSE; }
  for (size_t j = 0; j < labs.size(); j++)
    for (int p = 0; p < 4; p++) g.add();
  auto P = [&](int j) { return 6 + 4 * j; };
  auto X = [&](int j, int p) { return 6 + 4 * j + 1 + p; };
  int n_terminal = (int)g.adj.size();
  std::unordered_map<std::string, std::vector<int>> occ;  // name -> occurrence nodes
  // root endpoint of a term; creates occurrence nodes for names
  auto root_of = [&](int n) -> int {
    if (syn[(size_t)n].name) {
      int o = g.add();
      occ[rd.text(syn[(size_t)n].tok)].push_back(o);
      return o;
    }
    return P(agent_of_syn[(size_t)n]);
  };
  // nesting edges
  for (size_t n = 0; n < syn.size(); n++) {
    int j = agent_of_syn[n];
    if (j < 0) continue;
    int p = 0;
    for (int k : kids_of(syn, (int)n)) g.edge(X(j, p++), root_of(k));
  }
  for (auto& q : eqs) g.edge(root_of(q.first), root_of(q.second));
  // names: linearity (each LHS name once in Theta, every other name twice)
  for (auto& kv : occ) {
    auto it = lhs.find(kv.first);
    if (it != lhs.end()) {
      if (kv.second.size() != 1) { err = "name " + kv.first + " of the left-hand side occurs " + std::to_string(kv.second.size()) + " times in the right-hand side"; return INET_ERR_LINEARITY; }
      g.edge(kv.second[0], it->second);
    } else {
      if (kv.second.size() != 2) { err = "name " + kv.first + " bound in the right-hand side occurs " + std::to_string(kv.second.size()) + " times"; return INET_ERR_LINEARITY; }
      g.edge(kv.second[0], kv.second[1]);
    }
  }
  for (auto& kv : lhs)
    if (!occ.count(kv.first)) { err = "name " + kv.first + " of the left-hand side is missing from the right-hand side"; return INET_ERR_LINEARITY; }
  // contract paths between terminals
  Template t;
  memset(&t, 0, sizeof t);
  memset(t.src, kValNone, sizeof t.src);
  memset(t.link, kValNone, sizeof t.link);
  t.n_new = (uint8_t)labs.size();
  t.rule = (uint8_t)out.tmpl.size();
  for (size_t j = 0; j < labs.size(); j++) t.lab[j] = (uint8_t)labs[j];
  int ext_count[6] = {0, 0, 0, 0, 0, 0};
  std::vector<char> done((size_t)n_terminal, 0);
  int arity_a = out.arity[(size_t)a], arity_b = out.arity[(size_t)b];
  auto is_live_terminal = [&](int v) {
    if (v < 6) return (v < 3) ? v < arity_a : (v - 3) < arity_b;
    int j = (v - 6) / 4, port = (v - 6) % 4;
    return port == 0 || port - 1 < out.arity[(size_t)labs[(size_t)j]];
  };
  auto code_of = [&](int v) -> int {  // terminal -> value code of what the OTHER end writes/reads
    if (v < 6) return kValExt + v;
    return kValNew + (v - 6) / 4;     // principal of agent j
  };
  for (int v = 0; v < n_terminal; v++) {
    if (done[(size_t)v] || !is_live_terminal(v)) continue;
    if (g.adj[(size_t)v].size() != 1) { err = "internal: port without exactly one connection"; return INET_ERR_PARSE; }
    int prev = v, cur = g.adj[(size_t)v][0];
    int guard = 0;
    while (cur >= n_terminal) {
      auto& ad = g.adj[(size_t)cur];
      int nxt = ad[0] == prev ? ad[1] : ad[0];
      if (ad.size() != 2) { err = "internal: broken wire"; return INET_ERR_PARSE; }
      prev = cur;
      cur = nxt;
      if (++guard > 10000) { err = "internal: wire loop"; return INET_ERR_PARSE; }
    }
    int w = cur;
    done[(size_t)v] = done[(size_t)w] = 1;
    auto kind = [&](int u) -> char {  // 'E', 'P', 'X'
      if (u < 6) return 'E';
      return (u - 6) % 4 == 0 ? 'P' : 'X';
    };
    char kv = kind(v), kw = kind(w);
    if (kv == 'E') ext_count[v]++;
    if (kw == 'E') ext_count[w]++;
    if (kv == 'X' && kw == 'X') {
      if (t.n_fresh >= kMaxFresh) { err = "rule needs more than 8 fresh names"; return INET_ERR_PARSE; }
      int f = kValFresh + t.n_fresh++;
      t.src[(v - 6) / 4][(v - 6) % 4 - 1] = (uint8_t)f;
      t.src[(w - 6) / 4][(w - 6) % 4 - 1] = (uint8_t)f;
    } else if (kv == 'X' || kw == 'X') {
      int x = kv == 'X' ? v : w, o = kv == 'X' ? w : v;
      t.src[(x - 6) / 4][(x - 6) % 4 - 1] = (uint8_t)code_of(o);
    } else {
      if (t.n_link >= kMaxLink) { err = "rule has more than 8 equations to link"; return INET_ERR_PARSE; }
      t.link[t.n_link][0] = (uint8_t)code_of(v);
      t.link[t.n_link][1] = (uint8_t)code_of(w);
      t.n_link++;
    }
  }
  for (int e = 0; e < 6; e++)
    if (is_live_terminal(e) && ext_count[e] != 1) { err = "internal: argument not wired once"; return INET_ERR_PARSE; }
  int idx = (int)out.tmpl.size();
  int L = out.n_labels();
  if (idx >= 16000) { err = "too many rules"; return INET_ERR_PARSE; }
  // grow the table to L x L
  std::vector<int16_t> tab((size_t)L * L, -1);
  int oldL = 0;
  while ((size_t)oldL * oldL < out.table.size()) oldL++;
  for (int i = 0; i < oldL; i++)
    for (int j = 0; j < oldL; j++) tab[(size_t)i * L + j] = out.table[(size_t)i * oldL + j];
  if (tab[(size_t)a * L + b] >= 0) { err = "two rules for one active pair"; return INET_ERR_PARSE; }
  tab[(size_t)a * L + b] = (int16_t)(idx << 1);
  tab[(size_t)b * L + a] = (int16_t)((idx << 1) | 1);
  out.table.swap(tab);
  t.lhs[0] = (uint8_t)a;
  t.lhs[1] = (uint8_t)b;
  out.tmpl.push_back(t);
  out.rule_names.push_back(out.labels[(size_t)a] + "><" + out.labels[(size_t)b]);
  (void)src;
  return 0;
}

}  // namespace

int compile_rules(const std::string& text, CompiledRules& out, std::string& err) {
  out = CompiledRules();
  std::vector<Tok> toks;
  if (!tokenize(text, toks, err)) return INET_ERR_PARSE;
  Reader rd(text, toks);
  while (rd.p < toks.size()) {
    int rc = compile_one(text, toks, rd, out, err);
    if (rc) return rc;
    if ((int)out.tmpl.size() > INET_MAX_RULES) { err = "more than 64 rules"; return INET_ERR_PARSE; }
  }
  // table must be L x L even if the last symbols came after the last rule
  int L = out.n_labels();
  if (out.table.size() != (size_t)L * L) {
    int oldL = 0;
    while ((size_t)oldL * oldL < out.table.size()) oldL++;
    std::vector<int16_t> tab((size_t)L * L, -1);
    for (int i = 0; i < oldL; i++)
      for (int j = 0; j < oldL; j++) tab[(size_t)i * L + j] = out.table[(size_t)i * oldL + j];
    out.table.swap(tab);
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Net flattener.

// Label index of an agent symbol, or -1 (a rule set has at most
// kMaxLabels symbols, so a scan beats building a string for a map lookup).
static int label_of(const CompiledRules& rules, std::string_view id) {
  for (size_t i = 0; i < rules.labels.size(); i++) {
    const std::string& l = rules.labels[i];
    if (l.size() == id.size() && memcmp(l.data(), id.data(), id.size()) == 0) return (int)i;
  }
  return -1;
}

// One pass over the characters: agents are written as their terms are read
// (pre-order, left to right), names are numbered by first occurrence, and
// each equation is linked as soon as both sides are read.  The syntax is
// the tokenizer's: identifiers [A-Za-z][A-Za-z0-9_']*, a name when the
// first letter is lower-case, '#' comments to the end of the line.
namespace {

struct NetReader {
  const std::string& s;
  const CompiledRules& rules;
  uint32_t net_slot, agent_base, var_base;
  FlatNet& out;
  std::string& err;
  size_t p = 0;
  int rc = 0;
  std::unordered_map<std::string_view, uint32_t> slot;
  std::vector<uint8_t> count;
  struct Frame {
    uint32_t node;
    int port, arity;
  };
  std::vector<Frame> frames;

  bool fail(int code, const std::string& msg) {
    if (!rc) {
      rc = code;
      err = msg;
    }
    return false;
  }
  bool fail_at(const char* what) {
    return fail(INET_ERR_PARSE, std::string("expected ") + what +
                                    (p < s.size() ? " at offset " + std::to_string(p) : " at end"));
  }
  void skip() {
    while (p < s.size()) {
      const char c = s[p];
      if (c == '#') {
        while (p < s.size() && s[p] != '\n') p++;
      } else if (isspace((unsigned char)c)) {
        p++;
      } else {
        break;
      }
    }
  }
  // the next character after blanks, or 0 at the end
  char peek() {
    skip();
    return p < s.size() ? s[p] : '\0';
  }
  bool take(char c) {
    if (peek() != c) return false;
    p++;
    return true;
  }
  bool ident(std::string_view& id) {
    if (!isalpha((unsigned char)peek())) return false;
    const size_t b = p++;
    while (p < s.size() && (isalnum((unsigned char)s[p]) || s[p] == '_' || s[p] == '\'')) p++;
    id = std::string_view(s).substr(b, p - b);
    return true;
  }
  bool bad_char() {
    const char c = peek();
    if (c && !isalpha((unsigned char)c) && !strchr("(),=|<>;", c) && !(c == '-' && p + 1 < s.size() && s[p + 1] == '>'))
      return fail(INET_ERR_PARSE, "unexpected character '" + std::string(1, c) + "' at offset " + std::to_string(p));
    return true;
  }

  // One term; *w gets its word.
  bool term(uint32_t* w_out) {
    frames.clear();
    for (;;) {
      std::string_view id;
      if (!bad_char()) return false;
      if (!ident(id)) return fail_at("a term");
      uint32_t w;
      bool opened = false;
      uint32_t me = 0;
      int arity = 0;
      if (islower((unsigned char)id[0])) {
        auto it = slot.find(id);
        uint32_t v;
        if (it == slot.end()) {
          v = (uint32_t)count.size();
          slot.emplace(id, v);
          count.push_back(0);
          out.vars.push_back(kEmpty);
        } else {
          v = it->second;
        }
        if (++count[v] > 2) return fail(INET_ERR_LINEARITY, "name " + std::string(id) + " occurs more than twice");
        w = mk_var(var_base + v);
      } else {
        const int lab = label_of(rules, id);
        if (lab < 0) return fail(INET_ERR_PARSE, "unknown agent symbol " + std::string(id));
        arity = rules.arity[(size_t)lab];
        me = (uint32_t)out.nodes.size();
        Node nd;
        nd.head = (int32_t)((uint32_t)lab | (net_slot << 8));
        nd.aux[0] = nd.aux[1] = nd.aux[2] = kEmpty;
        out.nodes.push_back(nd);
        w = mk_agent(agent_base + me);
        if (take('(')) {
          if (!take(')')) opened = true;
          else if (arity != 0) return fail(INET_ERR_PARSE, "wrong arity for " + std::string(id));
        } else if (arity != 0) {
          return fail(INET_ERR_PARSE, "wrong arity for " + std::string(id));
        }
      }
      if (frames.empty()) {
        *w_out = w;
      } else {
        Frame& f = frames.back();
        if (f.port >= f.arity) return fail(INET_ERR_PARSE, "wrong arity for an agent at offset " + std::to_string(p));
        out.nodes[f.node].aux[f.port++] = w;
      }
      if (opened) {
        frames.push_back({me, 0, arity});
        continue;
      }
      for (;;) {
        if (frames.empty()) return true;
        if (take(',')) break;
        if (!bad_char()) return false;
        if (!take(')')) return fail_at("')' or ','");
        const Frame& f = frames.back();
        if (f.port != f.arity) return fail(INET_ERR_PARSE, "wrong arity for an agent before offset " + std::to_string(p));
        frames.pop_back();
      }
    }
  }

  // ->com on the staged slots: the second arrival takes the value
  bool link(uint32_t t, uint32_t u) {
    for (size_t guard = 0;; guard++) {
      if (guard > out.vars.size() + 2) return fail(INET_ERR_PARSE, "internal: link loop");
      if (is_agent(t) && is_agent(u)) {
        out.pairs.push_back({idx_of(t), idx_of(u)});
        return true;
      }
      if (!is_var(t)) std::swap(t, u);
      uint32_t& cell = out.vars[idx_of(t) - var_base];
      const uint32_t old = cell;
      cell = u;
      if (old == kEmpty) return true;
      cell = kEmpty;  // both top-level occurrences met: the slot is done
      t = old;
    }
  }

  bool net() {
    if (!bad_char()) return false;
    if (!take('<')) return fail_at("'<'");
    if (!take('|')) {
      for (;;) {
        uint32_t w = kEmpty;
        if (!term(&w)) return false;
        out.iface.push_back(w);
        if (take('|')) break;
        if (!bad_char()) return false;
        if (!take(',')) return fail_at("',' or '|'");
      }
    }
    if (!take('>')) {
      for (;;) {
        uint32_t t = kEmpty, u = kEmpty;
        if (!term(&t)) return false;
        if (!bad_char()) return false;
        if (!take('=')) return fail_at("'='");
        if (!term(&u)) return false;
        if (!link(t, u)) return false;
        if (take('>')) break;
        if (!bad_char()) return false;
        if (!take(',')) return fail_at("',' or '>'");
      }
    }
    if (!bad_char()) return false;
    if (peek()) return fail(INET_ERR_PARSE, "text after the end of the net");
    if ((uint64_t)var_base + out.vars.size() > kMaxIndex || (uint64_t)agent_base + out.nodes.size() > kMaxIndex)
      return fail(INET_ERR_ARENA_FULL, "net does not fit the index range");
    return true;
  }
};

}  // namespace

int flatten_net(const std::string& text, const CompiledRules& rules, uint32_t net_slot,
                uint32_t agent_base, uint32_t var_base, FlatNet& out, std::string& err) {
  out = FlatNet();
  NetReader rd{text, rules, net_slot, agent_base, var_base, out, err};
  if (!rd.net()) return rd.rc ? rd.rc : INET_ERR_PARSE;
  return 0;
}

// ---------------------------------------------------------------------------
// Readback walk.

// k when the interface is one numeral S^k(Z), else -1.
static int64_t numeral_of(const Node* nodes, uint64_t n_nodes, const uint32_t* vars, uint64_t n_vars,
                          const std::vector<uint32_t>& iface, const CompiledRules& rules) {
  auto si = rules.index.find("S");
  auto zi = rules.index.find("Z");
  if (iface.size() != 1 || si == rules.index.end() || zi == rules.index.end() ||
      rules.arity[(size_t)si->second] != 1 || rules.arity[(size_t)zi->second] != 0)
    return -1;
  auto resolve = [&](uint32_t w) -> uint32_t {
    uint64_t hops = 0;
    while (is_var(w) && idx_of(w) < n_vars && vars[idx_of(w)] != kEmpty && hops++ <= n_vars) w = vars[idx_of(w)];
    return w;
  };
  int64_t k = 0;
  uint32_t w = resolve(iface[0]);
  uint64_t guard = 0;
  while (is_agent(w) && idx_of(w) < n_nodes && (nodes[idx_of(w)].head & 0xFF) == si->second && guard++ < n_nodes) {
    k++;
    w = resolve(nodes[idx_of(w)].aux[0]);
  }
  return is_agent(w) && idx_of(w) < n_nodes && (nodes[idx_of(w)].head & 0xFF) == zi->second ? k : -1;
}

void read_net(const Node* nodes, uint64_t n_nodes, const uint32_t* vars, uint64_t n_vars,
              const std::vector<uint32_t>& iface, const CompiledRules& rules, size_t max_chars,
              bool want_text, Readback& out) {
  out = Readback();
  std::unordered_map<uint32_t, int64_t> canon;
  uint64_t budget = n_nodes + n_vars + 16;
  // follow name slots that hold a term (->col / ->sub)
  auto resolve = [&](uint32_t w) -> uint32_t {
    uint64_t hops = 0;
    while (is_var(w) && idx_of(w) < n_vars && vars[idx_of(w)] != kEmpty && hops++ <= n_vars) w = vars[idx_of(w)];
    return w;
  };
  // the walk visits agents in random order in a large snapshot: start the
  // load of a child's record when it is pushed, so that most of them have
  // arrived when it is popped
  auto prefetch = [&](uint32_t w) {
    if (is_agent(w) && idx_of(w) < n_nodes) __builtin_prefetch(nodes + idx_of(w));
    else if (is_var(w) && idx_of(w) < n_vars) __builtin_prefetch(vars + idx_of(w));
  };
  std::string& s = out.text;
  struct Item { uint32_t w; char emit; };  // emit != 0: literal ')' or ','
  for (size_t i = 0; i < iface.size(); i++) {
    if (i && want_text) s += ", ";
    std::vector<Item> st{{iface[i], 0}};
    while (!st.empty()) {
      Item it = st.back();
      st.pop_back();
      if (want_text && s.size() > max_chars) { out.truncated = true; want_text = false; }
      if (it.emit) {
        if (want_text) s += it.emit == ',' ? ", " : ")";
        continue;
      }
      if (budget-- == 0) { out.truncated = true; return; }
      uint32_t w = resolve(it.w);
      if (!is_agent(w)) {
        if (want_text) {
          auto c = canon.find(w);
          int64_t k;
          if (c == canon.end()) { k = (int64_t)canon.size(); canon.emplace(w, k); }
          else k = c->second;
          s += "x" + std::to_string(k);
        }
        continue;
      }
      uint32_t a = idx_of(w);
      if (a >= n_nodes) { out.truncated = true; continue; }
      out.reached++;
      int lab = nodes[a].head & 0xFF;
      int ar = lab < (int)rules.arity.size() ? rules.arity[(size_t)lab] : 0;
      if (want_text) s += lab < (int)rules.labels.size() ? rules.labels[(size_t)lab] : "?";
      if (ar == 0) continue;
      if (want_text) s += "(";
      st.push_back({0, ')'});
      // the children's name slots are read here, independently of each
      // other, and their records prefetched
      for (int k = ar - 1; k >= 0; k--) {
        const uint32_t cw = resolve(nodes[a].aux[k]);
        prefetch(cw);
        st.push_back({cw, 0});
        if (k) st.push_back({0, ','});
      }
    }
  }
  out.nat = numeral_of(nodes, n_nodes, vars, n_vars, iface, rules);
}

// Text readback of a large net in parallel.  The forest of interface terms
// is unfolded breadth-first from the roots until it has about 128 pending
// subterms (or nothing is left to unfold); the pending subterms are then
// rendered on the host pool, each by the depth-first walk of read_net, and
// the pieces joined in order.  Names are rendered as placeholders (the
// resolved word between two control bytes) and renamed x0, x1, .. in one
// pass over the joined text, in order of first occurrence, as read_net
// does, so the result is the same text.
void read_net_text(const Node* nodes, uint64_t n_nodes, const uint32_t* vars, uint64_t n_vars,
                   const std::vector<uint32_t>& iface, const CompiledRules& rules, Readback& out) {
  out = Readback();
  auto resolve = [&](uint32_t w) -> uint32_t {
    uint64_t hops = 0;
    while (is_var(w) && idx_of(w) < n_vars && vars[idx_of(w)] != kEmpty && hops++ <= n_vars) w = vars[idx_of(w)];
    return w;
  };
  auto label = [&](int lab) -> const std::string& {
    static const std::string unknown = "?";
    return lab < (int)rules.labels.size() ? rules.labels[(size_t)lab] : unknown;
  };
  auto arity = [&](int lab) { return lab < (int)rules.arity.size() ? rules.arity[(size_t)lab] : 0; };
  constexpr char kOpen = '\x01', kClose = '\x02';  // around a name's word, rendered later
  auto name_mark = [&](std::string& s, uint32_t w) {
    char buf[16];
    const int n = snprintf(buf, sizeof buf, "%c%08x%c", kOpen, w, kClose);
    s.append(buf, (size_t)n);
  };
  // pieces in text order: literal text, or a subterm still to render
  struct Piece {
    bool sub;
    uint32_t w;
    std::string text;
  };
  std::vector<Piece> pieces;
  for (size_t i = 0; i < iface.size(); i++) {
    if (i) pieces.push_back({false, 0, ", "});
    pieces.push_back({true, iface[i], std::string()});
  }
  std::atomic<int64_t> reached{0};
  std::atomic<bool> truncated{false}, exhausted{false};
  constexpr size_t kSubs = 128;
  for (int round = 0; round < 32; round++) {
    size_t subs = 0;
    for (const Piece& p : pieces) subs += p.sub ? 1 : 0;
    if (subs == 0 || subs >= kSubs) break;
    std::vector<Piece> next;
    next.reserve(pieces.size() * 2);
    for (Piece& p : pieces) {
      if (!p.sub) {
        next.push_back(std::move(p));
        continue;
      }
      const uint32_t w = resolve(p.w);
      if (!is_agent(w) || idx_of(w) >= n_nodes) {
        if (!is_agent(w)) {
          Piece t{false, 0, std::string()};
          name_mark(t.text, w);
          next.push_back(std::move(t));
        } else {
          truncated = true;
        }
        continue;
      }
      const Node& nd = nodes[idx_of(w)];
      reached++;
      const int lab = nd.head & 0xFF, ar = arity(lab);
      next.push_back({false, 0, label(lab) + (ar ? "(" : "")});
      for (int k = 0; k < ar; k++) {
        if (k) next.push_back({false, 0, ", "});
        next.push_back({true, nd.aux[k], std::string()});
      }
      if (ar) next.push_back({false, 0, ")"});
    }
    pieces.swap(next);
  }
  // render the pending subterms: the depth-first walk of read_net, names
  // as placeholders
  std::vector<size_t> todo;
  for (size_t i = 0; i < pieces.size(); i++)
    if (pieces[i].sub) todo.push_back(i);
  HostPool::get().run((int32_t)todo.size(), 1, [&](int32_t lo, int32_t hi) {
    struct Item { uint32_t w; char emit; };
    std::vector<Item> st;
    for (int32_t t = lo; t < hi; t++) {
      Piece& p = pieces[todo[(size_t)t]];
      std::string& s = p.text;
      int64_t got = 0;
      uint64_t budget = n_nodes + n_vars + 16;
      st.assign(1, Item{p.w, 0});
      while (!st.empty()) {
        const Item it = st.back();
        st.pop_back();
        if (it.emit) {
          s += it.emit == ',' ? ", " : ")";
          continue;
        }
        if (budget-- == 0) {
          truncated = true;
          exhausted = true;
          break;
        }
        const uint32_t w = resolve(it.w);
        if (!is_agent(w)) {
          name_mark(s, w);
          continue;
        }
        const uint32_t a = idx_of(w);
        if (a >= n_nodes) {
          truncated = true;
          continue;
        }
        got++;
        const int lab = nodes[a].head & 0xFF, ar = arity(lab);
        s += label(lab);
        if (ar == 0) continue;
        s += '(';
        st.push_back({0, ')'});
        for (int k = ar - 1; k >= 0; k--) {
          const uint32_t cw = resolve(nodes[a].aux[k]);
          if (is_agent(cw) && idx_of(cw) < n_nodes) __builtin_prefetch(nodes + idx_of(cw));
          st.push_back({cw, 0});
          if (k) st.push_back({0, ','});
        }
      }
      p.sub = false;
      reached += got;
    }
  });
  // join, renaming the names in order of first occurrence
  size_t total = 0;
  for (const Piece& p : pieces) total += p.text.size();
  std::string& s = out.text;
  s.reserve(total);
  std::unordered_map<uint32_t, int64_t> canon;
  for (const Piece& p : pieces) {
    const std::string& t = p.text;
    size_t i = 0;
    while (i < t.size()) {
      const size_t m = t.find(kOpen, i);
      if (m == std::string::npos) {
        s.append(t, i, std::string::npos);
        break;
      }
      s.append(t, i, m - i);
      const uint32_t w = (uint32_t)strtoul(t.substr(m + 1, 8).c_str(), nullptr, 16);
      auto c = canon.find(w);
      int64_t k;
      if (c == canon.end()) {
        k = (int64_t)canon.size();
        canon.emplace(w, k);
      } else {
        k = c->second;
      }
      s += "x" + std::to_string(k);
      i = m + 10;  // kOpen, 8 hex digits, kClose
    }
  }
  out.reached = reached;
  out.truncated = truncated;
  // (a walk that ran out of its budget leaves no numeral, as in read_net)
  out.nat = exhausted ? -1 : numeral_of(nodes, n_nodes, vars, n_vars, iface, rules);
}

}  // namespace inet
