// CPU check of the host readback: the parallel renderer read_net_text must
// give the same text, reached count and numeral as the sequential walk
// read_net, on random forests of terms laid out at random in an arena
// (agents reached directly or through chains of bound name slots, free
// names occurring twice, numerals), small and large.
#include <sys/wait.h>
#include <unistd.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "inet_text.h"

using namespace inet;

namespace {

struct Arena {
  std::vector<Node> nodes;
  std::vector<uint32_t> vars;
};

struct Gen {
  std::mt19937_64 rng;
  const CompiledRules& rules;
  Arena& A;
  std::vector<int> by_arity[4];
  std::vector<uint32_t> open_names;  // free names used once so far
  Gen(uint64_t seed, const CompiledRules& r, Arena& a) : rng(seed), rules(r), A(a) {
    for (int l = 0; l < r.n_labels(); l++) by_arity[r.arity[(size_t)l]].push_back(l);
  }
  uint32_t pick(uint32_t n) { return (uint32_t)(rng() % n); }
  // a word that leads to `w` through 0..3 bound name slots
  uint32_t wrap(uint32_t w) {
    const uint32_t hops = pick(4);
    for (uint32_t h = 0; h < hops; h++) {
      const uint32_t x = (uint32_t)A.vars.size();
      A.vars.push_back(w);
      w = mk_var(x);
    }
    return w;
  }
  uint32_t free_name() {
    if (!open_names.empty() && pick(2)) {
      const size_t i = pick((uint32_t)open_names.size());
      const uint32_t w = open_names[i];
      open_names.erase(open_names.begin() + (long)i);
      return w;
    }
    const uint32_t x = (uint32_t)A.vars.size();
    A.vars.push_back(kEmpty);
    open_names.push_back(mk_var(x));
    return mk_var(x);
  }
  // a random term of about `size` agents; returns its word
  uint32_t term(uint64_t size, int depth) {
    if (size == 0 || depth > 2000) return pick(8) == 0 ? free_name() : leaf();
    int ar = 1 + (int)pick(3);
    while (by_arity[ar].empty()) ar = 1 + (int)pick(3);
    const int lab = by_arity[ar][pick((uint32_t)by_arity[ar].size())];
    Node nd;
    nd.head = lab;
    nd.aux[0] = nd.aux[1] = nd.aux[2] = kEmpty;
    const uint32_t me = (uint32_t)A.nodes.size();
    A.nodes.push_back(nd);
    uint64_t left = size - 1;
    for (int k = 0; k < ar; k++) {
      const uint64_t part = k == ar - 1 ? left : (left ? rng() % (left + 1) : 0);
      left -= part;
      A.nodes[me].aux[k] = wrap(term(part, depth + 1));
    }
    return mk_agent(me);
  }
  uint32_t leaf() {
    const int lab = by_arity[0][pick((uint32_t)by_arity[0].size())];
    Node nd;
    nd.head = lab;
    nd.aux[0] = nd.aux[1] = nd.aux[2] = kEmpty;
    A.nodes.push_back(nd);
    return mk_agent((uint32_t)A.nodes.size() - 1);
  }
  uint32_t numeral(int s, int z, uint64_t k) {
    Node zn;
    zn.head = z;
    zn.aux[0] = zn.aux[1] = zn.aux[2] = kEmpty;
    A.nodes.push_back(zn);
    uint32_t w = mk_agent((uint32_t)A.nodes.size() - 1);
    for (uint64_t i = 0; i < k; i++) {
      Node sn;
      sn.head = s;
      sn.aux[0] = wrap(w);
      sn.aux[1] = sn.aux[2] = kEmpty;
      A.nodes.push_back(sn);
      w = mk_agent((uint32_t)A.nodes.size() - 1);
    }
    return w;
  }
};

// moves every agent and name slot to a random place, rewriting the words
void shuffle(Arena& A, std::vector<uint32_t>& iface, std::mt19937_64& rng) {
  std::vector<uint32_t> pa(A.nodes.size()), pv(A.vars.size());
  for (size_t i = 0; i < pa.size(); i++) pa[i] = (uint32_t)i;
  for (size_t i = 0; i < pv.size(); i++) pv[i] = (uint32_t)i;
  std::shuffle(pa.begin(), pa.end(), rng);
  std::shuffle(pv.begin(), pv.end(), rng);
  auto mv = [&](uint32_t w) {
    return is_agent(w) ? mk_agent(pa[idx_of(w)]) : is_var(w) ? mk_var(pv[idx_of(w)]) : w;
  };
  std::vector<Node> nodes(A.nodes.size());
  std::vector<uint32_t> vars(A.vars.size());
  for (size_t i = 0; i < A.nodes.size(); i++) {
    Node n = A.nodes[i];
    for (uint32_t& w : n.aux) w = mv(w);
    nodes[pa[i]] = n;
  }
  for (size_t i = 0; i < A.vars.size(); i++) vars[pv[i]] = mv(A.vars[i]);
  A.nodes.swap(nodes);
  A.vars.swap(vars);
  for (uint32_t& w : iface) w = mv(w);
}

}  // namespace

int main() {
  CompiledRules rules;
  std::string err;
  const std::string text =
      "Add(y, r) = Z -> r = y;\n"
      "Add(y, r) = S(x) -> Add(y, w) = x, r = S(w);\n"
      "T(a, b, c) = Z -> a = b, c = Z;\n"
      "Pred(r) = Z -> r = Z;\n";
  if (compile_rules(text, rules, err)) {
    std::printf("rules: %s\n", err.c_str());
    return 2;
  }
  const int s_lab = rules.index.at("S"), z_lab = rules.index.at("Z");
  int cases = 0, with_names = 0, large = 0;
  for (uint64_t seed = 1; seed <= 60; seed++) {
    std::mt19937_64 rng(seed * 7919);
    Arena A;
    Gen g(seed, rules, A);
    std::vector<uint32_t> iface;
    const int kind = (int)(seed % 4);
    const uint64_t big = seed % 10 == 0 ? 300000 : (seed % 3 == 0 ? 20000 : 40);
    if (kind == 3) {
      iface.push_back(g.wrap(g.numeral(s_lab, z_lab, big)));
    } else {
      const int roots = 1 + (int)g.pick(kind == 0 ? 1 : 5);
      for (int r = 0; r < roots; r++) iface.push_back(g.pick(10) == 0 ? g.free_name() : g.wrap(g.term(big, 0)));
      for (uint32_t w : g.open_names) iface.push_back(w);  // every free name twice
    }
    shuffle(A, iface, rng);
    Readback a, b;
    read_net(A.nodes.data(), A.nodes.size(), A.vars.data(), A.vars.size(), iface, rules, (size_t)-1 / 2, true, a);
    read_net_text(A.nodes.data(), A.nodes.size(), A.vars.data(), A.vars.size(), iface, rules, b);
    if (a.text != b.text || a.reached != b.reached || a.nat != b.nat || a.truncated != b.truncated) {
      std::printf("mismatch seed %llu: reached %lld/%lld nat %lld/%lld len %zu/%zu\n", (unsigned long long)seed,
                  (long long)a.reached, (long long)b.reached, (long long)a.nat, (long long)b.nat, a.text.size(),
                  b.text.size());
      return 1;
    }
    cases++;
    with_names += a.text.find('x') != std::string::npos ? 1 : 0;
    large += a.reached > 10000 ? 1 : 0;
  }
  // two renderers at once (the second finds the host pool busy and renders
  // on its own thread): both must still equal the sequential walk
  {
    Arena A1, A2;
    Gen g1(1001, rules, A1), g2(1002, rules, A2);
    std::vector<uint32_t> i1{g1.wrap(g1.term(200000, 0))}, i2{g2.wrap(g2.term(200000, 0))};
    for (uint32_t w : g1.open_names) i1.push_back(w);
    for (uint32_t w : g2.open_names) i2.push_back(w);
    Readback s1, s2, p1, p2;
    read_net(A1.nodes.data(), A1.nodes.size(), A1.vars.data(), A1.vars.size(), i1, rules, (size_t)-1 / 2, true, s1);
    read_net(A2.nodes.data(), A2.nodes.size(), A2.vars.data(), A2.vars.size(), i2, rules, (size_t)-1 / 2, true, s2);
    std::thread t([&] {
      read_net_text(A2.nodes.data(), A2.nodes.size(), A2.vars.data(), A2.vars.size(), i2, rules, p2);
    });
    read_net_text(A1.nodes.data(), A1.nodes.size(), A1.vars.data(), A1.vars.size(), i1, rules, p1);
    t.join();
    if (s1.text != p1.text || s2.text != p2.text || s1.reached != p1.reached || s2.reached != p2.reached) {
      std::printf("mismatch with two renderers at once\n");
      return 1;
    }
    cases++;
  }
  // a process forked after the pool started renders on its own thread and
  // exits normally
  {
    Arena A1;
    Gen g1(2001, rules, A1);
    std::vector<uint32_t> i1{g1.wrap(g1.term(50000, 0))};
    for (uint32_t w : g1.open_names) i1.push_back(w);
    Readback s1;
    read_net(A1.nodes.data(), A1.nodes.size(), A1.vars.data(), A1.vars.size(), i1, rules, (size_t)-1 / 2, true, s1);
    const pid_t pid = fork();
    if (pid == 0) {
      Readback p1;
      read_net_text(A1.nodes.data(), A1.nodes.size(), A1.vars.data(), A1.vars.size(), i1, rules, p1);
      std::exit(p1.text == s1.text ? 0 : 3);
    }
    int status = 0;
    if (pid < 0 || waitpid(pid, &status, 0) != pid || !WIFEXITED(status) || WEXITSTATUS(status) != 0) {
      std::printf("forked renderer failed\n");
      return 1;
    }
    cases++;
  }
  std::printf("ok %d cases, %d with free names, %d with more than 10000 agents\n", cases, with_names, large);
  return 0;
}
