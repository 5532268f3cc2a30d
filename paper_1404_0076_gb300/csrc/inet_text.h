// Host side of the evaluator: text front end, rule compiler, net flattener
// and readback walk.  Plain C++17; no CUDA.
#pragma once

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "inet_layout.h"

namespace inet {

struct CompiledRules {
  std::vector<std::string> labels;      // label index -> symbol
  std::vector<int> arity;               // label index -> arity (<= kMaxArity)
  std::map<std::string, int> index;     // symbol -> label index
  std::vector<int16_t> table;           // L*L: (template << 1) | flipped, or -1
  std::vector<Template> tmpl;           // one per rule, in text order
  std::vector<std::string> rule_names;  // "Alpha><Beta"
  int n_labels() const { return (int)labels.size(); }
};

// Parses and compiles a rule set.  Returns 0 or a negative inet status code;
// `err` gets a message.
int compile_rules(const std::string& text, CompiledRules& out, std::string& err);

// A net flattened into device records.  Agent ids start at agent_base and
// name slots at var_base; the caller owns those ranges.
struct FlatNet {
  std::vector<Node> nodes;              // agents [agent_base, agent_base + nodes.size())
  std::vector<uint32_t> vars;           // name slots [var_base, var_base + vars.size())
  std::vector<uint32_t> iface;          // interface term words
  std::vector<Pair> pairs;              // initial active pairs
};

// Parses and flattens one configuration < t.. | Delta >: nested terms become
// agent records, each name a slot, and the equations are linked (->com) on
// the staged slots.  Returns 0 or a negative inet status code.
int flatten_net(const std::string& text, const CompiledRules& rules, uint32_t net_slot,
                uint32_t agent_base, uint32_t var_base, FlatNet& out, std::string& err);

// Readback of one net from a host snapshot of the arena: walks the
// interface through name slots (->col / ->sub) and renders it with names
// renamed x0, x1, .. in order of first occurrence.  `reached` counts the
// agents visited.  `nat` gets k when the interface is one numeral S^k(Z),
// else -1.  Rendering stops after max_chars characters (truncated = true).
struct Readback {
  std::string text;
  bool truncated = false;
  int64_t nat = -1;
  int64_t reached = 0;
};
void read_net(const Node* nodes, uint64_t n_nodes, const uint32_t* vars, uint64_t n_vars,
              const std::vector<uint32_t>& iface, const CompiledRules& rules, size_t max_chars,
              bool want_text, Readback& out);
// The same text as read_net without a character limit, rendered on several
// host threads (for large normal forms).
void read_net_text(const Node* nodes, uint64_t n_nodes, const uint32_t* vars, uint64_t n_vars,
                   const std::vector<uint32_t>& iface, const CompiledRules& rules, Readback& out);

}  // namespace inet
