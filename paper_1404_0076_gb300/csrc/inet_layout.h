// Device data layout shared by host and device code of the evaluator.
//
// Term word (uint32): 0 = EMPTY, (i << 2) | 1 = AGENT i (the principal port
// of agent i), (i << 2) | 2 = VAR i (name slot i).  30-bit indexes.
//
// Agent record (16 bytes, one per slot): word 0 = label | net << 8, words
// 1..3 = the term words on auxiliary ports 1..3.  The principal port is not
// stored: it is a side of an equation, i.e. an entry of the frontier or the
// value of a name slot.  Every access to an agent reads or writes the whole
// record, so it is one 32-byte DRAM sector instead of one per field.
//
// Name slot (uint32): EMPTY while no equation "x = t" with x at the top level
// has been seen; otherwise the term t.  A name occurs at most twice (Sec.
// 2.2), so a slot sees at most two such arrivals; the second one performs
// ->com and frees the slot.
#pragma once

#include <cstdint>

namespace inet {

constexpr uint32_t kEmpty = 0;
constexpr uint32_t kTagAgent = 1;
constexpr uint32_t kTagVar = 2;

#ifdef __CUDACC__
#define INET_HD __host__ __device__ __forceinline__
#else
#define INET_HD inline
#endif

INET_HD uint32_t mk_agent(uint32_t i) { return (i << 2) | kTagAgent; }
INET_HD uint32_t mk_var(uint32_t i) { return (i << 2) | kTagVar; }
INET_HD uint32_t tag_of(uint32_t w) { return w & 3u; }
INET_HD uint32_t idx_of(uint32_t w) { return w >> 2; }
INET_HD bool is_agent(uint32_t w) { return (w & 3u) == kTagAgent; }
INET_HD bool is_var(uint32_t w) { return (w & 3u) == kTagVar; }

constexpr int kMaxArity = 3;
constexpr uint32_t kMaxIndex = (1u << 30) - 1;
constexpr uint32_t kMaxLabels = 64;   // rule table is kMaxLabels^2 int16 in shared memory
constexpr uint32_t kMaxNetSlots = (1u << 24) - 1;

// Head word of a free agent slot: label 0xFF and net 0xFFFFFF, neither of
// which a live agent can carry (labels < kMaxLabels, nets < kMaxNetSlots).
// Every path that frees an agent slot writes it, so a scan of the arena
// tells live agents (and their net) from free slots.
constexpr int32_t kFreeHead = -1;
// Owner word of a free name slot (the owner array holds the net of every
// name slot in use).
constexpr uint32_t kNoNet = 0xFFFFFFFFu;

struct alignas(16) Node {
  int32_t head;   // label | net << 8
  uint32_t aux[3];
};
static_assert(sizeof(Node) == 16, "agent record is 16 bytes");

struct alignas(8) Pair {
  uint32_t a, b;  // agent ids whose principal ports are connected
};

// Instantiation template of one rule (Sec. 2.2, ->int: Theta with bound
// names fresh and LHS names replaced by the actual arguments).  A "value
// code" names a term word known to the interacting thread:
//   0..2   the auxiliary ports of alpha (the LHS names x1..x3)
//   3..5   the auxiliary ports of beta (y1..y3)
//   6..13  AGENT(new agent j)
//   14..21 VAR(fresh name v)
//   0xFF   none
constexpr int kMaxNew = 8;
constexpr int kMaxFresh = 8;
constexpr int kMaxLink = 8;
constexpr int kValExt = 0;
constexpr int kValNew = 6;
constexpr int kValFresh = 14;
constexpr int kNumVals = 22;
constexpr uint8_t kValNone = 0xFF;

struct alignas(16) Template {
  uint8_t n_new;               // agents of Theta
  uint8_t n_fresh;             // names bound inside Theta that join two auxiliary ports
  uint8_t n_link;              // equations left to link after instantiation
  uint8_t rule;                // rule index (text order)
  uint8_t lab[kMaxNew];        // labels of the new agents
  uint8_t src[kMaxNew][3];     // value codes written to their auxiliary ports
  uint8_t link[kMaxLink][2];   // value codes of each equation t = u to link
  uint8_t lhs[2];              // labels of the left-hand side's agents (alpha, beta)
  uint8_t pad[10];
};
static_assert(sizeof(Template) == 64, "template is 64 bytes");

// Per-net counter: low 40 bits = interactions, high 24 bits = active pairs
// of the net in the frontier.  One 64-bit atomic add updates both.
constexpr int kNetPairShift = 40;
constexpr uint64_t kNetIntMask = (1ull << kNetPairShift) - 1;

}  // namespace inet
