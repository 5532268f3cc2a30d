// Numeral readback of many nets on the device (->col / ->sub of Theorem 1
// restricted to interfaces S^k(Z)).  A numeral is a linked list: each S
// agent's port leads, directly or through name slots, to the next agent.
// Walking it costs one dependent load per element, so one thread walking a
// long numeral is slow.  Here every net is first walked for a bounded
// number of elements; when some walk did not reach its end, every element
// of the arena is ranked by pointer jumping (list ranking): agent slots and
// name slots form one index space [0, n_agents) ++ [0, n_vars), each element
// points at its successor with a weight (1 for an S agent, 0 for a name
// slot), and each round replaces successor and weight by those of the
// successor's successor, so ranks are known after ceil(log2 length) rounds.
// An unfinished net reads the rank of the element where its walk stopped.
// Slots that are free still hold stale records: they join the ranking but no
// live list leads into them, and the rounds stop once every stopped walk's
// element has reached Z (or a non-numeral element), whatever stale chains do.
#pragma once

#include "inet_kernels.cuh"

namespace inet {

constexpr unsigned long long kNatNone = ~0ull;   // interface is not S^k(Z)
constexpr uint32_t kJumpZ = 0xFFFFFFFEu;         // successor: the list ends at Z
constexpr uint32_t kJumpBad = 0xFFFFFFFFu;       // successor: the list is not a numeral
constexpr int kJumpCtl = 64;                     // control words of one readback

// A walk that ran out of budget: top bits 10, the S agents passed (30 bits),
// the element where it stopped (32 bits).  Values and kNatNone never have
// these top bits.
__device__ __forceinline__ unsigned long long nat_pending(uint32_t k, uint32_t e) {
  return (2ull << 62) | ((unsigned long long)k << 32) | e;
}
__device__ __forceinline__ bool is_nat_pending(unsigned long long v) { return (v >> 62) == 2ull; }

// Index of the element a term word leads to, or kJumpBad.
__device__ __forceinline__ uint32_t jump_slot(uint32_t w, uint32_t n_agents, uint32_t n_vars) {
  if (is_agent(w)) return idx_of(w) < n_agents ? idx_of(w) : kJumpBad;
  if (is_var(w)) return idx_of(w) < n_vars ? n_agents + idx_of(w) : kJumpBad;
  return kJumpBad;
}

// One thread per net: from the interface word, at most `budget` elements.
// out[i] = the numeral, kNatNone, or nat_pending(...) with ctl[0] set.
__global__ void k_nat_walk(Dev d, const uint32_t* roots, uint32_t n, uint32_t n_agents, uint32_t n_vars,
                           int s_label, int z_label, uint32_t budget, unsigned long long* out, uint32_t* ctl) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long res = kNatNone;
  uint32_t w = roots[i], k = 0;
  for (uint32_t hop = 0;; hop++) {
    const uint32_t e = jump_slot(w, n_agents, n_vars);
    if (e == kJumpBad) break;
    if (hop == budget) {
      res = nat_pending(k, e);
      atomicExch(&ctl[0], 1u);
      break;
    }
    if (e >= n_agents) {
      w = __ldcg(d.var + (e - n_agents));
      continue;
    }
    const int4 r = ld_node(d.node + e);
    const int lab = r.x & 0xFF;
    if (lab == z_label) {
      res = k;
      break;
    }
    if (lab != s_label) break;
    k++;
    w = (uint32_t)r.y;
  }
  out[i] = res;
}

// Pointer jumping, set-up: successor and weight of every element.
__global__ void k_nat_jump_init(Dev d, uint32_t n_agents, uint32_t n_vars, int s_label, int z_label,
                                const uint32_t* ctl, uint2* buf) {
  if (!ctl[0]) return;
  const uint32_t n_slots = n_agents + n_vars;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += gridDim.x * blockDim.x) {
    uint2 o = make_uint2(kJumpBad, 0u);
    if (i < n_agents) {
      const int4 r = ld_node(d.node + i);
      const int lab = r.x & 0xFF;
      if (lab == z_label) o.x = kJumpZ;
      else if (lab == s_label) o = make_uint2(jump_slot((uint32_t)r.y, n_agents, n_vars), 1u);
    } else {
      o.x = jump_slot(__ldcg(d.var + (i - n_agents)), n_agents, n_vars);
    }
    buf[i] = o;
  }
}

// Round r: buffer r % 2 to the other.  ctl[1] = rounds run; ctl[2 + r] is
// set by the check after round r when a stopped walk is still unranked, and
// round r + 1 runs only then.
__global__ void k_nat_jump_round(uint32_t n_slots, uint32_t r, uint32_t* ctl, uint2* buf0, uint2* buf1) {
  if (!ctl[0] || (r > 0 && !ctl[2 + r - 1])) return;
  const uint2* in = (r & 1u) ? buf1 : buf0;
  uint2* out = (r & 1u) ? buf0 : buf1;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += gridDim.x * blockDim.x) {
    uint2 o = in[i];
    if (o.x < n_slots) {
      const uint2 q = in[o.x];
      o = make_uint2(q.x, o.y + q.y);
    }
    out[i] = o;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl[1] = r + 1;
}

// After round r: is any stopped walk's element still short of its end?
__global__ void k_nat_jump_check(const unsigned long long* vals, uint32_t n, uint32_t n_slots, uint32_t r,
                                 uint32_t* ctl, const uint2* buf0, const uint2* buf1) {
  if (!ctl[0] || ctl[1] != r + 1) return;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long v = vals[i];
  if (!is_nat_pending(v)) return;
  const uint2* buf = ((r + 1) & 1u) ? buf1 : buf0;
  if (buf[(uint32_t)v].x < n_slots) atomicExch(&ctl[2 + r], 1u);
}

// Stopped walks add the rank of their element, from the buffer the last
// round wrote.
__global__ void k_nat_jump_gather(unsigned long long* vals, uint32_t n, const uint32_t* ctl, const uint2* buf0,
                                  const uint2* buf1) {
  if (!ctl[0]) return;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long v = vals[i];
  if (!is_nat_pending(v)) return;
  const uint2 q = ((ctl[1] & 1u) ? buf1 : buf0)[(uint32_t)v];
  vals[i] = q.x == kJumpZ ? ((v >> 32) & 0x3FFFFFFFull) + q.y : kNatNone;
}

}  // namespace inet
