// Numeral readback of many nets on the device (->col / ->sub of Theorem 1
// restricted to interfaces S^k(Z)).  A numeral is a linked list: each S
// agent's port leads, directly or through name slots, to the next agent.
// Walking it costs one dependent load per element, so one thread walking a
// long numeral is slow.  Here every net is first walked for a bounded
// number of agents; the nets whose walk did not reach its end are marked,
// one scan of the arena lists their agents (the net is in every agent
// record), each with its successor agent (name slots resolved on the way)
// and a weight (1 for an S agent), and pointer jumping (list ranking) runs
// over that list only: each round replaces successor and weight by those of
// the successor's successor, so ranks are known after ceil(log2 length)
// rounds.  An unfinished net reads the rank of the agent where its walk
// stopped.  Free slots may still carry a listed net in a stale record: they
// join the list, but no live list leads into them, and the rounds stop once
// every stopped walk's agent has reached Z (or a non-numeral agent).
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
  for (uint32_t hop = 0, vhops = 0;; hop++) {
    const uint32_t e = jump_slot(w, n_agents, n_vars);
    if (e == kJumpBad) break;
    if (e >= n_agents) {  // a name slot: follow it (not counted against the budget)
      if (++vhops > n_vars) break;
      w = __ldcg(d.var + (e - n_agents));
      continue;
    }
    if (hop >= budget) {
      res = nat_pending(k, e);
      atomicExch(&ctl[0], 1u);
      break;
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

// The nets of the walks that stopped are marked (mark[net] = 1).
__global__ void k_nat_mark(Dev d, const unsigned long long* vals, uint32_t n, uint32_t n_agents, uint8_t* mark) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !is_nat_pending(vals[i])) return;
  const uint32_t a = (uint32_t)vals[i];
  if (a >= n_agents) return;
  const uint32_t net = (uint32_t)__ldcg(&d.node[a].head) >> 8;
  if (net < d.max_nets) mark[net] = 1;
}

// The agent a word leads to through name slots, or kJumpBad.
__device__ __forceinline__ uint32_t nat_next(const Dev& d, uint32_t w, uint32_t n_agents, uint32_t n_vars) {
  for (uint32_t hop = 0; hop <= n_vars && is_var(w) && idx_of(w) < n_vars; hop++) {
    const uint32_t v = __ldcg(d.var + idx_of(w));
    if (v == kEmpty) return kJumpBad;
    w = v;
  }
  return is_agent(w) && idx_of(w) < n_agents ? idx_of(w) : kJumpBad;
}

// One scan of the agent slots: every agent of a marked net joins the list
// `lst` (*cnt of them) with (successor, weight) in buf.  Loops go by whole
// warps, so one atomic per warp appends.
__global__ void k_nat_list(Dev d, uint32_t n_agents, uint32_t n_vars, int s_label, int z_label, const uint8_t* mark,
                           const uint32_t* ctl, uint32_t* lst, uint32_t* cnt, uint2* buf) {
  if (!ctl[0]) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  const uint32_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  for (uint32_t a0 = w * 32; a0 < n_agents; a0 += warps * 32) {
    const uint32_t a = a0 + (uint32_t)lane;
    bool mine = false;
    int4 r = make_int4(0, 0, 0, 0);
    if (a < n_agents) {
      r = ld_node(d.node + a);
      const uint32_t net = (uint32_t)r.x >> 8;
      mine = r.x != kFreeHead && net < d.max_nets && mark[net] != 0;
    }
    const unsigned m = __ballot_sync(kFull, mine);
    if (!m) continue;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(cnt, (uint32_t)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (mine) {
      lst[base + __popc(m & lanemask_lt())] = a;
      const int lab = r.x & 0xFF;
      uint2 o = make_uint2(kJumpBad, 0u);
      if (lab == z_label) o.x = kJumpZ;
      else if (lab == s_label) o = make_uint2(nat_next(d, (uint32_t)r.y, n_agents, n_vars), 1u);
      buf[a] = o;
    }
  }
}

// Round r over the listed agents only: buffer r % 2 to the other.
// ctl[1] = rounds run; ctl[2 + r] is set by the check after round r when a
// stopped walk's agent is still short of its end, and round r + 1 runs
// only then.
__global__ void k_nat_lround(uint32_t n_agents, uint32_t r, uint32_t* ctl, const uint32_t* lst, const uint32_t* cnt,
                             uint2* buf0, uint2* buf1) {
  if (!ctl[0] || (r > 0 && !ctl[2 + r - 1])) return;
  const uint2* in = (r & 1u) ? buf1 : buf0;
  uint2* out = (r & 1u) ? buf0 : buf1;
  const uint32_t n = *cnt;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t a = lst[i];
    uint2 o = in[a];
    if (o.x < n_agents) {
      const uint2 q = in[o.x];
      o = make_uint2(q.x, o.y + q.y);
    }
    out[a] = o;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl[1] = r + 1;
}

// After round r: is any stopped walk's agent still short of its end?
__global__ void k_nat_jump_check(const unsigned long long* vals, uint32_t n, uint32_t n_agents, uint32_t r,
                                 uint32_t* ctl, const uint2* buf0, const uint2* buf1) {
  if (!ctl[0] || ctl[1] != r + 1) return;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long v = vals[i];
  if (!is_nat_pending(v)) return;
  const uint2* buf = ((r + 1) & 1u) ? buf1 : buf0;
  if ((uint32_t)v < n_agents && buf[(uint32_t)v].x < n_agents) atomicExch(&ctl[2 + r], 1u);
}

// The marks go (before the gather turns pending walks into values).
__global__ void k_nat_unmark(Dev d, const unsigned long long* vals, uint32_t n, uint32_t n_agents, uint8_t* mark) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !is_nat_pending(vals[i])) return;
  const uint32_t a = (uint32_t)vals[i];
  if (a >= n_agents) return;
  const uint32_t net = (uint32_t)__ldcg(&d.node[a].head) >> 8;
  if (net < d.max_nets) mark[net] = 0;
}

// Stopped walks add the rank of their agent, from the buffer the last
// round wrote.
__global__ void k_nat_jump_gather(unsigned long long* vals, uint32_t n, uint32_t n_agents, const uint32_t* ctl,
                                  const uint2* buf0, const uint2* buf1) {
  if (!ctl[0]) return;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long v = vals[i];
  if (!is_nat_pending(v)) return;
  if ((uint32_t)v >= n_agents) {
    vals[i] = kNatNone;
    return;
  }
  const uint2 q = ((ctl[1] & 1u) ? buf1 : buf0)[(uint32_t)v];
  vals[i] = q.x == kJumpZ ? ((v >> 32) & 0x3FFFFFFFull) + q.y : kNatNone;
}

}  // namespace inet
