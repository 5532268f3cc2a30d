// The paper's own loop form (Sec. 3.6, evaluate()): an interaction phase,
// then one communication phase, repeated until neither an interaction nor a
// communication happened.  The interaction phase is Sec. 3.4: the step
// kernel gives every active pair a fixed number n of result slots (n = the
// most equations any right-hand side has), writes the pair's name equations
// there instead of linking them and leaves the other slots as dummies
// (agent = agent equations are active pairs at once); the dummies are then
// removed by a stable stream compaction that appends the equations to the
// equation array.  The communication phase is Sec. 3.5: all name-headed
// equations are sorted by the name (stable LSD radix sort,
// inet_control.cuh) and adjacent equations x = t, x = s are folded into
// s = t, one ->com per name and pass.
// While this form runs, name bindings live in the equation array only: the
// bindings already in name slots are collected into it first, and what is
// left at the end is deposited back, so any loop form can continue.
#pragma once

#include "inet_control.cuh"
#include "inet_kernels.cuh"

namespace inet {

constexpr int kCpThreads = 256;
constexpr int kCpItems = 16;                     // consecutive slots per thread
constexpr int kCpTile = kCpThreads * kCpItems;   // 4096 slots per block

// Removal of the dummies (Sec. 3.4), step 1: non-dummy slots per tile.
__global__ void __launch_bounds__(kCpThreads) k_paper_compact_count(const unsigned long long* fix,
                                                                    unsigned long long m, uint32_t* counts) {
  __shared__ uint32_t wsum[kCpThreads / 32];
  const unsigned long long base = (unsigned long long)blockIdx.x * kCpTile + (unsigned long long)threadIdx.x * kCpItems;
  uint32_t c = 0;
  for (int r = 0; r < kCpItems; r++)
    if (base + r < m && fix[base + r]) c++;
  c = __reduce_add_sync(0xFFFFFFFFu, c);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kCpThreads / 32; w++) t += wsum[w];
    counts[blockIdx.x] = t;
  }
}

// Step 2 (after an exclusive scan of the tile counts): each tile writes its
// equations, in slot order, after the equations already in the array
// (*d.eq_n of them); the last tile leaves the total in *total.
__global__ void __launch_bounds__(kCpThreads) k_paper_compact_scatter(Dev d, const unsigned long long* fix,
                                                                      unsigned long long m, const uint32_t* offsets,
                                                                      uint32_t* total) {
  __shared__ uint32_t wsum[kCpThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned long long base = (unsigned long long)blockIdx.x * kCpTile + (unsigned long long)threadIdx.x * kCpItems;
  uint32_t c = 0;
  for (int r = 0; r < kCpItems; r++)
    if (base + r < m && fix[base + r]) c++;
  // exclusive prefix of c over the block: within the warp, then the warps
  uint32_t inc = c;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  uint32_t before = 0, all = 0;
  for (int w = 0; w < kCpThreads / 32; w++) {
    if (w < wid) before += wsum[w];
    all += wsum[w];
  }
  const uint32_t e0 = __ldcg(d.eq_n);
  uint32_t at = e0 + offsets[blockIdx.x] + before + inc - c;
  for (int r = 0; r < kCpItems; r++) {
    if (base + r >= m) break;
    const unsigned long long v = fix[base + r];
    if (!v) continue;
    if (at < d.cap_eq) d.eq[at] = v;
    else set_error(d.ctrl, INET_ERR_ARENA_FULL, 27);
    at++;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = offsets[blockIdx.x] + all;
}

// Step 3: the equation count grows by the compacted total.
__global__ void k_paper_compact_done(Dev d, const uint32_t* total) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *d.eq_n += *total;
}

// Before a paper-form reduction: every bound name slot becomes an equation
// x = value and the slot is cleared.
__global__ void k_paper_collect(Dev d, uint64_t n_vars) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n_vars) return;
  const uint32_t v = d.var[i];
  if (v == kEmpty) return;
  const uint32_t k = atomicAdd(d.eq_n, 1u);
  if (k < d.cap_eq) {
    d.eq[k] = (unsigned long long)mk_var((uint32_t)i) | ((unsigned long long)v << 32);
    d.var[i] = kEmpty;
  } else {
    set_error(d.ctrl, INET_ERR_ARENA_FULL, 20);
  }
}

// Before an interaction phase: the step kernel runs even when the previous
// step's frontier came out empty (a communication may have refilled it).
__global__ void k_paper_prep(Dev d) {
  Ctrl* c = d.ctrl;
  c->done = 0;
  c->hit_slice = 0;
  c->slice_t0 = 0;
  __threadfence();
}

// Communication, step 1: every equation name-first, keyed by the name.
__global__ void k_paper_orient(Dev d, uint32_t n, uint32_t* keys, unsigned long long* vals) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t t = (uint32_t)d.eq[i], u = (uint32_t)(d.eq[i] >> 32);
  if (!is_var(t)) {
    const uint32_t w = t;
    t = u;
    u = w;
  }
  keys[i] = is_var(t) ? idx_of(t) : 0xFFFFFFFFu;
  vals[i] = (unsigned long long)t | ((unsigned long long)u << 32);
}

// Communication, step 2 (after the sort): x = t, x = s become s = t (the
// functor of Sec. 3.5).  An agent pair joins the frontier of the next
// interaction phase (and its net's pending count); a name-headed result or
// an equation without a partner goes back to the equation array.  The name
// of a merged pair is done and returns to the free ring.
__global__ void k_paper_merge(Dev d, const uint32_t* keys, const unsigned long long* vals, uint32_t n,
                              uint32_t* merged) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys[i];
  if (i > 0 && keys[i - 1] == k) return;  // handled by the first of its group
  const bool two = i + 1 < n && keys[i + 1] == k && k != 0xFFFFFFFFu;
  Ctrl* c = d.ctrl;
  if (two && i + 2 < n && keys[i + 2] == k) set_error(c, INET_ERR_STATE, 21);  // a name seen three times
  uint32_t t, u;
  if (two) {
    t = (uint32_t)(vals[i + 1] >> 32);
    u = (uint32_t)(vals[i] >> 32);
    atomicAdd(merged, 1u);
    if (d.vown && k < d.cap_vars) __stcg(d.vown + k, kNoNet);
    const unsigned long long tp = atomicAdd(&c->v_tail, 1ull);
    __stcg(d.vfree + tp % d.cap_vars, k);
    if (is_agent(t) && is_agent(u)) {
      const uint32_t a = idx_of(t), b = idx_of(u);
      if (a >= d.cap_agents || b >= d.cap_agents) {
        set_error(c, INET_ERR_STATE, 22);
        return;
      }
      const uint32_t cur = ld_volatile(&c->step) & 1u;
      const uint32_t p = atomicAdd(&c->fcount[cur], 1u);
      if (p < d.cap_pairs) {
        d.front[cur][p] = Pair{a, b};
        const uint32_t net = (uint32_t)__ldcg(&d.node[a].head) >> 8;
        if (net < d.max_nets) atomicAdd(d.netctr + net, 1ull << kNetPairShift);
      } else {
        set_error(c, INET_ERR_ARENA_FULL, 23);
      }
      return;
    }
  } else {
    t = (uint32_t)vals[i];
    u = (uint32_t)(vals[i] >> 32);
  }
  const uint32_t o = atomicAdd(d.eq_n, 1u);
  if (o < d.cap_eq) d.eq[o] = (unsigned long long)t | ((unsigned long long)u << 32);
  else set_error(c, INET_ERR_ARENA_FULL, 24);
}

// After a paper-form reduction: each remaining equation x = t binds its
// name, as the first arrival of ->com would have left it.
__global__ void k_paper_deposit(Dev d, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t t = (uint32_t)d.eq[i], u = (uint32_t)(d.eq[i] >> 32);
  if (!is_var(t)) {
    const uint32_t w = t;
    t = u;
    u = w;
  }
  if (is_var(t) && idx_of(t) < d.cap_vars) d.var[idx_of(t)] = u;
  else set_error(d.ctrl, INET_ERR_STATE, 25);
}

}  // namespace inet
