// Control for the paper's own communication phase (Sec. 3.5), measured on
// the same GPU against the atomic linker of this evaluator.
//
// Sec. 3.5 finds the equations x = t and x = s that share a name by sorting
// all name-headed equations by the name and folding adjacent equations with
// the same name into s = t (reduce_by_key with that predicate and functor);
// one pass resolves one ->com per name, so a chain A = x, x = y, y = B needs
// a pass per link (Sec. 3.6), and the loop repeats until nothing merges.
// Here: a stable LSD radix sort (8-bit digits) of (name, equation), a merge
// pass, repeated to the fixpoint.  The atomic linker resolves the same set
// in one launch: an exchange on each name slot, the second arrival
// continuing with the stored term (->com, Sec. 2.2).
#pragma once

#include <cstdint>

#include "inet_layout.h"

namespace inet {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;                       // elements per thread per tile
constexpr int kRsTile = kRsThreads * kRsItems;     // 4096
constexpr int kRsWarps = kRsThreads / 32;

// Histogram of digit (key >> shift) & 255 per tile: counts[digit * nblocks + block].
__global__ void __launch_bounds__(kRsThreads) k_rs_upsweep(const uint32_t* keys, uint32_t n, int shift,
                                                          uint32_t* counts) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t base = blockIdx.x * (uint32_t)kRsTile;
  for (int r = 0; r < kRsItems; r++) {
    const uint32_t i = base + (uint32_t)r * kRsThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of counts[0..m) in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* counts, uint32_t m) {
  __shared__ uint32_t part[1024];
  const uint32_t per = (m + 1023) / 1024;
  const uint32_t lo = threadIdx.x * per, hi = min(m, lo + per);
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; i++) s += counts[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (uint32_t o = 1; o < 1024; o <<= 1) {
    const uint32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - s;  // exclusive prefix of this chunk
  for (uint32_t i = lo; i < hi; i++) {
    const uint32_t c = counts[i];
    counts[i] = run;
    run += c;
  }
}

// Stable scatter of one digit pass.  A tile is taken in rounds of
// kRsThreads consecutive elements; within a round the rank of an element
// among equal digits is its rank in its warp (match) plus the counts of the
// earlier warps, plus what earlier rounds of the tile placed.
__global__ void __launch_bounds__(kRsThreads) k_rs_downsweep(const uint32_t* keys, const unsigned long long* vals,
                                                            uint32_t n, int shift, const uint32_t* offsets,
                                                            uint32_t* keys_out, unsigned long long* vals_out) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[kRsWarps][256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  run[threadIdx.x] = offsets[threadIdx.x * gridDim.x + blockIdx.x];
  const uint32_t base = blockIdx.x * (uint32_t)kRsTile;
  for (int r = 0; r < kRsItems; r++) {
    for (int w = 0; w < kRsWarps; w++) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const uint32_t i = base + (uint32_t)r * kRsThreads + threadIdx.x;
    const bool ok = i < n;
    const uint32_t k = ok ? keys[i] : 0u;
    const uint32_t dg = (k >> shift) & 255u;
    const unsigned vm = __ballot_sync(0xFFFFFFFFu, ok);
    uint32_t wrank = 0;
    if (ok) {
      const unsigned peers = __match_any_sync(vm, dg);
      wrank = (uint32_t)__popc(peers & ((1u << lane) - 1u));
      if (wrank == 0) wcnt[wid][dg] = (uint32_t)__popc(peers);
    }
    __syncthreads();
    // per digit: exclusive prefix over the warps, then advance the run
    {
      const uint32_t dgt = threadIdx.x;
      uint32_t s = run[dgt];
      for (int w = 0; w < kRsWarps; w++) {
        const uint32_t c = wcnt[w][dgt];
        wcnt[w][dgt] = s;
        s += c;
      }
      run[dgt] = s;
    }
    __syncthreads();
    if (ok) {
      const uint32_t dst = wcnt[wid][dg] + wrank;
      keys_out[dst] = k;
      vals_out[dst] = vals[i];
    }
    __syncthreads();
  }
}

// Orients each equation name-first (key = the name's index); agent = agent
// equations are active pairs already.
__global__ void k_ctl_orient(const unsigned long long* eq, uint32_t n, uint32_t* keys, unsigned long long* vals,
                             uint32_t* n_keep, uint2* pairs, uint32_t* n_pairs) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t t = (uint32_t)eq[i], u = (uint32_t)(eq[i] >> 32);
  if (is_agent(t) && is_agent(u)) {
    pairs[atomicAdd(n_pairs, 1u)] = make_uint2(idx_of(t), idx_of(u));
    return;
  }
  if (!is_var(t)) {
    const uint32_t w = t;
    t = u;
    u = w;
  }
  const uint32_t k = atomicAdd(n_keep, 1u);
  keys[k] = idx_of(t);
  vals[k] = (unsigned long long)t | ((unsigned long long)u << 32);
}

// One merge pass over name-sorted equations: two adjacent equations x = t,
// x = s become s = t (the functor of Sec. 3.5); a single one is kept.  The
// result is an active pair (two agents) or a name-headed equation for the
// next pass.  A name seen more than twice breaks linearity: *bad is set.
__global__ void k_ctl_merge(const uint32_t* keys, const unsigned long long* vals, uint32_t n, uint32_t* keys_out,
                            unsigned long long* vals_out, uint32_t* n_out, uint2* pairs, uint32_t* n_pairs,
                            uint32_t* merged, uint32_t* bad) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys[i];
  const bool first = i == 0 || keys[i - 1] != k;
  if (!first) return;  // handled by the first of its group
  const bool two = i + 1 < n && keys[i + 1] == k;
  if (two && i + 2 < n && keys[i + 2] == k) atomicExch(bad, 1u);
  uint32_t t, u;
  if (two) {
    // (x, t), (x, s) -> (s, t)
    t = (uint32_t)(vals[i + 1] >> 32);
    u = (uint32_t)(vals[i] >> 32);
    atomicAdd(merged, 1u);
    if (is_agent(t) && is_agent(u)) {
      pairs[atomicAdd(n_pairs, 1u)] = make_uint2(idx_of(t), idx_of(u));
      return;
    }
    if (!is_var(t)) {
      const uint32_t w = t;
      t = u;
      u = w;
    }
  } else {
    t = (uint32_t)vals[i];
    u = (uint32_t)(vals[i] >> 32);
  }
  const uint32_t o = atomicAdd(n_out, 1u);
  keys_out[o] = idx_of(t);
  vals_out[o] = (unsigned long long)t | ((unsigned long long)u << 32);
}

// The atomic linker on the same equations: one thread per equation, an
// exchange on the name slot; the second arrival continues with the stored
// term until it deposits or meets an agent (chains resolve in one launch).
__global__ void k_ctl_link_atomic(const unsigned long long* eq, uint32_t n, uint32_t* slots, uint32_t n_vars,
                                  uint2* pairs, uint32_t* n_pairs, uint32_t* bad) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t t = (uint32_t)eq[i], u = (uint32_t)(eq[i] >> 32);
  for (uint32_t guard = 0; guard <= n; guard++) {
    if (is_agent(t) && is_agent(u)) {
      pairs[atomicAdd(n_pairs, 1u)] = make_uint2(idx_of(t), idx_of(u));
      return;
    }
    if (!is_var(t)) {
      const uint32_t w = t;
      t = u;
      u = w;
    }
    if (!is_var(t) || idx_of(t) >= n_vars) {
      atomicExch(bad, 1u);
      return;
    }
    const uint32_t old = atomicExch(slots + idx_of(t), u);
    if (old == kEmpty) return;  // first arrival: deposited
    t = old;
  }
  atomicExch(bad, 1u);
}

// reduce_by_key with equality of adjacent keys and + (the example of
// Sec. 3.5): out holds the sum of every run of equal adjacent values.
__global__ void k_ctl_segsum(const int32_t* in, uint32_t n, int32_t* out, uint32_t* n_out, const uint32_t* rank) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i > 0 && in[i - 1] == in[i]) return;
  int32_t s = 0;
  uint32_t j = i;
  while (j < n && in[j] == in[i]) s += in[j++];
  out[rank[i]] = s;
  if (j == n) *n_out = rank[i] + 1;
}

// rank[i] = number of runs that start before i (serial; the example is tiny).
__global__ void k_ctl_runs(const int32_t* in, uint32_t n, uint32_t* rank) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  uint32_t r = 0;
  for (uint32_t i = 0; i < n; i++) {
    rank[i] = r;
    if (i + 1 >= n || in[i + 1] != in[i]) r++;
  }
}

}  // namespace inet
