// Microbenchmark of the linker's memory primitive: 32-bit atomic exchanges
// that return the old value (->com on a name slot, Sec. 2.2), at random
// slots of an array of a given size.  It bounds the interaction rate from
// the side of the L2 atomic units, beside the HBM roofline: an interaction
// links a handful of equations, each one such exchange.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace inet {

// splitmix64 (Steele, Lea and Flood, 2014): a counter-based mixer of a
// 64-bit state, here the address stream of each thread.
__device__ __forceinline__ uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_bench_exch(uint32_t* slots, uint64_t n_slots, uint32_t ops_per_thread, uint64_t seed,
                             unsigned long long* sink) {
  uint64_t s = seed + (uint64_t)(blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) * 0x2545F4914F6CDD1Dull;
  uint32_t acc = 0;
  for (uint32_t i = 0; i < ops_per_thread; i++) {
    const uint64_t r = splitmix64(s);
    const uint64_t idx = __umul64hi(r, n_slots);  // uniform in [0, n_slots)
    acc ^= atomicExch(slots + idx, (uint32_t)r);
  }
  if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);  // keeps the returned values live
}

// Dependent memory round trips of one thread: the latency floor of a chain
// of interactions.  `rec` is a random cyclic permutation (rec[i].x = the
// next index, the other words padding: one 16-byte record per slot, like
// an agent record); xs[i] holds the same successor for the exchange
// variants and is consumed by them (at most one lap).
//   variant 0: i = rec[i].x                        (one record load per hop)
//   variant 1: j = exch(xs[i]); i = rec[j].x ^ rec[j].y (exchange, then the
//              record it leads to; .y is 0)
//   variant 2: store a record at wrk[i]; fence; j = exch(xs[i]); i = rec[j].x
//              (what one level of a chain of second arrivals needs: the new
//              record, the fence that publishes it, the exchange that finds
//              the waiting agent, and that agent's record)
__global__ void k_bench_chase(const int4* rec, uint32_t* xs, int4* wrk, uint32_t start, uint32_t hops, int variant,
                              unsigned long long* sink) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t i = start;
  if (variant == 0) {
    for (uint32_t h = 0; h < hops; h++) i = (uint32_t)__ldcg(rec + i).x;
  } else if (variant == 1) {
    for (uint32_t h = 0; h < hops; h++) {
      const uint32_t j = atomicExch(xs + i, 0u);
      const int4 r = __ldcg(rec + j);
      i = (uint32_t)(r.x ^ r.y);
    }
  } else {
    for (uint32_t h = 0; h < hops; h++) {
      __stcg(wrk + i, make_int4((int)h, (int)i, 0, 0));
      __threadfence();
      const uint32_t j = atomicExch(xs + i, 0u);
      i = (uint32_t)__ldcg(rec + j).x;
    }
  }
  sink[0] = i;
}

}  // namespace inet
