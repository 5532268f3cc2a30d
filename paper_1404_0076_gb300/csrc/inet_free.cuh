// Per-net reclamation and placement into recycled slots.
//
// Nets are independent configurations (Sec. 2.2, Configurations): once a
// net is in normal form and its result has been read back (->col/->sub,
// Theorem 1), no other net can reach any of its agents or names, so every
// slot it still holds can go back to the free rings.  Ownership is read off
// the arena itself: an agent record carries its net in the head word (free
// slots carry kFreeHead), and the owner array holds the net of every name
// slot in use (kNoNet when free).  One scan over the slots in use frees the
// slots of a whole batch of nets.
//
// Newly loaded nets are uploaded above the bump pointers, as before, and
// then placed: the top part of the uploaded range moves into slots taken
// from the free rings, with every term word that points into the moved
// part rewritten, so the bump pointers advance only by what the rings could
// not supply.  All of this runs between reductions (stream-ordered), when
// every free slot is in a ring and no kernel holds one privately.
#pragma once

#include "inet_kernels.cuh"

namespace inet {

// Warp-aggregated push of `v` (lanes with `has`) onto a free ring.  Every
// lane of the warp must call it.
__device__ __forceinline__ uint32_t ring_push_warp(unsigned long long* tail, uint32_t* ring, unsigned long long cap,
                                                   bool has, uint32_t v) {
  const unsigned m = __ballot_sync(kFull, has);
  if (!m) return 0;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(tail, (unsigned long long)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  if (has) __stcg(ring + (base + __popc(m & lanemask_lt())) % cap, v);
  return (uint32_t)__popc(m);
}

// One block.  st[0] = 1 if some listed net is out of range or still has an
// active pair (then nothing is marked and the scan frees nothing); else the
// listed nets are marked.  st[1], st[2] = agents and names freed (counted
// by the scan).
__global__ void k_free_check(Dev d, const int32_t* ids, uint32_t n, uint8_t* mark, unsigned long long* st) {
  bool bad = false;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t id = ids[i];
    if (id < 0 || (uint32_t)id >= d.max_nets) bad = true;
    else if ((__ldcg(d.netctr + id) >> kNetPairShift) != 0) bad = true;
  }
  const int any = __syncthreads_or(bad ? 1 : 0);
  if (threadIdx.x == 0) {
    st[0] = any ? 1ull : 0ull;
    st[1] = 0;
    st[2] = 0;
  }
  if (any) return;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) mark[ids[i]] = 1;
}

// Every agent slot below n_agents whose head names a marked net, and every
// name slot below n_vars owned by one, is cleared and pushed to its ring.
// Warp-uniform loops (grid-stride by whole warps), so the pushes aggregate.
__global__ void k_free_scan(Dev d, uint32_t n_agents, uint32_t n_vars, const uint8_t* mark, unsigned long long* st) {
  if (st[0]) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  const uint32_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  uint32_t fa = 0, fv = 0;
  for (uint32_t i0 = w * 32; i0 < n_agents; i0 += warps * 32) {
    const uint32_t i = i0 + (uint32_t)lane;
    bool has = false;
    if (i < n_agents) {
      const int32_t h = __ldcg(&d.node[i].head);
      if (h != kFreeHead) {
        const uint32_t net = (uint32_t)h >> 8;
        has = net < d.max_nets && mark[net] != 0;
      }
      if (has) __stcg(&d.node[i].head, kFreeHead);
    }
    fa += ring_push_warp(&d.ctrl->a_tail, d.afree, d.cap_agents, has, i);
  }
  for (uint32_t x0 = w * 32; x0 < n_vars; x0 += warps * 32) {
    const uint32_t x = x0 + (uint32_t)lane;
    bool has = false;
    if (x < n_vars) {
      const uint32_t o = __ldcg(d.vown + x);
      has = o < d.max_nets && mark[o] != 0;
      if (has) {
        __stcg(d.var + x, kEmpty);
        __stcg(d.vown + x, kNoNet);
      }
    }
    fv += ring_push_warp(&d.ctrl->v_tail, d.vfree, d.cap_vars, has, x);
  }
  if (lane == 0) {
    if (fa) {
      atomicAdd(&st[1], (unsigned long long)fa);
      atomicAdd(reinterpret_cast<unsigned long long*>(&d.ctrl->live), (unsigned long long)(-(long long)fa));
    }
    if (fv) atomicAdd(&st[2], (unsigned long long)fv);
  }
}

// The freed nets' marks and counters are cleared; their ids count as
// reported, so inet_net_finished does not list them until they are reused.
__global__ void k_free_unmark(Dev d, const int32_t* ids, uint32_t n, uint8_t* mark, const unsigned long long* st) {
  if (st[0]) return;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t id = ids[i];
  mark[id] = 0;
  d.netctr[id] = 0;
  d.netstat[id] = 0;
  d.netrep[id] = 1;
  d.netlive[id] = 0;
  d.netquota[id] = 0;
}

// Per-net counters of newly uploaded nets whose ids are not one run:
// (id, counter, live agents), status, reported flag and quota cleared.
__global__ void k_net_ctr_scatter(Dev d, const int32_t* ids, const unsigned long long* ctr, const long long* live,
                                  uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t id = ids[i];
  if (id < 0 || (uint32_t)id >= d.max_nets) {
    set_error(d.ctrl, INET_ERR_STATE, 30);
    return;
  }
  d.netctr[id] = ctr[i];
  d.netstat[id] = 0;
  d.netrep[id] = 0;
  if (d.netlive) {
    d.netlive[id] = live[i];
    d.netquota[id] = 0;
  }
}

// netquota[ids[i]] = q[i].
__global__ void k_net_set_quota(Dev d, const int32_t* ids, const unsigned long long* q, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && ids[i] >= 0 && (uint32_t)ids[i] < d.max_nets) d.netquota[ids[i]] = q[i];
}

// Quotas, between launches: a net that still has active pairs and holds
// more live agents than its quota gets INET_ERR_ARENA_FULL as its status and
// is marked for k_quota_purge; *hit counts them.  Other nets are untouched.
__global__ void k_quota_check(Dev d, uint32_t n_nets, uint8_t* mark, unsigned long long* hit) {
  for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nets; n += gridDim.x * blockDim.x) {
    const unsigned long long q = d.netquota[n];
    if (!q || d.netlive[n] <= (long long)q || (d.netctr[n] >> kNetPairShift) == 0) continue;
    atomicCAS(d.netstat + n, 0, INET_ERR_ARENA_FULL);
    mark[n] = 1;
    atomicAdd(hit, 1ull);
  }
}

// One block: the frontier `cur` loses the pairs of marked nets (compacted in
// place, chunk by chunk: every write lands below the chunk being read), and
// those nets count no pending pair any more, so they are finished (with
// their error status) and can be freed.
__global__ void k_quota_purge(Dev d, uint8_t* mark, uint32_t n_nets, const unsigned long long* hit) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t kept;
  if (*hit == 0) return;  // no net went over its quota
  Ctrl* c = d.ctrl;
  const uint32_t cur = c->step & 1u;
  const uint32_t n = min(c->fcount[cur], d.cap_pairs);
  Pair* f = d.front[cur];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t wr = 0;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    Pair p{0, 0};
    bool keep = false;
    if (i < n) {
      p = f[i];
      keep = true;
      if (p.a < d.cap_agents) {
        const uint32_t net = (uint32_t)__ldcg(&d.node[p.a].head) >> 8;
        if (net < n_nets && mark[net]) keep = false;
      }
    }
    const unsigned m = __ballot_sync(kFull, keep);
    if (lane == 0) wsum[wid] = __popc(m);
    __syncthreads();  // every pair of the chunk has been read, the warp counts are there
    uint32_t before = 0;
    for (int w = 0; w < wid; w++) before += wsum[w];
    if (keep) f[wr + before + __popc(m & lanemask_lt())] = p;
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (int w = 0; w < nw; w++) t += wsum[w];
      kept = t;
    }
    __syncthreads();
    wr += kept;
    __syncthreads();
  }
  if (threadIdx.x == 0) c->fcount[cur] = wr;
  for (uint32_t k = threadIdx.x; k < n_nets; k += blockDim.x) {
    if (!mark[k]) continue;
    d.netctr[k] &= kNetIntMask;
    mark[k] = 0;
  }
}

// Placement, step 1 (one thread): publish both rings (between reductions
// every pushed entry is written) and take up to ta agent and tv name slots
// from them.
__global__ void k_place_prep(Dev d, uint32_t ta, uint32_t tv) {
  Ctrl* c = d.ctrl;
  if (c->a_head > c->a_pub) c->a_head = c->a_pub;
  c->a_pub = c->a_tail;
  if (c->v_head > c->v_pub) c->v_head = c->v_pub;
  c->v_pub = c->v_tail;
  c->place_ka = min((unsigned long long)ta, c->a_tail - c->a_head);
  c->place_kv = min((unsigned long long)tv, c->v_tail - c->v_head);
  c->place_ah = c->a_head % d.cap_agents;
  c->place_vh = c->v_head % d.cap_vars;
}

// The ring entry of the k-th slot taken (k < the number taken).
__device__ __forceinline__ uint32_t taken_slot(const uint32_t* ring, unsigned long long cap, unsigned long long h,
                                               uint32_t k) {
  unsigned long long p = h + k;
  if (p >= cap) p -= cap;
  return __ldcg(ring + p);
}

// Placement, step 2: uploaded agents [a0, a0 + ta) and names [v0, v0 + tv);
// the last place_ka agents and place_kv names move to the slots taken, and
// every word pointing at a moved element is rewritten.  A moved name's old
// slot is cleared (it lies above the new bump pointer, where a fresh name
// must find EMPTY).  Ring slots all lie below a0 / v0, so no thread writes
// what another reads.
__global__ void k_place(Dev d, uint32_t a0, uint32_t ta, uint32_t v0, uint32_t tv) {
  const Ctrl* c = d.ctrl;
  const uint32_t ka = (uint32_t)c->place_ka, kv = (uint32_t)c->place_kv;
  const unsigned long long ah = c->place_ah, vh = c->place_vh;
  const uint32_t amov = a0 + ta - ka, vmov = v0 + tv - kv;
  auto tr = [&](uint32_t w) -> uint32_t {
    if (is_agent(w)) {
      const uint32_t i = idx_of(w);
      if (i >= amov && i < a0 + ta) return mk_agent(taken_slot(d.afree, d.cap_agents, ah, i - amov));
    } else if (is_var(w)) {
      const uint32_t x = idx_of(w);
      if (x >= vmov && x < v0 + tv) return mk_var(taken_slot(d.vfree, d.cap_vars, vh, x - vmov));
    }
    return w;
  };
  const uint32_t n = max(ta, tv);
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    if (j < ta) {
      const uint32_t src = a0 + j;
      int4 r = ld_node(d.node + src);
      r.y = (int32_t)tr((uint32_t)r.y);
      r.z = (int32_t)tr((uint32_t)r.z);
      r.w = (int32_t)tr((uint32_t)r.w);
      const uint32_t dst = src >= amov ? taken_slot(d.afree, d.cap_agents, ah, src - amov) : src;
      if (dst >= a0 && dst != src) set_error(d.ctrl, INET_ERR_STATE, 31);
      else st_node(d.node + dst, r);
    }
    if (j < tv) {
      const uint32_t src = v0 + j;
      const uint32_t w = tr(__ldcg(d.var + src));
      const uint32_t dst = src >= vmov ? taken_slot(d.vfree, d.cap_vars, vh, src - vmov) : src;
      if (dst >= v0 && dst != src) {
        set_error(d.ctrl, INET_ERR_STATE, 32);
      } else {
        __stcg(d.var + dst, w);
        if (d.vown) __stcg(d.vown + dst, __ldcg(d.vown + src));
        if (dst != src) {
          __stcg(d.var + src, kEmpty);
          if (d.vown) __stcg(d.vown + src, kNoNet);
        }
      }
    }
  }
}

// Placement, step 3 (one thread): consume the ring entries taken and lower
// the bump pointers by as much.
__global__ void k_place_post(Dev d, uint32_t a0, uint32_t ta, uint32_t v0, uint32_t tv) {
  Ctrl* c = d.ctrl;
  c->a_head += c->place_ka;
  c->v_head += c->place_kv;
  c->a_bump = (unsigned long long)a0 + ta - c->place_ka;
  c->v_bump = (unsigned long long)v0 + tv - c->place_kv;
  __threadfence();
}

}  // namespace inet
