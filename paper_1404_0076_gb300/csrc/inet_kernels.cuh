// Device side of the evaluator: the data-parallel reduction step of Sec.
// 3.3-3.6 on an id-indexed arena (the representation proposed in Sec. 4.2,
// "A more efficient net representation"), with allocation by warp/block
// aggregated atomics (Sec. 4.2, "Remove result array merging", and the
// parallel-scan allocation cited there) instead of fixed-size results plus a
// filter pass (Sec. 3.4), and ->com resolved by atomic exchange on name
// slots, touching only the equations of the interacting pair (Sec. 4.2,
// "Improved communication") instead of a sort + reduce_by_key (Sec. 3.5).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "inet.h"
#include "inet_layout.h"

namespace inet {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kVarStage = 4;        // staged freed name slots per thread (overflow goes to the ring)
constexpr int kLocalPerThread = 2;  // block-local free-slot stack capacity per thread, per pool

// Control block.  Hot atomic counters sit on their own 128-byte lines.
struct Ctrl {
  // line 0: loop state; written by one thread at a time (finalizer or coordinator)
  uint32_t step;          // steps executed since the last reset; parity selects the frontier
  uint32_t done;          // 1 = loop finished
  int32_t error;          // first error (inet_status), 0 if none
  uint32_t error_info;    // net slot or detail
  uint32_t stop_step;     // absolute step at which the call stops (0xffffffff: never)
  uint32_t hit_limit;     // 1 if stop_step ended the call
  uint32_t trace_on;
  uint32_t call_step0;    // step at the start of the call
  int32_t fatal;          // first error that stops the loop (arena, state, timeout)
  uint32_t hit_slice;     // 1 if the launch's time slice ended it (the host relaunches)
  unsigned long long max_frontier;
  long long peak_live;
  unsigned long long slice_t0;  // globaltimer at the first step boundary of the launch
  uint32_t pad0[16];
  // line 1: frontier sizes (one atomic per block per step)
  alignas(128) uint32_t fcount[2];
  // pools
  alignas(128) unsigned long long a_head;
  alignas(128) unsigned long long a_tail;
  alignas(128) unsigned long long a_pub;    // ring entries below this are poppable
  unsigned long long v_pub;
  alignas(128) unsigned long long v_head;
  alignas(128) unsigned long long v_tail;
  alignas(128) unsigned long long a_bump;   // next never-used agent slot
  alignas(128) unsigned long long v_bump;   // next never-used name slot
  // persistent kernel: arrivals at the step barrier, and the published step
  // word (frontier size, generation, parity, done) that waiting blocks poll
  alignas(128) uint32_t bar_count;
  alignas(128) unsigned long long bar_word;
  alignas(128) uint32_t blocks_done;        // k_step: blocks finished this launch
  alignas(128) long long live;              // live agents, all nets
  // asynchronous kernel: ticket queue, pairs in flight, stop/quiesce/exit
  alignas(128) unsigned long long q_head;   // next ticket to claim (read together with q_tail)
  unsigned long long q_tail;                // next ticket to fill
  alignas(128) long long inflight;          // active pairs not yet reduced (queued or held)
  alignas(128) uint32_t astop;              // 1: stop taking work, drain, exit
  alignas(128) uint32_t quiesce;            // warps that stopped producing
  alignas(128) uint32_t aexit;              // pairs written back to the other frontier buffer
  uint32_t qinit;                           // queue sequence numbers initialised since the reset
  unsigned long long qdirty;                // cells [0, qdirty) may hold a previous launch's sequence
  // placement of newly loaded nets into recycled slots (k_place_*): slots
  // taken from each ring and the ring positions they start at
  unsigned long long place_ka, place_kv, place_ah, place_vh;
};

// Published step word of the persistent kernel.
__host__ __device__ inline unsigned long long pack_word(uint32_t n, uint32_t gen, uint32_t cur, uint32_t done) {
  return (unsigned long long)n | ((unsigned long long)(gen & 0xFFFFu) << 32) |
         ((unsigned long long)(cur & 1u) << 48) | ((unsigned long long)(done & 1u) << 49);
}
__host__ __device__ inline uint32_t word_n(unsigned long long w) { return (uint32_t)w; }
__host__ __device__ inline uint32_t word_gen(unsigned long long w) { return (uint32_t)(w >> 32) & 0xFFFFu; }
__host__ __device__ inline uint32_t word_cur(unsigned long long w) { return (uint32_t)(w >> 48) & 1u; }
__host__ __device__ inline uint32_t word_done(unsigned long long w) { return (uint32_t)(w >> 49) & 1u; }

struct Dev {
  Node* node;
  uint32_t* var;
  Pair* front[2];
  unsigned long long* qseq;  // asynchronous kernel: sequence number of each ticket queue cell
  uint32_t* afree;
  uint32_t* vfree;
  uint32_t* vown;        // net owning each name slot in use (kNoNet when free); NULL: owners not kept
  unsigned long long* netctr;
  int32_t* netstat;
  uint32_t* netrep;      // 1 once inet_net_finished reported the net
  long long* netlive;    // live agents of each net (kept with owner tracking only)
  unsigned long long* netquota;  // most live agents a net may hold (0: no limit; owner tracking only)
  uint32_t paper;        // the paper's loop form: name equations go to `eq_fix` instead of being linked
  unsigned long long* eq;  // equations t | u << 32 of the paper's form (communication phase)
  uint32_t* eq_n;
  uint32_t cap_eq;
  unsigned long long* eq_fix;  // interaction phase of the paper's form: eq_fix_n result slots per pair
  uint32_t eq_fix_n;
  unsigned long long cap_fix;
  unsigned long long* rule_hist;
  Ctrl* ctrl;
  const int16_t* table;
  const Template* tmpl;
  const uint8_t* arity;
  long long* trace_front;
  long long* trace_live;
  unsigned long long cap_agents, cap_vars;
  uint32_t cap_pairs, trace_cap;
  uint32_t n_labels, n_tmpl;
  uint32_t solo_max;   // persistent kernel: frontiers up to this size run on block 0 alone
  uint32_t max_nets;
  unsigned long long timeout_ns;
  unsigned long long slice_ns;   // a launch stops at the first step boundary after this
  cudaGraphConditionalHandle cond;
  int use_cond;
  uint32_t qcur;   // asynchronous kernel: frontier buffer used as the ticket queue
  uint32_t pad2;
  unsigned long long rules_key;  // hash of the templates (a rule-specialised kernel checks it)
};

// ---------------------------------------------------------------------------
// Memory helpers.  Arena reads bypass L1 (ld.global.cg): slots are rewritten
// by other SMs between steps and L1 is not coherent inside a persistent
// kernel.

__device__ __forceinline__ int4 ld_node(const Node* p) {
  return __ldcg(reinterpret_cast<const int4*>(p));
}
__device__ __forceinline__ void st_node(Node* p, int4 v) {
  __stcg(reinterpret_cast<int4*>(p), v);
}
__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ long long ld_volatile_s64(const long long* p) {
  return *reinterpret_cast<const volatile long long*>(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Records the first error.  Every code except INET_ERR_NO_RULE (which only
// stops its own net) is fatal and ends the loop at the next step boundary.
__device__ __forceinline__ void set_error(Ctrl* c, int32_t code, uint32_t info) {
  if (atomicCAS(reinterpret_cast<int*>(&c->error), 0, code) == 0) c->error_info = info;
  if (code != INET_ERR_NO_RULE) atomicCAS(reinterpret_cast<int*>(&c->fatal), 0, code);
}

// ---------------------------------------------------------------------------
// Shared memory of one block.

struct Smem {
  Template* tmpl;            // n_tmpl
  unsigned long long* warp;  // scan slots and 64-bit broadcast values
  Pair* push;                // kMaxLink * blockDim: staged new pairs (wide steps)
  uint32_t* vals;            // kNumVals * blockDim: per-thread value table
  uint32_t* vstage;          // kVarStage * blockDim: names freed during linking
  uint32_t* la;              // block-local stack of free agent slots
  uint32_t* lv;              // block-local stack of free name slots
  Pair* sf[2];               // solo frontier (persistent kernel, block 0)
  uint32_t* hist;            // INET_MAX_RULES
  int32_t* misc;             // counters and broadcast values
  int16_t* tab;              // n_labels^2
  uint8_t* arity;            // n_labels
};

enum {
  M_NPUSH = 0, M_NVSTAGE, M_FAIL, M_LAST, M_TIMEOUT, M_PBASE,
  M_LA, M_LA_BASE, M_LA_TAKE, M_LA_KEEP,   // agent stack: count, taken range, frees kept locally
  M_LV, M_LV_BASE, M_LV_TAKE, M_LV_KEEP, M_LV_FBASE,
  M_LIVE,                                  // live-agent delta not yet published
  M_SFN,                                   // pairs pushed into the next solo frontier
  M_STOP,                                  // solo loop: leave after this step
  M_NNEXT,
  M_COUNT
};
enum {
  W_TOTAL = 32,  // block_scan total
  W_ARING = 34, W_AAVAIL, W_ABUMP, W_VRING, W_VAVAIL, W_VBUMP, W_AFREE, W_VFREE, W_WORD,
  // coordinator state (block 0 of the persistent kernel)
  W_STEP, W_LIVE, W_PEAK, W_MAXF, W_APUB, W_VPUB, W_T0, W_STOP, W_TRACE, W_STEP0,
  W_LD0, W_LD1, W_LD2, W_LD3, W_LD4, W_LD5, W_LD6,
  W_SLOTS
};

__host__ __device__ inline size_t smem_bytes(uint32_t block, uint32_t n_labels, uint32_t n_tmpl, uint32_t solo_cap) {
  size_t b = 0;
  auto take = [&](size_t n, size_t align) { b = (b + align - 1) / align * align; b += n; };
  take(sizeof(Template) * (n_tmpl ? n_tmpl : 1), 16);
  take(sizeof(unsigned long long) * W_SLOTS, 16);
  take(sizeof(Pair) * kMaxLink * block, 16);
  take(sizeof(uint32_t) * kNumVals * block, 16);
  take(sizeof(uint32_t) * kVarStage * block, 16);
  take(sizeof(uint32_t) * kLocalPerThread * block, 16);
  take(sizeof(uint32_t) * kLocalPerThread * block, 16);
  take(sizeof(Pair) * kMaxLink * solo_cap, 16);
  take(sizeof(Pair) * kMaxLink * solo_cap, 16);
  take(sizeof(uint32_t) * INET_MAX_RULES, 16);
  take(sizeof(int32_t) * M_COUNT, 16);
  take(sizeof(int16_t) * n_labels * n_labels, 16);
  take(n_labels, 16);
  return b + 16;
}

__device__ __forceinline__ Smem carve(const Dev& d, uint32_t solo_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  size_t b = 0;
  auto take = [&](size_t n, size_t align) -> unsigned char* {
    b = (b + align - 1) / align * align;
    unsigned char* p = smem_raw + b;
    b += n;
    return p;
  };
  Smem s;
  const uint32_t B = blockDim.x;
  s.tmpl = reinterpret_cast<Template*>(take(sizeof(Template) * (d.n_tmpl ? d.n_tmpl : 1), 16));
  s.warp = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * W_SLOTS, 16));
  s.push = reinterpret_cast<Pair*>(take(sizeof(Pair) * kMaxLink * B, 16));
  s.vals = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * kNumVals * B, 16));
  s.vstage = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * kVarStage * B, 16));
  s.la = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * kLocalPerThread * B, 16));
  s.lv = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * kLocalPerThread * B, 16));
  s.sf[0] = reinterpret_cast<Pair*>(take(sizeof(Pair) * kMaxLink * solo_cap, 16));
  s.sf[1] = reinterpret_cast<Pair*>(take(sizeof(Pair) * kMaxLink * solo_cap, 16));
  s.hist = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * INET_MAX_RULES, 16));
  s.misc = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * M_COUNT, 16));
  s.tab = reinterpret_cast<int16_t*>(take(sizeof(int16_t) * d.n_labels * d.n_labels, 16));
  s.arity = reinterpret_cast<uint8_t*>(take(d.n_labels, 16));
  return s;
}

__device__ void load_tables(const Dev& d, const Smem& s) {
  const uint32_t nt = d.n_tmpl * (sizeof(Template) / 16);
  for (uint32_t i = threadIdx.x; i < nt; i += blockDim.x)
    reinterpret_cast<int4*>(s.tmpl)[i] = reinterpret_cast<const int4*>(d.tmpl)[i];
  for (uint32_t i = threadIdx.x; i < d.n_labels * d.n_labels; i += blockDim.x) s.tab[i] = d.table[i];
  for (uint32_t i = threadIdx.x; i < d.n_labels; i += blockDim.x) s.arity[i] = d.arity[i];
  for (uint32_t i = threadIdx.x; i < INET_MAX_RULES; i += blockDim.x) s.hist[i] = 0;
  for (uint32_t i = threadIdx.x; i < M_COUNT; i += blockDim.x) s.misc[i] = 0;
  __syncthreads();
}

__device__ void flush_hist(const Dev& d, const Smem& s) {
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < d.n_tmpl; i += blockDim.x) {
    uint32_t v = s.hist[i];
    if (v) {
      atomicAdd(&d.rule_hist[i], (unsigned long long)v);
      s.hist[i] = 0;
    }
  }
  __syncthreads();
}

// Publishes this block's live-agent delta (thread 0; fire and forget).
__device__ __forceinline__ void flush_live(const Dev& d, const Smem& s) {
  if (threadIdx.x == 0) {
    const int32_t v = s.misc[M_LIVE];
    if (v) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&d.ctrl->live), (unsigned long long)(long long)v);
      s.misc[M_LIVE] = 0;
    }
  }
}

// Block-wide exclusive scan of a packed 64-bit value (four 16-bit fields).
// Every thread gets its exclusive prefix; the block total is in s.warp[W_TOTAL].
__device__ __forceinline__ unsigned long long block_scan(unsigned long long v, const Smem& s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  unsigned long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long t = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s.warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    unsigned long long w = lane < nw ? s.warp[lane] : 0ull;
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long t = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) s.warp[lane] = wi - w;
    if (lane == nw - 1) s.warp[W_TOTAL] = wi;
  }
  __syncthreads();
  return s.warp[wid] + inc - v;
}

// ---------------------------------------------------------------------------
// Pools.  Each block keeps a stack of free slot ids of each kind in shared
// memory: slots freed by the block are handed out again by the block, with
// no global traffic.  Beyond that, a ring of freed slot ids per kind in
// global memory: pops only take entries published before the step (a_pub /
// v_pub), pushes append at the tail and the step bookkeeping publishes the
// tail between steps, so an entry is never read before it is written.  When
// the ring runs dry the bump pointer hands out never-used slots.  (A freed
// slot has no remaining reference: a consumed agent was only reachable
// through its active pair, and a name slot is freed after the second of its
// two arrivals.)

__device__ __forceinline__ bool pool_pop(unsigned long long* head, const unsigned long long* pub_p,
                                         unsigned long long* bump, unsigned long long cap,
                                         uint32_t k, unsigned long long* ring_base,
                                         uint32_t* ring_avail, unsigned long long* bump_base) {
  *ring_avail = 0;
  *ring_base = 0;
  *bump_base = 0;
  if (k == 0) return true;
  const unsigned long long pub = ld_volatile64(pub_p);
  unsigned long long h = atomicAdd(head, (unsigned long long)k);
  uint32_t avail = h < pub ? (uint32_t)min((unsigned long long)k, pub - h) : 0u;
  *ring_base = h % cap;  // reduced once here; pool_slot adds k < cap without dividing
  *ring_avail = avail;
  if (avail < k) {
    unsigned long long need = k - avail;
    unsigned long long b = atomicAdd(bump, need);
    *bump_base = b;
    if (b + need > cap) return false;
  }
  return true;
}

__device__ __forceinline__ uint32_t pool_slot(const uint32_t* ring, unsigned long long cap,
                                              unsigned long long ring_base, uint32_t ring_avail,
                                              unsigned long long bump_base, uint32_t k) {
  if (k < ring_avail) {
    unsigned long long p = ring_base + k;  // ring_base < cap and k < cap
    if (p >= cap) p -= cap;
    return __ldcg(ring + p);
  }
  return (uint32_t)(bump_base + (k - ring_avail));
}

// ->com on name slots (Sec. 2.2, Communication; Sec. 3.5-3.6).  Links the
// equation t = u.  Two agents form an active pair.  Otherwise the equation
// arrives at a name slot x (t or u a name): the first arrival stores its
// other side; the second finds the stored term s and continues with s = u,
// which resolves chains x1 = x2 = .. of any length in one call (the chains of
// Sec. 3.6 that need several passes of the sorting algorithm).  Returns true
// and the pair when an active pair results.
template <bool kTrack>
__device__ __forceinline__ bool link_eq(const Dev& d, const Smem& s, uint32_t t, uint32_t u, Pair* out,
                                        unsigned long long slot) {
  for (uint32_t guard = 0;; guard++) {
    if (is_agent(t) && is_agent(u)) {
      out->a = idx_of(t);
      out->b = idx_of(u);
      return true;
    }
    if (d.paper) {
      // the paper's form (Sec. 3.4): the equation goes to its result slot
      // and waits for the communication phase
      if (slot < d.cap_fix) d.eq_fix[slot] = (unsigned long long)t | ((unsigned long long)u << 32);
      else set_error(d.ctrl, INET_ERR_ARENA_FULL, 26);
      return false;
    }
    if (!is_var(t)) {
      uint32_t w = t;
      t = u;
      u = w;
    }
    if (!is_var(t) || guard > (1u << 24) || idx_of(t) >= d.cap_vars) {
      set_error(d.ctrl, INET_ERR_STATE, 1);  // corrupted word: record and skip the access
      return false;
    }
    const uint32_t x = idx_of(t);
    const uint32_t old = atomicExch(d.var + x, u);
    if (old == kEmpty) return false;
    // second arrival: the slot is finished; clear it and free it
    __stcg(d.var + x, kEmpty);
    if constexpr (kTrack) __stcg(d.vown + x, kNoNet);
    const int pos = atomicAdd(&s.misc[M_NVSTAGE], 1);
    if (pos < kVarStage * (int)blockDim.x) {
      s.vstage[pos] = x;
    } else {
      const unsigned long long tpos = atomicAdd(&d.ctrl->v_tail, 1ull);
      __stcg(d.vfree + tpos % d.cap_vars, x);
    }
    t = old;
  }
}

// One chunk of the frontier: pairs [base, base + blockDim.x) of frontier
// `cur` (n pairs), read from global memory or, for SOLO, from the block's
// shared solo frontier.  All threads of the block call it together.
// kTrack (contexts created with INET_ARENA_FREE_NETS): the owning net of
// every fresh name and the free mark of every agent slot freed are kept for
// inet_free_nets; the other instantiation carries none of that code.
template <bool SOLO, bool kTrack>
__device__ void process_chunk(const Dev& d, const Smem& s, uint32_t base, uint32_t n, uint32_t cur) {
  const uint32_t tid = threadIdx.x, B = blockDim.x;
  const int lane = tid & 31;
  const uint32_t capL = kLocalPerThread * B;
  Ctrl* c = d.ctrl;
  const uint32_t i = base + tid;
  bool valid = i < n;
  uint32_t a = 0, b = 0, net = 0, ti = 0;
  int4 ra = make_int4(0, 0, 0, 0), rb = ra;
  // a1: frontier read + dispatch through the (label, label) table
  if (valid) {
    if (SOLO) {
      const Pair p = s.sf[cur][i];
      a = p.a;
      b = p.b;
    } else {
      const unsigned long long pv = __ldcg(reinterpret_cast<const unsigned long long*>(d.front[cur] + i));
      a = (uint32_t)pv;
      b = (uint32_t)(pv >> 32);
    }
    if (a >= d.cap_agents || b >= d.cap_agents) {
      set_error(c, INET_ERR_STATE, 2);
      valid = false;
    }
  }
  if (valid) {
    ra = ld_node(d.node + a);
    rb = ld_node(d.node + b);
    uint32_t la = (uint32_t)ra.x & 0xFFu, lb = (uint32_t)rb.x & 0xFFu;
    int e = (la < d.n_labels && lb < d.n_labels) ? s.tab[la * d.n_labels + lb] : -1;
    net = (uint32_t)ra.x >> 8;
    if (net >= d.max_nets) {
      set_error(c, INET_ERR_STATE, 3);
      valid = false;
    } else if (e < 0) {
      valid = false;
      atomicCAS(d.netstat + net, 0, INET_ERR_NO_RULE);
      set_error(c, INET_ERR_NO_RULE, net);
      // the pair leaves the frontier without an interaction
      atomicAdd(d.netctr + net, (unsigned long long)(-(1ll << kNetPairShift)));
    } else {
      if (e & 1) {
        int4 t = ra; ra = rb; rb = t;
        uint32_t u = a; a = b; b = u;
      }
      ti = (uint32_t)e >> 1;
    }
  }
  const Template& T = s.tmpl[ti];
  const uint32_t n_new = valid ? T.n_new : 0u;
  const uint32_t n_fresh = valid ? T.n_fresh : 0u;
  // a3: allocation.  Consumed slots a and b are reused in place for the
  // first two new agents; the rest comes from the block's stacks, then the
  // global pools.
  const uint32_t need_a = n_new > 2 ? n_new - 2 : 0u;
  const uint32_t free_a = valid && n_new < 2 ? 2 - n_new : 0u;
  const unsigned long long packed = (unsigned long long)need_a | ((unsigned long long)n_fresh << 16) |
                                    ((unsigned long long)free_a << 32);
  const unsigned long long ex = block_scan(packed, s);
  if (tid == 0) {
    const unsigned long long tot = s.warp[W_TOTAL];
    const uint32_t Ka = (uint32_t)(tot & 0xFFFF), Kv = (uint32_t)((tot >> 16) & 0xFFFF);
    const uint32_t Fa = (uint32_t)((tot >> 32) & 0xFFFF);
    bool ok = true;
    unsigned long long rb0, bb0;
    uint32_t av0;
    // agents: take from the local stack, the rest from the global pool
    uint32_t la = (uint32_t)s.misc[M_LA];
    const uint32_t ta = min(la, Ka);
    la -= ta;
    s.misc[M_LA_BASE] = (int)la;
    s.misc[M_LA_TAKE] = (int)ta;
    ok = pool_pop(&c->a_head, &c->a_pub, &c->a_bump, d.cap_agents, Ka - ta, &rb0, &av0, &bb0) && ok;
    s.warp[W_ARING] = rb0;
    s.warp[W_AAVAIL] = av0;
    s.warp[W_ABUMP] = bb0;
    // agent frees go on the local stack where the taken entries were
    // (written after everyone has read them); the overflow goes to the ring
    const uint32_t keep = min(capL - la, Fa);
    s.misc[M_LA_KEEP] = (int)keep;
    s.misc[M_LA] = (int)(la + keep);
    s.warp[W_AFREE] = Fa > keep ? atomicAdd(&c->a_tail, (unsigned long long)(Fa - keep)) : 0ull;
    // names
    uint32_t lv = (uint32_t)s.misc[M_LV];
    const uint32_t tv = min(lv, Kv);
    lv -= tv;
    s.misc[M_LV_BASE] = (int)lv;
    s.misc[M_LV_TAKE] = (int)tv;
    s.misc[M_LV] = (int)lv;
    ok = pool_pop(&c->v_head, &c->v_pub, &c->v_bump, d.cap_vars, Kv - tv, &rb0, &av0, &bb0) && ok;
    s.warp[W_VRING] = rb0;
    s.warp[W_VAVAIL] = av0;
    s.warp[W_VBUMP] = bb0;
    s.misc[M_LIVE] += (int)Ka - (int)Fa;
    if (!ok) {
      set_error(c, INET_ERR_ARENA_FULL, 0);
      s.misc[M_FAIL] = 1;
    }
    s.misc[M_NPUSH] = 0;
    s.misc[M_NVSTAGE] = 0;
  }
  __syncthreads();
  if (s.misc[M_FAIL]) valid = false;
  // a2: instantiate Theta' (Sec. 2.2, Interaction)
  uint32_t* vals = s.vals + tid;
  uint32_t n_link = 0;
  if (valid) {
    const uint32_t oa = (uint32_t)(ex & 0xFFFF), ov = (uint32_t)((ex >> 16) & 0xFFFF);
    const uint32_t ta = (uint32_t)s.misc[M_LA_TAKE], la0 = (uint32_t)s.misc[M_LA_BASE];
    const uint32_t tv = (uint32_t)s.misc[M_LV_TAKE], lv0 = (uint32_t)s.misc[M_LV_BASE];
    vals[(kValExt + 0) * B] = (uint32_t)ra.y;
    vals[(kValExt + 1) * B] = (uint32_t)ra.z;
    vals[(kValExt + 2) * B] = (uint32_t)ra.w;
    vals[(kValExt + 3) * B] = (uint32_t)rb.y;
    vals[(kValExt + 4) * B] = (uint32_t)rb.z;
    vals[(kValExt + 5) * B] = (uint32_t)rb.w;
    bool in_range = true;
#pragma unroll
    for (int j = 0; j < kMaxNew; j++) {
      if ((uint32_t)j < n_new) {
        uint32_t sl;
        if (j == 0) {
          sl = a;
        } else if (j == 1) {
          sl = b;
        } else {
          const uint32_t k = oa + (uint32_t)j - 2;
          if (k < ta) sl = s.la[la0 + k];
          else sl = pool_slot(d.afree, d.cap_agents, s.warp[W_ARING], (uint32_t)s.warp[W_AAVAIL],
                              s.warp[W_ABUMP], k - ta);
          if (sl >= d.cap_agents) in_range = false;
        }
        vals[(kValNew + j) * B] = mk_agent(sl);
      }
    }
#pragma unroll
    for (int v = 0; v < kMaxFresh; v++) {
      if ((uint32_t)v < n_fresh) {
        const uint32_t k = ov + (uint32_t)v;
        uint32_t x;
        if (k < tv) x = s.lv[lv0 + k];
        else x = pool_slot(d.vfree, d.cap_vars, s.warp[W_VRING], (uint32_t)s.warp[W_VAVAIL], s.warp[W_VBUMP], k - tv);
        if (x >= d.cap_vars) in_range = false;
        else if constexpr (kTrack) __stcg(d.vown + x, net);  // the owner, before the name is published
        vals[(kValFresh + v) * B] = mk_var(x);
      }
    }
    if (!in_range) {
      set_error(c, INET_ERR_STATE, 4);
      valid = false;
    }
  }
  if (valid) {
    const int32_t head_net = (int32_t)(net << 8);
#pragma unroll
    for (int j = 0; j < kMaxNew; j++) {
      if ((uint32_t)j < n_new) {
        const uint8_t c0 = T.src[j][0], c1 = T.src[j][1], c2 = T.src[j][2];
        int4 rec;
        rec.x = head_net | (int32_t)T.lab[j];
        rec.y = c0 == kValNone ? 0 : (int32_t)vals[c0 * B];
        rec.z = c1 == kValNone ? 0 : (int32_t)vals[c1 * B];
        rec.w = c2 == kValNone ? 0 : (int32_t)vals[c2 * B];
        st_node(d.node + idx_of(vals[(kValNew + j) * B]), rec);
      }
    }
    n_link = T.n_link;
  }
  // a4 + a5: link the equations of Theta' and compact the new active pairs
  // (warp ballot + popc, one shared reservation per warp; in wide steps one
  // global reservation per block).
  uint32_t pushed = 0;
  const uint32_t max_link = __reduce_max_sync(kFull, n_link);
  // the paper's form (Sec. 3.4): every pair of the step owns eq_fix_n result
  // slots; those its name equations do not fill stay dummies (0)
  const unsigned long long slot0 = (unsigned long long)i * d.eq_fix_n;
  if (d.paper && i < n)
    for (uint32_t k = 0; k < d.eq_fix_n; k++)
      if (slot0 + k < d.cap_fix) d.eq_fix[slot0 + k] = 0ull;
  for (uint32_t k = 0; k < max_link; k++) {
    Pair out;
    bool has = false;
    if (k < n_link) has = link_eq<kTrack>(d, s, vals[T.link[k][0] * B], vals[T.link[k][1] * B], &out, slot0 + k);
    const unsigned m = __ballot_sync(kFull, has);
    if (m) {
      const int leader = __ffs(m) - 1;
      int wb = 0;
      if (lane == leader) wb = atomicAdd(&s.misc[SOLO ? M_SFN : M_NPUSH], __popc(m));
      wb = __shfl_sync(kFull, wb, leader);
      if (has) {
        const uint32_t at = (uint32_t)wb + __popc(m & lanemask_lt());
        if (SOLO) s.sf[cur ^ 1][at] = out;
        else s.push[at] = out;
      }
    }
    pushed += has ? 1u : 0u;
  }
  // a6: per-net counters (interactions, pending pairs) and the rule histogram
  const unsigned vm = __ballot_sync(kFull, valid);
  if (valid) {
    const unsigned peers = __match_any_sync(vm, net);
    if (peers == vm) {
      const uint32_t tp = __reduce_add_sync(vm, pushed);
      const uint32_t cnt = __popc(vm);
      if (lane == __ffs(vm) - 1)
        atomicAdd(d.netctr + net, (unsigned long long)cnt +
                                      ((unsigned long long)((long long)tp - (long long)cnt) << kNetPairShift));
    } else {
      atomicAdd(d.netctr + net, 1ull + ((unsigned long long)((long long)pushed - 1) << kNetPairShift));
    }
    // live agents of the net (its quota is checked between launches)
    if constexpr (kTrack) {
      if (n_new != 2) atomicAdd(reinterpret_cast<unsigned long long*>(d.netlive + net),
                                (unsigned long long)((long long)n_new - 2));
    }
    const unsigned rp = __match_any_sync(vm, (unsigned)T.rule);
    if (lane == __ffs(rp) - 1) atomicAdd(&s.hist[T.rule], (uint32_t)__popc(rp));
  }
  __syncthreads();
  if (tid == 0) {
    if (!SOLO) {
      const uint32_t np = (uint32_t)s.misc[M_NPUSH];
      s.misc[M_PBASE] = -1;
      if (np) {
        const uint32_t pb = atomicAdd(&c->fcount[cur ^ 1], np);
        if ((unsigned long long)pb + np > d.cap_pairs) set_error(c, INET_ERR_ARENA_FULL, 1);
        else s.misc[M_PBASE] = (int)pb;
      }
    }
    // freed names: onto the local stack, the overflow to the global ring
    const uint32_t nv = min((uint32_t)s.misc[M_NVSTAGE], kVarStage * B);
    const uint32_t lv = (uint32_t)s.misc[M_LV];
    const uint32_t keep = min(capL - lv, nv);
    s.misc[M_NVSTAGE] = (int)nv;
    s.misc[M_LV_FBASE] = (int)lv;
    s.misc[M_LV_KEEP] = (int)keep;
    s.misc[M_LV] = (int)(lv + keep);
    s.warp[W_VFREE] = nv > keep ? atomicAdd(&c->v_tail, (unsigned long long)(nv - keep)) : 0ull;
  }
  __syncthreads();
  {
    if (!SOLO) {
      const uint32_t np = (uint32_t)s.misc[M_NPUSH];
      const int pb = s.misc[M_PBASE];
      if (pb >= 0) {
        Pair* dst = d.front[cur ^ 1] + pb;
        for (uint32_t j = tid; j < np; j += B)
          __stcg(reinterpret_cast<unsigned long long*>(dst + j), *reinterpret_cast<const unsigned long long*>(&s.push[j]));
      }
    }
    // agent frees (the taken local entries have all been read by now)
    if (free_a && valid) {
      const uint32_t of = (uint32_t)((ex >> 32) & 0xFFFF);
      const uint32_t keep = (uint32_t)s.misc[M_LA_KEEP], base0 = (uint32_t)s.misc[M_LA_BASE];
      for (uint32_t f = 0; f < free_a; f++) {
        const uint32_t slot = (n_new == 0 && f == 0) ? a : b;
        const uint32_t k = of + f;
        if constexpr (kTrack) __stcg(&d.node[slot].head, kFreeHead);
        if (k < keep) s.la[base0 + k] = slot;
        else __stcg(d.afree + (s.warp[W_AFREE] + (k - keep)) % d.cap_agents, slot);
      }
    }
    const uint32_t nv = (uint32_t)s.misc[M_NVSTAGE], keep = (uint32_t)s.misc[M_LV_KEEP];
    const uint32_t fb = (uint32_t)s.misc[M_LV_FBASE];
    const unsigned long long vb = s.warp[W_VFREE];
    for (uint32_t j = tid; j < nv; j += B) {
      if (j < keep) s.lv[fb + j] = s.vstage[j];
      else __stcg(d.vfree + (vb + (j - keep)) % d.cap_vars, s.vstage[j]);
    }
  }
  __syncthreads();
}

// Hands the block's local free-slot stacks back to the global rings (at the
// end of a launch, so that no free slot is known only to a block).
__device__ void spill_local(const Dev& d, const Smem& s) {
  Ctrl* c = d.ctrl;
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t la = (uint32_t)s.misc[M_LA], lv = (uint32_t)s.misc[M_LV];
    s.warp[W_AFREE] = la ? atomicAdd(&c->a_tail, (unsigned long long)la) : 0ull;
    s.warp[W_VFREE] = lv ? atomicAdd(&c->v_tail, (unsigned long long)lv) : 0ull;
  }
  __syncthreads();
  const uint32_t la = (uint32_t)s.misc[M_LA], lv = (uint32_t)s.misc[M_LV];
  for (uint32_t j = threadIdx.x; j < la; j += blockDim.x)
    __stcg(d.afree + (s.warp[W_AFREE] + j) % d.cap_agents, s.la[j]);
  for (uint32_t j = threadIdx.x; j < lv; j += blockDim.x)
    __stcg(d.vfree + (s.warp[W_VFREE] + j) % d.cap_vars, s.lv[j]);
  __syncthreads();
  if (threadIdx.x == 0) {
    s.misc[M_LA] = 0;
    s.misc[M_LV] = 0;
  }
  __syncthreads();
}

// Step bookkeeping of k_step, run by the last block to finish: publish the
// freed slots, swap the frontiers, record the trace and decide termination
// (Sec. 3.6: stop when no active pair is left).
__device__ void finalize_step(const Dev& d) {
  Ctrl* c = d.ctrl;
  __threadfence();
  const uint32_t step = ld_volatile(&c->step);
  const uint32_t cur = step & 1u, nxt = cur ^ 1u;
  const uint32_t n_cur = ld_volatile(&c->fcount[cur]);
  const uint32_t n_next = ld_volatile(&c->fcount[nxt]);
  unsigned long long h = ld_volatile64(&c->a_head), p = ld_volatile64(&c->a_pub);
  if (h > p) c->a_head = p;
  c->a_pub = ld_volatile64(&c->a_tail);
  h = ld_volatile64(&c->v_head);
  p = ld_volatile64(&c->v_pub);
  if (h > p) c->v_head = p;
  c->v_pub = ld_volatile64(&c->v_tail);
  const long long live = ld_volatile_s64(&c->live);
  if (n_cur) {
    if (live > c->peak_live) c->peak_live = live;
    if (n_cur > c->max_frontier) c->max_frontier = n_cur;
    if (c->trace_on) {
      const uint32_t k = step - c->call_step0;
      if (k < d.trace_cap) {
        d.trace_front[k] = n_cur;
        d.trace_live[k] = live;
      }
    }
    c->fcount[cur] = 0;
    c->step = step + 1;
  }
  const uint32_t done_limit = (n_cur && step + 1 >= c->stop_step) ? 1u : 0u;
  if (done_limit && n_next) c->hit_limit = 1;
  // bound the time one launch holds the GPU; the host resumes the loop
  const unsigned long long now = globaltimer();
  bool slice_over = false;
  if (c->slice_t0 == 0) c->slice_t0 = now;
  else if (now - c->slice_t0 > d.slice_ns) slice_over = true;
  if (slice_over && n_next && !done_limit) c->hit_slice = 1;
  const bool done = n_next == 0 || ld_volatile((const uint32_t*)&c->fatal) != 0 || done_limit || n_cur == 0 ||
                    slice_over;
  c->done = done ? 1u : 0u;
  __threadfence();
}

// One step of the loop; the last block to finish runs finalize_step().
// Used by the plain host loop and by the CUDA-graph loop.
template <bool kTrack>
__global__ void __launch_bounds__(512) k_step(Dev d) {
  Smem s = carve(d, 0);
  load_tables(d, s);
  Ctrl* c = d.ctrl;
  const uint32_t step = ld_volatile(&c->step);
  const uint32_t cur = step & 1u;
  const uint32_t n = min(ld_volatile(&c->fcount[cur]), d.cap_pairs);
  const bool stop = ld_volatile(&c->done) != 0;
  if (!stop) {
    for (uint32_t chunk = blockIdx.x; (unsigned long long)chunk * blockDim.x < n; chunk += gridDim.x)
      process_chunk<false, kTrack>(d, s, chunk * blockDim.x, n, cur);
  }
  spill_local(d, s);
  flush_live(d, s);
  flush_hist(d, s);
  __threadfence();
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(&c->blocks_done, 1u);
    s.misc[M_LAST] = (t == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (s.misc[M_LAST] && threadIdx.x == 0) {
    c->blocks_done = 0;
    if (!stop) finalize_step(d);
    if (d.use_cond) cudaGraphSetConditional(d.cond, ld_volatile(&c->done) ? 0u : 1u);
  }
}

// ---------------------------------------------------------------------------
// Persistent kernel.  Block 0 coordinates: in a wide step the blocks that
// hold a chunk of the frontier process it and arrive; block 0 waits for the
// arrivals, does the step bookkeeping (with state it keeps in shared memory)
// and publishes the next step's frontier size and parity in bar_word, which
// the other blocks poll.  A frontier of at most solo_max pairs is reduced by
// block 0 alone, step after step, with the frontier in shared memory and
// block barriers only.  Every wait is bounded: a waiter gives up after
// timeout_ns without progress, records INET_ERR_TIMEOUT and returns.

// Step bookkeeping shared by wide and solo steps (thread 0 of block 0).
// `n_cur` pairs were processed and `n_next` are pending.  Returns whether
// the loop is done.
__device__ bool coord_account(const Dev& d, const Smem& s, uint32_t n_cur, uint32_t n_next, long long live,
                              int32_t fatal) {
  Ctrl* c = d.ctrl;
  const uint32_t step = (uint32_t)s.warp[W_STEP];
  if ((long long)s.warp[W_PEAK] < live) s.warp[W_PEAK] = (unsigned long long)live;
  if (s.warp[W_MAXF] < n_cur) s.warp[W_MAXF] = n_cur;
  if (s.warp[W_TRACE]) {
    const uint32_t k = step - (uint32_t)s.warp[W_STEP0];
    if (k < d.trace_cap) {
      d.trace_front[k] = n_cur;
      d.trace_live[k] = live;
    }
  }
  s.warp[W_STEP] = step + 1;
  c->step = step + 1;  // also the progress signal of bounded waits
  const bool done_limit = step + 1 >= (uint32_t)s.warp[W_STOP];
  if (done_limit && n_next) c->hit_limit = 1;
  const unsigned long long now = globaltimer();
  bool slice_over = false;
  if (s.warp[W_T0] == 0) s.warp[W_T0] = now;
  else if (now - s.warp[W_T0] > d.slice_ns) slice_over = true;
  if (slice_over && n_next && !done_limit) c->hit_slice = 1;
  return n_next == 0 || fatal != 0 || done_limit || slice_over;
}

// Publishes the step word (thread 0 of block 0, after the step's stores).
__device__ __forceinline__ void coord_publish(const Dev& d, const Smem& s, uint32_t n, uint32_t cur, bool done) {
  Ctrl* c = d.ctrl;
  const unsigned long long old = s.warp[W_WORD];
  const unsigned long long w = pack_word(n, word_gen(old) + 1, cur, done ? 1u : 0u);
  c->done = done ? 1u : 0u;
  c->peak_live = (long long)s.warp[W_PEAK];
  c->max_frontier = s.warp[W_MAXF];
  c->bar_count = 0;
  __threadfence();
  *reinterpret_cast<volatile unsigned long long*>(&c->bar_word) = w;
  s.warp[W_WORD] = w;
}

// Loads the counters other blocks update, one per lane of warp 0, with one
// load instruction (no serial round trips).
__device__ __forceinline__ void coord_gather(const Dev& d, const Smem& s) {
  Ctrl* c = d.ctrl;
  const uint32_t t = threadIdx.x;
  if (t < 7) {
    const unsigned long long* p =
        t == 0 ? reinterpret_cast<const unsigned long long*>(&c->fcount[0])
      : t == 1 ? &c->a_head
      : t == 2 ? &c->a_tail
      : t == 3 ? &c->v_head
      : t == 4 ? &c->v_tail
      : t == 5 ? reinterpret_cast<const unsigned long long*>(&c->live)
               : reinterpret_cast<const unsigned long long*>(&c->fatal);
    s.warp[W_LD0 + t] = ld_volatile64(p);
  }
  __syncthreads();
}

// Publishes the ring tails (thread 0 of block 0, after coord_gather).
__device__ __forceinline__ void coord_pools(const Dev& d, const Smem& s) {
  Ctrl* c = d.ctrl;
  if (s.warp[W_LD1] > s.warp[W_APUB]) c->a_head = s.warp[W_APUB];
  s.warp[W_APUB] = s.warp[W_LD2];
  c->a_pub = s.warp[W_LD2];
  if (s.warp[W_LD3] > s.warp[W_VPUB]) c->v_head = s.warp[W_VPUB];
  s.warp[W_VPUB] = s.warp[W_LD4];
  c->v_pub = s.warp[W_LD4];
}

// Bounded wait of one thread until `pred` holds; progress of the step
// counter restarts the clock.  Returns false on timeout (error recorded).
// Polls back off (up to `nap_max` ns between polls) so that hundreds of
// waiting blocks do not flood the L2 slice that holds the word they watch.
template <class Pred>
__device__ bool bounded_wait(const Dev& d, Pred pred, uint32_t nap_max) {
  Ctrl* c = d.ctrl;
  unsigned long long t0 = globaltimer();
  uint32_t seen = ld_volatile(&c->step);
  uint32_t nap = 32;
  for (uint32_t spin = 0;; spin++) {
    if (pred()) return true;
    __nanosleep(nap);
    if (nap < nap_max) nap <<= 1;
    if ((spin & 15) == 15) {
      const unsigned long long now = globaltimer();
      const uint32_t st = ld_volatile(&c->step);
      if (st != seen) {
        seen = st;
        t0 = now;
      } else if (now - t0 > d.timeout_ns) {
        set_error(c, INET_ERR_TIMEOUT, blockIdx.x);
        return false;
      }
    }
  }
}

// Block 0 alone: steps with the frontier in shared memory, until it is
// empty, grows beyond solo_max, or the call must stop; then the frontier
// goes back to global memory and the step word is published.
template <bool kTrack>
__device__ void solo_phase(const Dev& d, const Smem& s, uint32_t n, uint32_t gcur) {
  Ctrl* c = d.ctrl;
  const uint32_t tid = threadIdx.x, B = blockDim.x;
  for (uint32_t j = tid; j < n; j += B) {
    const unsigned long long pv = __ldcg(reinterpret_cast<const unsigned long long*>(d.front[gcur] + j));
    s.sf[0][j] = *reinterpret_cast<const Pair*>(&pv);
  }
  if (tid == 0) {
    s.misc[M_SFN] = 0;
    s.warp[W_LIVE] = (unsigned long long)ld_volatile_s64(&c->live);
  }
  __syncthreads();
  uint32_t lc = 0;
  bool done = false;
  for (uint32_t it = 0;; it++) {
    const int32_t fatal_seen = (it & 15) == 15 ? (int32_t)ld_volatile((const uint32_t*)&c->fatal) : 0;
    for (uint32_t base = 0; base < n; base += B) process_chunk<true, kTrack>(d, s, base, n, lc);
    if (tid == 0) {
      const uint32_t n_next = (uint32_t)s.misc[M_SFN];
      s.misc[M_SFN] = 0;
      const long long live = (long long)s.warp[W_LIVE] + s.misc[M_LIVE];
      s.warp[W_LIVE] = (unsigned long long)live;
      s.misc[M_LIVE] = 0;
      const bool dn = coord_account(d, s, n, n_next, live, fatal_seen);
      s.misc[M_STOP] = (dn ? 2 : 0) | (n_next > d.solo_max ? 1 : 0);
      s.misc[M_NNEXT] = (int)n_next;
    }
    __syncthreads();
    n = (uint32_t)s.misc[M_NNEXT];
    const int stop = s.misc[M_STOP];
    done = (stop & 2) != 0;
    lc ^= 1u;
    __syncthreads();
    if (stop) break;
  }
  // hand the frontier back at the parity of the step count
  const uint32_t g = (uint32_t)s.warp[W_STEP] & 1u;
  for (uint32_t j = tid; j < n; j += B)
    __stcg(reinterpret_cast<unsigned long long*>(d.front[g] + j), *reinterpret_cast<const unsigned long long*>(&s.sf[lc][j]));
  coord_gather(d, s);
  if (tid == 0) {
    coord_pools(d, s);
    c->fcount[g] = n;
    c->fcount[g ^ 1u] = 0;
    c->live = (long long)s.warp[W_LIVE];
    done = done || (int32_t)(uint32_t)s.warp[W_LD6] != 0;
    coord_publish(d, s, n, g, done);
  }
  __syncthreads();
}

template <bool kTrack>
__global__ void __launch_bounds__(512) k_persistent(Dev d) {
  Smem s = carve(d, d.solo_max);
  load_tables(d, s);
  Ctrl* c = d.ctrl;
  const uint32_t tid = threadIdx.x, B = blockDim.x;
  const bool coord = blockIdx.x == 0;
  if (tid == 0) {
    s.warp[W_WORD] = ld_volatile64(&c->bar_word);
    if (coord) {
      s.warp[W_STEP] = ld_volatile(&c->step);
      s.warp[W_PEAK] = (unsigned long long)c->peak_live;
      s.warp[W_MAXF] = c->max_frontier;
      s.warp[W_APUB] = ld_volatile64(&c->a_pub);
      s.warp[W_VPUB] = ld_volatile64(&c->v_pub);
      s.warp[W_T0] = 0;
      s.warp[W_STOP] = c->stop_step;
      s.warp[W_TRACE] = c->trace_on;
      s.warp[W_STEP0] = c->call_step0;
    }
  }
  __syncthreads();
  for (;;) {
    const unsigned long long w = s.warp[W_WORD];
    const bool stop = word_done(w) || s.misc[M_TIMEOUT];
    __syncthreads();
    if (stop) break;
    const uint32_t n = word_n(w), cur = word_cur(w);
    const bool solo = n <= d.solo_max;
    const uint32_t nchunks = (n + B - 1) / B;
    const uint32_t A = solo ? 1u : min(gridDim.x, nchunks);
    if (coord) {
      if (solo) {
        solo_phase<kTrack>(d, s, n, cur);
      } else {
        for (uint32_t ch = 0; ch < nchunks; ch += A) process_chunk<false, kTrack>(d, s, ch * B, n, cur);
        flush_live(d, s);
        if (tid == 0 && A > 1) {
          if (!bounded_wait(d, [&] { return ld_volatile(&c->bar_count) >= A - 1; }, 64)) s.misc[M_TIMEOUT] = 1;
          __threadfence();
        }
        __syncthreads();
        coord_gather(d, s);
        if (tid == 0) {
          coord_pools(d, s);
          const uint32_t fc = (uint32_t)(s.warp[W_LD0] >> ((cur ^ 1u) * 32));
          const uint32_t n_next = min(fc, d.cap_pairs);
          c->fcount[cur] = 0;
          const long long live = (long long)s.warp[W_LD5];
          bool done = coord_account(d, s, n, n_next, live, (int32_t)(uint32_t)s.warp[W_LD6]);
          done = done || s.misc[M_TIMEOUT] != 0;
          coord_publish(d, s, n_next, cur ^ 1u, done);
        }
        __syncthreads();
      }
    } else {
      if (!solo && blockIdx.x < A) {
        for (uint32_t ch = blockIdx.x; ch < nchunks; ch += A) process_chunk<false, kTrack>(d, s, ch * B, n, cur);
        flush_live(d, s);
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          atomicAdd(&c->bar_count, 1u);
        }
      }
      if (tid == 0) {
        const uint32_t gen = word_gen(w);
        unsigned long long nw = w;
        const bool ok = bounded_wait(d, [&] {
          nw = ld_volatile64(&c->bar_word);
          return word_gen(nw) != gen;
        }, d.solo_max && word_n(w) <= d.solo_max ? 2048u : 256u);
        __threadfence();
        if (ok) s.warp[W_WORD] = nw;
        else s.misc[M_TIMEOUT] = 1;
      }
      __syncthreads();
    }
  }
  spill_local(d, s);
  flush_live(d, s);
  flush_hist(d, s);
}

// Nets whose pending pairs reached zero and that were not reported before:
// their ids go to out[0 .. cap) and they are marked reported (nets that do
// not fit are left for the next call).  Runs between reductions.
__global__ void k_net_finished(Dev d, uint32_t n_nets, int32_t* out, uint32_t cap, uint32_t* count) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nets || d.netrep[i]) return;
  if ((__ldcg(d.netctr + i) >> kNetPairShift) != 0) return;
  const uint32_t k = atomicAdd(count, 1u);
  if (k < cap) {
    out[k] = (int32_t)i;
    d.netrep[i] = 1;
  }
}

}  // namespace inet
