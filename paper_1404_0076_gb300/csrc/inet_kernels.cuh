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
constexpr int kVarStage = 4;  // staged freed name slots per thread (overflow goes direct)

// Control block.  Hot atomic counters sit on their own 128-byte lines.
struct alignas(128) Line { unsigned long long w[16]; };
struct Ctrl {
  // line 0: step state (written by the finalizer only)
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
  // line 2..: agent pool
  alignas(128) unsigned long long a_head;
  alignas(128) unsigned long long a_tail;
  alignas(128) unsigned long long a_pub;    // ring entries below this are poppable
  unsigned long long v_pub;
  alignas(128) unsigned long long v_head;
  alignas(128) unsigned long long v_tail;
  alignas(128) unsigned long long a_bump;   // next never-used agent slot
  alignas(128) unsigned long long v_bump;   // next never-used name slot
  // barrier
  alignas(128) uint32_t bar_count;
  alignas(128) uint32_t bar_gen;
  alignas(128) uint32_t blocks_done;
  alignas(128) long long live;              // live agents, all nets
};

struct Dev {
  Node* node;
  uint32_t* var;
  Pair* front[2];
  uint32_t* afree;
  uint32_t* vfree;
  unsigned long long* netctr;
  int32_t* netstat;
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
  uint32_t solo_max;
  uint32_t max_nets;
  unsigned long long timeout_ns;
  unsigned long long slice_ns;   // a launch stops at the first step boundary after this
  cudaGraphConditionalHandle cond;
  int use_cond;
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
  int16_t* tab;        // n_labels^2
  Template* tmpl;      // n_tmpl
  uint8_t* arity;      // n_labels
  uint32_t* vals;      // kNumVals * blockDim
  Pair* push;          // kMaxLink * blockDim
  uint32_t* vstage;    // kVarStage * blockDim
  uint32_t* hist;      // INET_MAX_RULES
  unsigned long long* warp;  // 33 scan slots
  uint32_t* misc;      // counters and broadcast values
};
// misc slots
enum { M_NPUSH = 0, M_NVSTAGE, M_FAIL, M_LAST, M_STEP, M_N, M_DONE, M_TIMEOUT, M_PBASE, M_VFBASE,
       M_COUNT };
// 64-bit broadcast slots live in warp[] beyond the scan area
enum { W_ARING = 34, W_AAVAIL, W_ABUMP, W_VRING, W_VAVAIL, W_VBUMP, W_AFREE, W_SLOTS };

__host__ __device__ inline size_t smem_bytes(uint32_t block, uint32_t n_labels, uint32_t n_tmpl) {
  size_t b = 0;
  auto take = [&](size_t n, size_t align) { b = (b + align - 1) / align * align; b += n; };
  take(sizeof(Template) * (n_tmpl ? n_tmpl : 1), 16);
  take(sizeof(unsigned long long) * W_SLOTS, 16);
  take(sizeof(Pair) * kMaxLink * block, 16);
  take(sizeof(uint32_t) * kNumVals * block, 16);
  take(sizeof(uint32_t) * kVarStage * block, 16);
  take(sizeof(uint32_t) * INET_MAX_RULES, 16);
  take(sizeof(uint32_t) * M_COUNT, 16);
  take(sizeof(int16_t) * n_labels * n_labels, 16);
  take(n_labels, 16);
  return b + 16;
}

__device__ __forceinline__ Smem carve(const Dev& d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  size_t b = 0;
  auto take = [&](size_t n, size_t align) -> unsigned char* {
    b = (b + align - 1) / align * align;
    unsigned char* p = smem_raw + b;
    b += n;
    return p;
  };
  Smem s;
  uint32_t B = blockDim.x;
  s.tmpl = reinterpret_cast<Template*>(take(sizeof(Template) * (d.n_tmpl ? d.n_tmpl : 1), 16));
  s.warp = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * W_SLOTS, 16));
  s.push = reinterpret_cast<Pair*>(take(sizeof(Pair) * kMaxLink * B, 16));
  s.vals = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * kNumVals * B, 16));
  s.vstage = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * kVarStage * B, 16));
  s.hist = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * INET_MAX_RULES, 16));
  s.misc = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * M_COUNT, 16));
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

// Block-wide exclusive scan of a packed 64-bit value (four 16-bit fields).
// Every thread gets its exclusive prefix; the block total is in s.warp[32].
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
    if (lane == nw - 1) s.warp[32] = wi;
  }
  __syncthreads();
  return s.warp[wid] + inc - v;
}

// ---------------------------------------------------------------------------
// Pools.  A ring of freed slot ids per kind; pops only take entries published
// before the step (a_pub / v_pub), pushes append at the tail, and the
// finalizer publishes the tail between steps, so a slot is never handed out
// in the step that freed it.  When the ring runs dry the bump pointer hands
// out never-used slots.

__device__ __forceinline__ bool pool_pop(unsigned long long* head, unsigned long long pub,
                                         unsigned long long* bump, unsigned long long cap,
                                         uint32_t k, unsigned long long* ring_base,
                                         uint32_t* ring_avail, unsigned long long* bump_base) {
  *ring_avail = 0;
  *ring_base = 0;
  *bump_base = 0;
  if (k == 0) return true;
  unsigned long long h = atomicAdd(head, (unsigned long long)k);
  uint32_t avail = h < pub ? (uint32_t)min((unsigned long long)k, pub - h) : 0u;
  *ring_base = h;
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
  if (k < ring_avail) return __ldcg(ring + (ring_base + k) % cap);
  return (uint32_t)(bump_base + (k - ring_avail));
}

__device__ __forceinline__ void free_var_direct(const Dev& d, uint32_t x) {
  unsigned long long t = atomicAdd(&d.ctrl->v_tail, 1ull);
  __stcg(d.vfree + t % d.cap_vars, x);
}

// ->com on name slots (Sec. 2.2, Communication; Sec. 3.5-3.6).  Links the
// equation t = u.  Two agents form an active pair.  Otherwise the equation
// arrives at a name slot x (t or u a name): the first arrival stores its
// other side; the second finds the stored term s and continues with s = u,
// which resolves chains x1 = x2 = .. of any length in one call (the chains of
// Sec. 3.6 that need several passes of the sorting algorithm).  Returns true
// and the pair when an active pair results.
__device__ __forceinline__ bool link_eq(const Dev& d, const Smem& s, uint32_t t, uint32_t u,
                                        Pair* out) {
  for (uint32_t guard = 0;; guard++) {
    if (is_agent(t) && is_agent(u)) {
      out->a = idx_of(t);
      out->b = idx_of(u);
      return true;
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
    uint32_t pos = atomicAdd(&s.misc[M_NVSTAGE], 1u);
    if (pos < kVarStage * blockDim.x) s.vstage[pos] = x;
    else free_var_direct(d, x);
    t = old;
  }
}

// One chunk of the frontier: pairs [base, base + blockDim.x) of frontier
// `cur` (n pairs).  All threads of the block call it together.
__device__ void process_chunk(const Dev& d, const Smem& s, uint32_t base, uint32_t n, uint32_t cur) {
  const uint32_t tid = threadIdx.x, B = blockDim.x;
  const int lane = tid & 31;
  Ctrl* c = d.ctrl;
  const uint32_t i = base + tid;
  bool valid = i < n;
  uint32_t a = 0, b = 0, net = 0, ti = 0;
  int4 ra = make_int4(0, 0, 0, 0), rb = ra;
  // a1: frontier read + dispatch through the (label, label) table
  if (valid) {
    const unsigned long long pv = __ldcg(reinterpret_cast<const unsigned long long*>(d.front[cur] + i));
    a = (uint32_t)pv;
    b = (uint32_t)(pv >> 32);
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
      e = 0;
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
  // first two new agents; the rest comes from the pools.
  const uint32_t need_a = n_new > 2 ? n_new - 2 : 0u;
  const uint32_t free_a = valid && n_new < 2 ? 2 - n_new : 0u;
  const unsigned long long packed = (unsigned long long)need_a | ((unsigned long long)n_fresh << 16) |
                                    ((unsigned long long)free_a << 32) | ((unsigned long long)(valid ? 1 : 0) << 48);
  const unsigned long long ex = block_scan(packed, s);
  if (tid == 0) {
    const unsigned long long tot = s.warp[32];
    const uint32_t Ka = (uint32_t)(tot & 0xFFFF), Kv = (uint32_t)((tot >> 16) & 0xFFFF);
    const uint32_t Fa = (uint32_t)((tot >> 32) & 0xFFFF);
    unsigned long long rb0, bb0;
    uint32_t av0;
    bool ok = pool_pop(&c->a_head, ld_volatile64(&c->a_pub), &c->a_bump, d.cap_agents, Ka, &rb0, &av0, &bb0);
    s.warp[W_ARING] = rb0;
    s.warp[W_AAVAIL] = av0;
    s.warp[W_ABUMP] = bb0;
    ok = pool_pop(&c->v_head, ld_volatile64(&c->v_pub), &c->v_bump, d.cap_vars, Kv, &rb0, &av0, &bb0) && ok;
    s.warp[W_VRING] = rb0;
    s.warp[W_VAVAIL] = av0;
    s.warp[W_VBUMP] = bb0;
    s.warp[W_AFREE] = Fa ? atomicAdd(&c->a_tail, (unsigned long long)Fa) : 0ull;
    if (Ka != Fa)
      atomicAdd(reinterpret_cast<unsigned long long*>(&c->live), (unsigned long long)((long long)Ka - (long long)Fa));
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
    vals[(kValExt + 0) * B] = (uint32_t)ra.y;
    vals[(kValExt + 1) * B] = (uint32_t)ra.z;
    vals[(kValExt + 2) * B] = (uint32_t)ra.w;
    vals[(kValExt + 3) * B] = (uint32_t)rb.y;
    vals[(kValExt + 4) * B] = (uint32_t)rb.z;
    vals[(kValExt + 5) * B] = (uint32_t)rb.w;
    uint32_t slots[kMaxNew];
#pragma unroll
    for (int j = 0; j < kMaxNew; j++) {
      if ((uint32_t)j < n_new) {
        uint32_t sl = j == 0 ? a
                    : j == 1 ? b
                    : pool_slot(d.afree, d.cap_agents, s.warp[W_ARING], (uint32_t)s.warp[W_AAVAIL],
                                s.warp[W_ABUMP], oa + (uint32_t)j - 2);
        slots[j] = sl;
        vals[(kValNew + j) * B] = mk_agent(sl);
      }
    }
#pragma unroll
    for (int v = 0; v < kMaxFresh; v++) {
      if ((uint32_t)v < n_fresh) {
        uint32_t x = pool_slot(d.vfree, d.cap_vars, s.warp[W_VRING], (uint32_t)s.warp[W_VAVAIL],
                               s.warp[W_VBUMP], ov + (uint32_t)v);
        vals[(kValFresh + v) * B] = mk_var(x);
      }
    }
    bool in_range = true;
#pragma unroll
    for (int j = 2; j < kMaxNew; j++)
      if ((uint32_t)j < n_new && slots[j] >= d.cap_agents) in_range = false;
#pragma unroll
    for (int v = 0; v < kMaxFresh; v++)
      if ((uint32_t)v < n_fresh && idx_of(vals[(kValFresh + v) * B]) >= d.cap_vars) in_range = false;
    if (!in_range) {
      set_error(c, INET_ERR_STATE, 4);
      valid = false;
    }
  }
  if (valid) {
    const uint32_t of = (uint32_t)((ex >> 32) & 0xFFFF);
    uint32_t slots[kMaxNew];
#pragma unroll
    for (int j = 0; j < kMaxNew; j++) slots[j] = idx_of(vals[(kValNew + j) * B]);
    if (free_a) {
      const unsigned long long fb = s.warp[W_AFREE] + of;
      if (n_new == 0) {
        __stcg(d.afree + fb % d.cap_agents, a);
        __stcg(d.afree + (fb + 1) % d.cap_agents, b);
      } else {
        __stcg(d.afree + fb % d.cap_agents, b);
      }
    }
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
        st_node(d.node + slots[j], rec);
      }
    }
    n_link = T.n_link;
  }
  // a4 + a5: link the equations of Theta' and compact the new active pairs
  // (warp ballot + popc, one shared reservation per warp, one global
  // reservation per block).
  uint32_t pushed = 0;
  const uint32_t max_link = __reduce_max_sync(kFull, n_link);
  for (uint32_t k = 0; k < max_link; k++) {
    Pair out;
    bool has = false;
    if (k < n_link) has = link_eq(d, s, vals[T.link[k][0] * B], vals[T.link[k][1] * B], &out);
    const unsigned m = __ballot_sync(kFull, has);
    if (m) {
      const int leader = __ffs(m) - 1;
      uint32_t wb = 0;
      if (lane == leader) wb = atomicAdd(&s.misc[M_NPUSH], (uint32_t)__popc(m));
      wb = __shfl_sync(kFull, wb, leader);
      if (has) s.push[wb + __popc(m & lanemask_lt())] = out;
    }
    pushed += has ? 1u : 0u;
  }
  // a6: per-net counters (interactions, pending pairs) and the rule histogram
  const unsigned vm = __ballot_sync(kFull, valid);
  if (valid) {
    const unsigned peers = __match_any_sync(vm, net);
    const unsigned long long one = 1ull + ((unsigned long long)((long long)pushed - 1) << kNetPairShift);
    if (peers == vm) {
      const uint32_t tp = __reduce_add_sync(vm, pushed);
      const uint32_t cnt = __popc(vm);
      if (lane == __ffs(vm) - 1)
        atomicAdd(d.netctr + net, (unsigned long long)cnt +
                                      ((unsigned long long)((long long)tp - (long long)cnt) << kNetPairShift));
    } else {
      atomicAdd(d.netctr + net, one);
    }
    const unsigned rp = __match_any_sync(vm, (unsigned)T.rule);
    if (lane == __ffs(rp) - 1) atomicAdd(&s.hist[T.rule], (uint32_t)__popc(rp));
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t np = s.misc[M_NPUSH];
    if (np) {
      const uint32_t pb = atomicAdd(&c->fcount[cur ^ 1], np);
      if ((unsigned long long)pb + np > d.cap_pairs) {
        set_error(c, INET_ERR_ARENA_FULL, 1);
        s.misc[M_PBASE] = 0xFFFFFFFFu;
      } else {
        s.misc[M_PBASE] = pb;
      }
    }
    uint32_t nv = min(s.misc[M_NVSTAGE], kVarStage * B);
    s.misc[M_NVSTAGE] = nv;
    s.warp[W_AFREE] = nv ? atomicAdd(&c->v_tail, (unsigned long long)nv) : 0ull;
  }
  __syncthreads();
  {
    const uint32_t np = s.misc[M_NPUSH], pb = s.misc[M_PBASE];
    if (pb != 0xFFFFFFFFu) {
      Pair* dst = d.front[cur ^ 1] + pb;
      for (uint32_t j = tid; j < np; j += B)
        __stcg(reinterpret_cast<unsigned long long*>(dst + j), *reinterpret_cast<const unsigned long long*>(&s.push[j]));
    }
    const uint32_t nv = s.misc[M_NVSTAGE];
    const unsigned long long vb = s.warp[W_AFREE];
    for (uint32_t j = tid; j < nv; j += B) __stcg(d.vfree + (vb + j) % d.cap_vars, s.vstage[j]);
  }
  __syncthreads();
}

// Step bookkeeping, run by one thread once every pair of the step has been
// processed: publish the freed slots, swap the frontiers, record the trace
// and decide termination (Sec. 3.6: stop when no active pair is left).
__device__ void finalize_step(const Dev& d) {
  Ctrl* c = d.ctrl;
  __threadfence();
  const uint32_t step = ld_volatile(&c->step);
  const uint32_t cur = step & 1u, nxt = cur ^ 1u;
  const uint32_t n_cur = ld_volatile(&c->fcount[cur]);
  const uint32_t n_next = ld_volatile(&c->fcount[nxt]);
  // pools: drop overshoot of pops beyond the published part, publish pushes
  unsigned long long h = ld_volatile64(&c->a_head), p = ld_volatile64(&c->a_pub);
  if (h > p) c->a_head = p;
  c->a_pub = ld_volatile64(&c->a_tail);
  h = ld_volatile64(&c->v_head);
  p = ld_volatile64(&c->v_pub);
  if (h > p) c->v_head = p;
  c->v_pub = ld_volatile64(&c->v_tail);
  const long long live = *reinterpret_cast<volatile long long*>(&c->live);
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
__global__ void __launch_bounds__(512) k_step(Dev d) {
  Smem s = carve(d);
  load_tables(d, s);
  Ctrl* c = d.ctrl;
  const uint32_t step = ld_volatile(&c->step);
  const uint32_t cur = step & 1u;
  const uint32_t n = min(ld_volatile(&c->fcount[cur]), d.cap_pairs);
  const bool stop = ld_volatile(&c->done) != 0;
  if (!stop) {
    for (uint32_t chunk = blockIdx.x; (unsigned long long)chunk * blockDim.x < n; chunk += gridDim.x)
      process_chunk(d, s, chunk * blockDim.x, n, cur);
  }
  flush_hist(d, s);
  __threadfence();
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(&c->blocks_done, 1u);
    s.misc[M_LAST] = (t == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s.misc[M_LAST] && threadIdx.x == 0) {
    c->blocks_done = 0;
    if (!stop) finalize_step(d);
    if (d.use_cond) cudaGraphSetConditional(d.cond, ld_volatile(&c->done) ? 0u : 1u);
  }
}

// Grid barrier for the persistent kernel.  The last block to arrive runs
// finalize_step() (if asked) and releases the others.  Waits are bounded:
// a waiter gives up after timeout_ns without progress of the step counter,
// records INET_ERR_TIMEOUT and returns false.
__device__ bool grid_barrier(const Dev& d, const Smem& s, bool finalize) {
  Ctrl* c = d.ctrl;
  __syncthreads();
  if (threadIdx.x == 0) {
    s.misc[M_TIMEOUT] = 0;
    __threadfence();
    const uint32_t gen = ld_volatile(&c->bar_gen);
    const uint32_t arrived = atomicAdd(&c->bar_count, 1u) + 1u;
    if (arrived == gridDim.x) {
      c->bar_count = 0;
      if (finalize) finalize_step(d);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      unsigned long long t0 = globaltimer();
      uint32_t seen_step = ld_volatile(&c->step);
      while (ld_volatile(&c->bar_gen) == gen) {
        __nanosleep(256);
        const uint32_t st = ld_volatile(&c->step);
        const unsigned long long now = globaltimer();
        if (st != seen_step) {
          seen_step = st;
          t0 = now;
        } else if (now - t0 > d.timeout_ns) {
          set_error(c, INET_ERR_TIMEOUT, blockIdx.x);
          c->done = 1;
          s.misc[M_TIMEOUT] = 1;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s.misc[M_TIMEOUT] == 0;
}

// The whole loop in one cooperative launch.  Wide steps use every block and
// a grid barrier; a frontier of at most solo_max pairs is reduced by block 0
// alone, step after step with block-level barriers only, while the other
// blocks wait at the grid barrier.
__global__ void __launch_bounds__(512) k_persistent(Dev d) {
  Smem s = carve(d);
  load_tables(d, s);
  Ctrl* c = d.ctrl;
  for (;;) {
    if (threadIdx.x == 0) {
      s.misc[M_DONE] = ld_volatile(&c->done);
      s.misc[M_STEP] = ld_volatile(&c->step);
      s.misc[M_N] = min(ld_volatile(&c->fcount[s.misc[M_STEP] & 1u]), d.cap_pairs);
    }
    __syncthreads();
    if (s.misc[M_DONE]) break;
    uint32_t step = s.misc[M_STEP], n = s.misc[M_N];
    __syncthreads();
    if (n <= d.solo_max) {
      if (blockIdx.x == 0) {
        for (;;) {
          const uint32_t cur = step & 1u;
          for (uint32_t base = 0; base < n; base += blockDim.x) process_chunk(d, s, base, n, cur);
          if (threadIdx.x == 0) {
            finalize_step(d);
            s.misc[M_DONE] = ld_volatile(&c->done);
            s.misc[M_STEP] = ld_volatile(&c->step);
            s.misc[M_N] = min(ld_volatile(&c->fcount[s.misc[M_STEP] & 1u]), d.cap_pairs);
          }
          __syncthreads();
          step = s.misc[M_STEP];
          n = s.misc[M_N];
          const bool stop = s.misc[M_DONE] || n > d.solo_max;
          __syncthreads();
          if (stop) break;
        }
      }
      if (!grid_barrier(d, s, false)) break;
    } else {
      const uint32_t cur = step & 1u;
      for (uint32_t chunk = blockIdx.x; (unsigned long long)chunk * blockDim.x < n; chunk += gridDim.x)
        process_chunk(d, s, chunk * blockDim.x, n, cur);
      if (!grid_barrier(d, s, true)) break;
    }
  }
  flush_hist(d, s);
}

}  // namespace inet
