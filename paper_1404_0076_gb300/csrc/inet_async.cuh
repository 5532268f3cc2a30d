// Asynchronous driver of the reduction loop: the same interaction (Sec. 2.2,
// ->int), allocation and linking (->com) as the step kernels, but without
// steps.  Active pairs are independent (Sec. 2.1: reducing one cannot
// affect another), so nothing forces all pairs of a "loop iteration" to
// finish before the next begins: every warp of one cooperative launch loops
// on its own, each lane holding at most one active pair.  An interaction
// that creates active pairs keeps the first as the lane's next pair (and
// starts loading its records at once), so a sequential chain of
// interactions never leaves its lane; further pairs go to idle lanes of the
// same warp, and the rest to a FIFO of tickets that idle lanes claim: a
// bounded ring whose cells carry a 64-bit sequence number each, so that a
// producer and a consumer of the same cell in different laps can never be
// confused.  The loop ends when no active pair is left anywhere (the count
// of pairs in flight reaches zero), as in Sec. 3.6; a time slice or an error
// instead drains every pair back to a frontier buffer so that the host can
// resume.
//
// Ordering without barriers: a lane writes its new agent records and fresh
// names, then one fence, then the exchanges on name slots that publish
// references to them; the queue publishes a cell with a release store of its
// sequence and is read with an acquire load; pairs handed to lanes of the
// same warp pass through shared memory and __syncwarp.  A lane that learns
// of an agent through an exchange loads its record only after the exchange
// returned (address dependency), so it sees the record written before the
// fence.
//
// kTrack (contexts created with INET_ARENA_FREE_NETS): the kernel also keeps
// what inet_free_nets scans for: the owning net of every name it creates,
// the free mark of every agent slot it frees, and both marks on the unused
// slots its warps return at the end.  The other instantiation has none of
// that code in its loop (code the loop does not run still costs this kernel
// time through instruction fetch and scheduling).
//
// Rules (a rule set known when the kernel is compiled, see inet_jit.h): the
// library compiles k_async<kTrack, Rules> at run time for the loaded rule
// set; a warp whose lanes all reduce one of its small rules runs that rule's
// own straight-line code (uni_interact, rule_body), every other warp the
// general code below it.  NoRules is the general kernel built with the
// library.
#pragma once

#include "inet_kernels.cuh"

namespace inet {

constexpr int kAStack = 128;   // per-warp stack of free agent slots
constexpr int kVStack = 128;   // per-warp stack of free name slots
constexpr int kVStageW = 64;   // names freed while linking, per warp
constexpr int kRefill = 32;    // slots fetched for the warp's stack when it runs dry
constexpr unsigned long long kNoTicket = ~0ull;

struct WarpMem {
  uint32_t vals[kNumVals][32];
  Pair out[kMaxLink][32];
  Pair xl[(kMaxLink - 1) * 32];  // extra pairs of one iteration, in lane order
  uint32_t astk[kAStack];
  uint32_t vstk[kVStack];
  uint32_t vstage[kVStageW];
  int vstage_n, pad[3];
};

__host__ __device__ inline size_t async_smem_bytes(uint32_t block, uint32_t n_labels, uint32_t n_tmpl) {
  size_t b = 0;
  auto take = [&](size_t n, size_t align) { b = (b + align - 1) / align * align; b += n; };
  take(sizeof(Template) * (n_tmpl ? n_tmpl : 1), 16);
  take(sizeof(WarpMem) * (block / 32), 16);
  take(sizeof(uint32_t) * INET_MAX_RULES, 16);
  take(sizeof(int16_t) * n_labels * n_labels, 16);
  return b + 16;
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Ticket queue: ticket t lives in cell t % cap, whose sequence number
// moves t -> t + 1 (the producer wrote the pair) -> t + cap (the consumer
// took it, so the cell is free for ticket t + cap).  A producer writes only
// when the sequence equals its own ticket, a consumer takes only at its
// ticket + 1; both compare all 64 bits, so no lap can be mistaken for
// another however far ahead tickets were claimed.

// A second arrival at name slot x: the slot is finished (its owner mark
// cleared) and goes to the warp's staging list, or the ring when that is full.
template <bool kTrack>
__device__ __forceinline__ void release_name(const Dev& d, WarpMem& W, uint32_t x) {
  __stcg(d.var + x, kEmpty);
  if constexpr (kTrack) __stcg(d.vown + x, kNoNet);
  const int pos = atomicAdd(&W.vstage_n, 1);
  if (pos < kVStageW) {
    W.vstage[pos] = x;
  } else {
    const unsigned long long tp = atomicAdd(&d.ctrl->v_tail, 1ull);
    __stcg(d.vfree + tp % d.cap_vars, x);
  }
}

// ->com for the asynchronous kernel (the chase after a second arrival):
// link_eq with freed name slots staged per warp.  The lane has fenced its
// new records before linking; a lane that receives a reference through an
// exchange loads the referenced record only after the exchange returned
// (address dependency), so it sees the record written before the fence.
template <bool kTrack>
__device__ __forceinline__ bool link_async(const Dev& d, WarpMem& W, uint32_t t, uint32_t u, Pair* out) {
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
      set_error(d.ctrl, INET_ERR_STATE, 1);
      return false;
    }
    const uint32_t x = idx_of(t);
    const uint32_t old = atomicExch(d.var + x, u);
    if (old == kEmpty) return false;
    release_name<kTrack>(d, W, x);
    t = old;
  }
}

// Rule template as the asynchronous kernel reads it from shared memory: one
// 32-bit word per new agent (label and its three port codes) and one 16-bit
// word per equation, so an agent or an equation costs one load.
struct AsyncTpl {
  uint32_t hdr;                 // n_new | n_fresh << 8 | n_link << 16 | rule << 24
  uint32_t agent[kMaxNew];      // lab | src0 << 8 | src1 << 16 | src2 << 24
  uint16_t link[kMaxLink];      // code0 | code1 << 8
  uint32_t pad[3];
};
static_assert(sizeof(AsyncTpl) == 64, "packed template is 64 bytes");

__device__ __forceinline__ AsyncTpl pack_template(const Template& t) {
  AsyncTpl p;
  p.hdr = (uint32_t)t.n_new | ((uint32_t)t.n_fresh << 8) | ((uint32_t)t.n_link << 16) | ((uint32_t)t.rule << 24);
  for (int j = 0; j < kMaxNew; j++)
    p.agent[j] = (uint32_t)t.lab[j] | ((uint32_t)t.src[j][0] << 8) | ((uint32_t)t.src[j][1] << 16) |
                 ((uint32_t)t.src[j][2] << 24);
  for (int k = 0; k < kMaxLink; k++) p.link[k] = (uint16_t)(t.link[k][0] | (t.link[k][1] << 8));
  p.pad[0] = p.pad[1] = p.pad[2] = 0;
  return p;
}

// Port value of code c (0xFF: none) from the lane's value table.
__device__ __forceinline__ int32_t port_val(const WarpMem& W, uint32_t c, int lane) {
  return c == kValNone ? 0 : (int32_t)W.vals[c][lane];
}

// Free slots this warp holds privately: warp-uniform counts, kept in the
// registers of every lane.
struct WarpStacks {
  int ac, vc;
};

// Where one warp step's new slots come from (warp-uniform): this warp's
// stacks first (ta agent and tv name slots from abase / vbase up); when a
// stack runs dry, one global pop serves the rest of the step (ga, gv slots)
// and refills the stack with kRefill more (gra, grv).
struct PopPlan {
  uint32_t ta, tv, abase, vbase, ga, gv, gra, grv;
  unsigned long long arb, abb, vrb, vbb;
  uint32_t aav, vav;
};

// Plans the pops of Ka agent and Kv name slots (warp-collective).  Returns
// false when the arena is full (fatal: the loop stops).
__device__ __forceinline__ bool warp_pop(const Dev& d, const WarpStacks& S, uint32_t Ka, uint32_t Kv, int lane,
                                         PopPlan& P) {
  Ctrl* c = d.ctrl;
  P.ta = min((uint32_t)S.ac, Ka);
  P.tv = min((uint32_t)S.vc, Kv);
  P.abase = (uint32_t)S.ac - P.ta;
  P.vbase = (uint32_t)S.vc - P.tv;
  P.ga = Ka - P.ta;
  P.gv = Kv - P.tv;
  P.gra = P.ga ? (uint32_t)kRefill : 0u;
  P.grv = P.gv ? (uint32_t)kRefill : 0u;
  P.arb = P.abb = P.vrb = P.vbb = 0;
  P.aav = P.vav = 0;
  if (P.ga | P.gv) {
    uint32_t ok = 1;
    if (lane == 0) {
      ok = pool_pop(&c->a_head, &c->a_pub, &c->a_bump, d.cap_agents, P.ga + P.gra, &P.arb, &P.aav, &P.abb) ? 1u : 0u;
      ok &= pool_pop(&c->v_head, &c->v_pub, &c->v_bump, d.cap_vars, P.gv + P.grv, &P.vrb, &P.vav, &P.vbb) ? 1u : 0u;
      if (!ok) set_error(c, INET_ERR_ARENA_FULL, 0);
    }
    if (!__shfl_sync(kFull, ok, 0)) return false;
    P.arb = __shfl_sync(kFull, P.arb, 0);
    P.abb = __shfl_sync(kFull, P.abb, 0);
    P.aav = __shfl_sync(kFull, P.aav, 0);
    P.vrb = __shfl_sync(kFull, P.vrb, 0);
    P.vbb = __shfl_sync(kFull, P.vbb, 0);
    P.vav = __shfl_sync(kFull, P.vav, 0);
  }
  return true;
}

// The k-th agent / name slot of this warp step.
__device__ __forceinline__ uint32_t plan_agent(const Dev& d, const WarpMem& W, const PopPlan& P, uint32_t k) {
  return k < P.ta ? W.astk[P.abase + k] : pool_slot(d.afree, d.cap_agents, P.arb, P.aav, P.abb, k - P.ta);
}
__device__ __forceinline__ uint32_t plan_var(const Dev& d, const WarpMem& W, const PopPlan& P, uint32_t k) {
  return k < P.tv ? W.vstk[P.vbase + k] : pool_slot(d.vfree, d.cap_vars, P.vrb, P.vav, P.vbb, k - P.tv);
}

// After every lane has read its stack entries (warp-collective): the
// refills of the stacks, then the agent slots this step frees (free_a of
// this lane, Fa of the warp; the lane's first at offset `of`) on top of the
// agent stack, the overflow to the ring.
template <bool kTrack>
__device__ __forceinline__ void warp_settle(const Dev& d, WarpMem& W, WarpStacks& S, const PopPlan& P, uint32_t Fa,
                                            uint32_t free_a, uint32_t of, bool first_is_a, uint32_t a, uint32_t b,
                                            int lane) {
  Ctrl* c = d.ctrl;
  if (P.gra | P.grv) {
    if ((uint32_t)lane < P.gra) W.astk[P.abase + lane] = pool_slot(d.afree, d.cap_agents, P.arb, P.aav, P.abb, P.ga + lane);
    if ((uint32_t)lane < P.grv) W.vstk[P.vbase + lane] = pool_slot(d.vfree, d.cap_vars, P.vrb, P.vav, P.vbb, P.gv + lane);
  }
  const uint32_t atop = P.abase + P.gra;
  const uint32_t keep = min((uint32_t)kAStack - atop, Fa);
  if (Fa) {
    unsigned long long over = 0;
    if (Fa > keep) {
      if (lane == 0) over = atomicAdd(&c->a_tail, (unsigned long long)(Fa - keep));
      over = __shfl_sync(kFull, over, 0);
    }
    for (uint32_t f = 0; f < free_a; f++) {
      const uint32_t slot = (first_is_a && f == 0) ? a : b;
      const uint32_t k = of + f;
      if constexpr (kTrack) __stcg(&d.node[slot].head, kFreeHead);
      if (k < keep) W.astk[atop + k] = slot;
      else __stcg(d.afree + (over + (k - keep)) % d.cap_agents, slot);
    }
  }
  S.ac = (int)(atop + keep);
  S.vc = (int)(P.vbase + P.grv);
}

// Names freed while linking (warp-collective): on the warp's stack, the
// overflow to the ring.
__device__ __forceinline__ void flush_vstage(const Dev& d, WarpMem& W, WarpStacks& S, int lane) {
  __syncwarp();
  const int nst = W.vstage_n;
  if (nst) {
    const int nv = min(nst, kVStageW);
    const int keepv = min(kVStack - S.vc, nv);
    unsigned long long over = 0;
    if (lane == 0 && nv > keepv) over = atomicAdd(&d.ctrl->v_tail, (unsigned long long)(nv - keepv));
    over = __shfl_sync(kFull, over, 0);
    for (int j = lane; j < nv; j += 32) {
      if (j < keepv) W.vstk[S.vc + j] = W.vstage[j];
      else __stcg(d.vfree + (over + (unsigned long long)(j - keepv)) % d.cap_vars, W.vstage[j]);
    }
    S.vc += keepv;
    __syncwarp();
    if (lane == 0) W.vstage_n = 0;
    __syncwarp();
  }
}

// Per-net counters (interactions and the change of pending pairs) and the
// rule histogram: one fire-and-forget atomic each; with kTrack the net's
// live agents too (its quota is checked between launches).
template <bool kTrack>
__device__ __forceinline__ void count_interaction(const Dev& d, uint32_t* hist, uint32_t net, uint32_t rule,
                                                  uint32_t np, uint32_t n_new) {
  atomicAdd(d.netctr + net, 1ull + ((unsigned long long)((long long)np - 1) << kNetPairShift));
  atomicAdd(&hist[rule], 1u);
  if constexpr (kTrack) {
    if (n_new != 2) atomicAdd(reinterpret_cast<unsigned long long*>(d.netlive + net),
                              (unsigned long long)((long long)n_new - 2));
  }
}

// ->com of one lane's equations t_k = u_k, k < nl, after its new records
// (per lane, no warp-collective step).  One fence makes this lane's new
// records and fresh names visible before an exchange can publish a
// reference to them; the first exchange of each of the first kBatch
// equations is then issued back to back, and only second arrivals continue
// (rarely) with a chase.  get(k, 0) and get(k, 1) are the two sides of
// equation k.  kNL >= 0: nl is that constant (the loops unroll); -1: nl is
// known at run time.  The new active pairs go to W.out[0..return)[lane].
template <bool kTrack, int kNL, class Get>
__device__ __forceinline__ uint32_t link_lane(const Dev& d, WarpMem& W, uint32_t nl, const Get& get, int lane) {
  if constexpr (kNL >= 0) nl = (uint32_t)kNL;
  constexpr uint32_t kBatch = 2;
  uint32_t np = 0;
  __threadfence();
  uint32_t lt[kBatch], lu[kBatch], lo[kBatch];
#pragma unroll
  for (uint32_t k = 0; k < kBatch; k++) {
    lt[k] = 0;
    lu[k] = 0;
    lo[k] = kEmpty;
    if (k < nl) {
      uint32_t t = get(k, 0), u = get(k, 1);
      if (!(is_agent(t) && is_agent(u))) {
        if (!is_var(t)) {
          const uint32_t w = t;
          t = u;
          u = w;
        }
        if (is_var(t) && idx_of(t) < d.cap_vars) lo[k] = atomicExch(d.var + idx_of(t), u);
        else set_error(d.ctrl, INET_ERR_STATE, 1);
      }
      lt[k] = t;
      lu[k] = u;
    }
  }
#pragma unroll
  for (uint32_t k = 0; k < kBatch; k++) {
    if (k < nl) {
      const uint32_t t = lt[k], u = lu[k];
      if (is_agent(t) && is_agent(u)) {
        W.out[np][lane] = Pair{idx_of(t), idx_of(u)};
        np++;
      } else if (lo[k] != kEmpty && is_var(t)) {
        // second arrival: the slot is finished; continue with old = u
        release_name<kTrack>(d, W, idx_of(t));
        Pair out;
        if (link_async<kTrack>(d, W, lo[k], u, &out)) {
          W.out[np][lane] = out;
          np++;
        }
      }
    }
  }
  if constexpr (kNL >= 0) {
#pragma unroll
    for (uint32_t k = kBatch; k < (uint32_t)kNL; k++) {
      Pair out;
      if (link_async<kTrack>(d, W, get(k, 0), get(k, 1), &out)) {
        W.out[np][lane] = out;
        np++;
      }
    }
  } else {
    for (uint32_t k = kBatch; k < nl; k++) {
      Pair out;
      if (link_async<kTrack>(d, W, get(k, 0), get(k, 1), &out)) {
        W.out[np][lane] = out;
        np++;
      }
    }
  }
  return np;
}

// The rule set a kernel is specialised for: kN templates known at compile
// time (kT, in rule-table order) and kKey, the hash of their bytes the host
// passes in Dev::rules_key.  NoRules (kN = 0): the general kernel, which
// reads the templates from shared memory.
struct NoRules {
  static constexpr int kN = 0;
  static constexpr unsigned long long kKey = 0;
  static constexpr Template kT[1] = {};
};

// Instantiation of rule I of a specialised rule set for one lane (Sec. 2.2,
// ->int, then ->com of Theta'): the template is a constant, so the values
// live in registers and every loop over agents, ports, names and equations
// is unrolled.  Slots: the lane's agents beyond the two it reuses start at
// offset oa of the warp's step, its fresh names at ov (taken from the
// warp's stacks below ta / tv, the rest from the global pops).  The linking
// is written out here rather than shared with the general path: the
// compiler then keeps each equation's known cases (a new agent is an agent,
// a fresh name a name) apart.
template <bool kTrack, class Rules, int I>
__device__ __forceinline__ uint32_t rule_body(const Dev& d, WarpMem& W, const int4& ra, const int4& rb, uint32_t a,
                                              uint32_t b, uint32_t net, uint32_t oa, uint32_t ov, uint32_t ta,
                                              uint32_t tv, uint32_t abase, uint32_t vbase, unsigned long long arb,
                                              uint32_t aav, unsigned long long abb, unsigned long long vrb,
                                              uint32_t vav, unsigned long long vbb, int lane, bool& valid) {
  constexpr Template R = Rules::kT[I];
  Ctrl* c = d.ctrl;
  uint32_t v[kNumVals];
  v[kValExt + 0] = (uint32_t)ra.y;
  v[kValExt + 1] = (uint32_t)ra.z;
  v[kValExt + 2] = (uint32_t)ra.w;
  v[kValExt + 3] = (uint32_t)rb.y;
  v[kValExt + 4] = (uint32_t)rb.z;
  v[kValExt + 5] = (uint32_t)rb.w;
#pragma unroll
  for (int j = kValNew; j < kNumVals; j++) v[j] = 0;
  bool in_range = true;
  if (R.n_new > 0) v[kValNew + 0] = mk_agent(a);
  if (R.n_new > 1) v[kValNew + 1] = mk_agent(b);
#pragma unroll
  for (int j = 2; j < (int)R.n_new; j++) {
    const uint32_t k = oa + (uint32_t)j - 2;
    const uint32_t sl = k < ta ? W.astk[abase + k] : pool_slot(d.afree, d.cap_agents, arb, aav, abb, k - ta);
    if (sl >= d.cap_agents) in_range = false;
    v[kValNew + j] = mk_agent(sl);
  }
#pragma unroll
  for (int f = 0; f < (int)R.n_fresh; f++) {
    const uint32_t k = ov + (uint32_t)f;
    const uint32_t x = k < tv ? W.vstk[vbase + k] : pool_slot(d.vfree, d.cap_vars, vrb, vav, vbb, k - tv);
    if (x >= d.cap_vars) {
      in_range = false;
    } else {
      __stcg(d.var + x, kEmpty);  // a fresh name starts empty; published by this lane's fence
      if constexpr (kTrack) __stcg(d.vown + x, net);
    }
    v[kValFresh + f] = mk_var(x);
  }
  if (!in_range) {
    set_error(c, INET_ERR_STATE, 4);
    valid = false;
    return 0u;
  }
  const uint32_t head_net = net << 8;
#pragma unroll
  for (int j = 0; j < (int)R.n_new; j++) {
    int4 rec;
    rec.x = (int32_t)(head_net | R.lab[j]);
    rec.y = R.src[j][0] == kValNone ? 0 : (int32_t)v[R.src[j][0]];
    rec.z = R.src[j][1] == kValNone ? 0 : (int32_t)v[R.src[j][1]];
    rec.w = R.src[j][2] == kValNone ? 0 : (int32_t)v[R.src[j][2]];
    st_node(d.node + idx_of(v[kValNew + j]), rec);
  }
  // ->com: the fence, the first exchanges of the first kBatch equations back
  // to back, then their second arrivals, then the other equations
  constexpr uint32_t kBatch = 2;
  uint32_t np = 0;
  if (R.n_link) __threadfence();
  uint32_t lt[kBatch], lu[kBatch], lo[kBatch];
#pragma unroll
  for (uint32_t k = 0; k < kBatch; k++) {
    lt[k] = 0;
    lu[k] = 0;
    lo[k] = kEmpty;
    if (k < R.n_link) {
      uint32_t t = v[R.link[k][0]], u = v[R.link[k][1]];
      if (!(is_agent(t) && is_agent(u))) {
        if (!is_var(t)) {
          const uint32_t w = t;
          t = u;
          u = w;
        }
        if (is_var(t) && idx_of(t) < d.cap_vars) lo[k] = atomicExch(d.var + idx_of(t), u);
        else set_error(c, INET_ERR_STATE, 1);
      }
      lt[k] = t;
      lu[k] = u;
    }
  }
#pragma unroll
  for (uint32_t k = 0; k < kBatch; k++) {
    if (k < R.n_link) {
      const uint32_t t = lt[k], u = lu[k];
      if (is_agent(t) && is_agent(u)) {
        W.out[np][lane] = Pair{idx_of(t), idx_of(u)};
        np++;
      } else if (lo[k] != kEmpty && is_var(t)) {
        release_name<kTrack>(d, W, idx_of(t));
        Pair out;
        if (link_async<kTrack>(d, W, lo[k], u, &out)) {
          W.out[np][lane] = out;
          np++;
        }
      }
    }
  }
#pragma unroll
  for (uint32_t k = kBatch; k < R.n_link; k++) {
    Pair out;
    if (link_async<kTrack>(d, W, v[R.link[k][0]], v[R.link[k][1]], &out)) {
      W.out[np][lane] = out;
      np++;
    }
  }
  return np;
}

// Rule I continues as a chain of itself when one of its equations joins an
// external port to a new agent of one of its own left-hand side's symbols:
// Add(y, w) = x of Add(y, r) = S(x) -> Add(y, w) = x, r = S(w), where an
// agent x in the port makes (Add', x) the next active pair, often of the
// same rule.
template <class Rules, int I>
__host__ __device__ constexpr bool chain_rule() {
  if constexpr (I < Rules::kN) {
    constexpr Template R = Rules::kT[I];
    for (int k = 0; k < R.n_link; k++) {
      const int c0 = R.link[k][0], c1 = R.link[k][1];
      const bool e0 = c0 < kValNew, e1 = c1 < kValNew;
      const bool n0 = c0 >= kValNew && c0 < kValFresh, n1 = c1 >= kValNew && c1 < kValFresh;
      if ((e0 && n1) || (n0 && e1)) {
        const int lab = R.lab[(e0 ? c1 : c0) - kValNew];
        if (lab == R.lhs[0] || lab == R.lhs[1]) return true;
      }
    }
  }
  return false;
}

constexpr int kLoneMax = 32;  // steps of one lone or uniform run before the warp's loop resumes

// A warp whose valid lanes all reduce rule I of a specialised rule set (the
// common case: one lane alone on a chain, or a batch of like pairs): the
// whole step with that rule's template as a constant.  Every lane needs the
// same slots, so a lane's offsets among the warp's needs are its rank among
// the valid lanes times the rule's counts, with no scan.
//
// Uniform runs: when `quiet` (no lane waits for a ticket and the queue was
// empty when the warp last looked), the rule continues as a chain of itself
// and every valid lane's step left exactly one new pair, of rule I again,
// the warp steps again at once with those pairs, without its loop between
// (up to kLoneMax steps): nothing is handed on, the count of pairs in flight
// does not change.  A warp with one valid lane leaves this to lone_chain.
template <bool kTrack, class Rules, int I>
__device__ __forceinline__ uint32_t uni_interact(const Dev& d, const int16_t* tab, uint32_t* hist, WarpMem& W,
                                                 WarpStacks& S, bool valid, unsigned vmask, uint32_t a, uint32_t b,
                                                 int4 ra, int4 rb, uint32_t net, long long& live, bool quiet) {
  constexpr Template R = Rules::kT[I];
  constexpr uint32_t NN = R.n_new, NF = R.n_fresh;
  constexpr uint32_t NA = NN > 2 ? NN - 2 : 0u, FA = NN < 2 ? 2 - NN : 0u;
  const int lane = threadIdx.x & 31;
  Ctrl* c = d.ctrl;
  const uint32_t nvl = __popc(vmask), rank = __popc(vmask & lanemask_lt());
  const uint32_t Ka = nvl * NA, Kv = nvl * NF, Fa = nvl * FA;
  const uint32_t oa = rank * NA, ov = rank * NF, of = rank * FA;
  uint32_t np = 0;
  for (int it = 0;; it++) {
    const uint32_t ta = min((uint32_t)S.ac, Ka), tv = min((uint32_t)S.vc, Kv);
    const uint32_t abase = (uint32_t)S.ac - ta, vbase = (uint32_t)S.vc - tv;
    const uint32_t ga = Ka - ta, gv = Kv - tv;
    const uint32_t gra = ga ? (uint32_t)kRefill : 0u, grv = gv ? (uint32_t)kRefill : 0u;
    unsigned long long arb = 0, abb = 0, vrb = 0, vbb = 0;
    uint32_t aav = 0, vav = 0;
    if (ga | gv) {
      uint32_t ok = 1;
      if (lane == 0) {
        ok = pool_pop(&c->a_head, &c->a_pub, &c->a_bump, d.cap_agents, ga + gra, &arb, &aav, &abb) ? 1u : 0u;
        ok &= pool_pop(&c->v_head, &c->v_pub, &c->v_bump, d.cap_vars, gv + grv, &vrb, &vav, &vbb) ? 1u : 0u;
        if (!ok) set_error(c, INET_ERR_ARENA_FULL, 0);
      }
      if (!__shfl_sync(kFull, ok, 0)) return 0u;  // fatal: the loop stops
      arb = __shfl_sync(kFull, arb, 0);
      abb = __shfl_sync(kFull, abb, 0);
      aav = __shfl_sync(kFull, aav, 0);
      vrb = __shfl_sync(kFull, vrb, 0);
      vbb = __shfl_sync(kFull, vbb, 0);
      vav = __shfl_sync(kFull, vav, 0);
    }
    if (lane == 0) live += (long long)Ka - (long long)Fa;
    const bool frees = valid;  // counted in Fa: freed even if the step fails below
    np = 0;
    if (valid)
      np = rule_body<kTrack, Rules, I>(d, W, ra, rb, a, b, net, oa, ov, ta, tv, abase, vbase, arb, aav, abb, vrb,
                                       vav, vbb, lane, valid);
    __syncwarp();  // every taken stack entry has been read
    if (gra | grv) {
      if ((uint32_t)lane < gra) W.astk[abase + lane] = pool_slot(d.afree, d.cap_agents, arb, aav, abb, ga + lane);
      if ((uint32_t)lane < grv) W.vstk[vbase + lane] = pool_slot(d.vfree, d.cap_vars, vrb, vav, vbb, gv + lane);
    }
    const uint32_t atop = abase + gra;
    const uint32_t keep = min((uint32_t)kAStack - atop, Fa);
    if (FA && Fa) {
      unsigned long long over = 0;
      if (Fa > keep) {
        if (lane == 0) over = atomicAdd(&c->a_tail, (unsigned long long)(Fa - keep));
        over = __shfl_sync(kFull, over, 0);
      }
      if (frees) {
#pragma unroll
        for (uint32_t f = 0; f < FA; f++) {
          const uint32_t slot = (NN == 0 && f == 0) ? a : b;
          const uint32_t k = of + f;
          if constexpr (kTrack) __stcg(&d.node[slot].head, kFreeHead);
          if (k < keep) W.astk[atop + k] = slot;
          else __stcg(d.afree + (over + (k - keep)) % d.cap_agents, slot);
        }
      }
    }
    S.ac = (int)(atop + keep);
    S.vc = (int)(vbase + grv);
    flush_vstage(d, W, S, lane);
    if (valid) count_interaction<kTrack>(d, hist, net, R.rule, np, NN);
    if constexpr (!chain_rule<Rules, I>()) {
      break;
    } else {
      // every lane's chain goes on with another pair of rule I: the warp
      // steps again without its loop (the records read here are wasted when
      // some lane's next pair is of another rule: once at the end of a chain)
      if (!quiet || nvl == 1 || it + 1 >= kLoneMax || !__all_sync(kFull, !valid || np == 1)) break;
      bool ok = true;
      if (valid) {
        ok = false;
        const Pair p = W.out[0][lane];
        if (p.a < d.cap_agents && p.b < d.cap_agents) {
          const int4 pra = ld_node(d.node + p.a), prb = ld_node(d.node + p.b);
          const uint32_t la = (uint32_t)pra.x & 0xFFu, lb = (uint32_t)prb.x & 0xFFu;
          const int e = (la < d.n_labels && lb < d.n_labels) ? tab[la * d.n_labels + lb] : -1;
          if (e >= 0 && ((uint32_t)e >> 1) == (uint32_t)I) {
            if (e & 1) {
              ra = prb;
              rb = pra;
              a = p.b;
              b = p.a;
            } else {
              ra = pra;
              rb = prb;
              a = p.a;
              b = p.b;
            }
            net = (uint32_t)ra.x >> 8;
            ok = net < d.max_nets;
          }
        }
      }
      if (!__all_sync(kFull, ok)) break;
    }
  }
  return valid ? np : 0u;
}

// Rule I of a specialised rule set, when the rule set has one and I's
// right-hand side has at most two agents (it reuses the pair's two slots:
// the rules that carry chains, Add(y, r) = S(x) and the like).  Larger
// rules stay on the general code: their own copies cost more in instruction
// fetch than they save (2048 Mul nets: 10.9 ms with rules of up to two
// agents, 11.0 ms up to three, 11.2 ms with every rule; only up to one
// leaves the Add chains out and gives no gain).

// A warp in which one lane holds a pair (no lane waits for a ticket, and the
// queue was empty when the warp last looked), of a rule that continues as a
// chain of itself: the lane runs up to kLoneMax interactions of that rule on
// its own, without the warp's loop between them.  Each leaves exactly one
// new pair, the chain's next, so nothing is handed on and the count of pairs
// in flight does not change.  The run stops when an interaction leaves no
// pair or several (returned as after any step, W.out filled), when the next
// pair is of another rule or its slots are not on the warp's stacks (it is
// then the lane's next pair), or after kLoneMax interactions.  Slots come
// from and return to the warp's stacks, names freed while linking too;
// counters per interaction as in the warp's step.  (Loading the next
// pair's records before an interaction's fence and exchanges returned, or
// handing the records this run loaded back to the warp's loop, was slower.)
template <bool kTrack, class Rules, int I>
__device__ __forceinline__ uint32_t lone_chain(const Dev& d, const int16_t* tab, uint32_t* hist, WarpMem& W,
                                               WarpStacks& S, bool valid, uint32_t a, uint32_t b, int4 ra, int4 rb,
                                               uint32_t net, long long& live) {
  constexpr Template R = Rules::kT[I];
  constexpr uint32_t NN = R.n_new, NF = R.n_fresh;
  constexpr uint32_t NA = NN > 2 ? NN - 2 : 0u, FA = NN < 2 ? 2 - NN : 0u;
  const int lane = threadIdx.x & 31;
  Ctrl* c = d.ctrl;
  const unsigned vm = __ballot_sync(kFull, valid);
  const int src = vm ? __ffs(vm) - 1 : 0;
  uint32_t np = 0;
  int ac = S.ac, vc = S.vc;
  long long dl = 0;
  if (valid) {
    for (int it = 0;; it++) {
      np = rule_body<kTrack, Rules, I>(d, W, ra, rb, a, b, net, 0u, 0u, NA, NF, (uint32_t)ac - NA,
                                       (uint32_t)vc - NF, 0ull, 0u, 0ull, 0ull, 0u, 0ull, lane, valid);
      ac -= (int)NA;
      vc -= (int)NF;
#pragma unroll
      for (uint32_t f = 0; f < FA; f++) {
        const uint32_t slot = (NN == 0 && f == 0) ? a : b;
        if constexpr (kTrack) __stcg(&d.node[slot].head, kFreeHead);
        if (ac < kAStack) {
          W.astk[ac++] = slot;
        } else {
          const unsigned long long tp = atomicAdd(&c->a_tail, 1ull);
          __stcg(d.afree + tp % d.cap_agents, slot);
        }
      }
      dl += (long long)NA - (long long)FA;
      // names freed while linking: this lane is the only user of the warp's stacks
      const int nst = min(W.vstage_n, kVStageW);
      for (int j = 0; j < nst; j++) {
        if (vc < kVStack) {
          W.vstk[vc++] = W.vstage[j];
        } else {
          const unsigned long long tp = atomicAdd(&c->v_tail, 1ull);
          __stcg(d.vfree + tp % d.cap_vars, W.vstage[j]);
        }
      }
      W.vstage_n = 0;
      if (!valid) break;
      count_interaction<kTrack>(d, hist, net, R.rule, np, NN);
      if (np != 1 || it + 1 >= kLoneMax) break;
      // the one new pair: the chain's next if it is of rule I again
      const Pair p = W.out[0][lane];
      if (p.a >= d.cap_agents || p.b >= d.cap_agents) break;
      const int4 pra = ld_node(d.node + p.a), prb = ld_node(d.node + p.b);
      const uint32_t la = (uint32_t)pra.x & 0xFFu, lb = (uint32_t)prb.x & 0xFFu;
      const int e = (la < d.n_labels && lb < d.n_labels) ? tab[la * d.n_labels + lb] : -1;
      if (e < 0 || ((uint32_t)e >> 1) != (uint32_t)I || ac < (int)NA || vc < (int)NF) break;
      if (e & 1) {
        ra = prb;
        rb = pra;
        a = p.b;
        b = p.a;
      } else {
        ra = pra;
        rb = prb;
        a = p.a;
        b = p.b;
      }
      net = (uint32_t)ra.x >> 8;
      if (net >= d.max_nets) break;  // left to the warp's step, which reports it
    }
  }
  __syncwarp();
  S.ac = __shfl_sync(kFull, ac, src);
  S.vc = __shfl_sync(kFull, vc, src);
  const long long dls = __shfl_sync(kFull, dl, src);
  if (lane == 0) live += dls;
  return valid ? np : 0u;
}

// The warp's stacks hold the slots of one interaction of rule I.
template <class Rules, int I>
__device__ __forceinline__ bool lone_slots(const WarpStacks& S) {
  constexpr uint32_t NN = Rules::kT[I].n_new;
  return S.ac >= (int)(NN > 2 ? NN - 2 : 0) && S.vc >= (int)Rules::kT[I].n_fresh;
}

constexpr int kSpecialisedMaxNew = 2;
// At most this many rules get their own code (the first in rule-table
// order): every one adds to the run-time compile (up to about a second each:
// a rule set of 64 rules compiles in about 33 s, once) and to the kernel's
// code.
constexpr int kSpecialisedMaxRules = 32;
// Bit I set: rule I has its own code.
template <class Rules>
__host__ __device__ constexpr unsigned long long spec_mask() {
  unsigned long long m = 0;
  int k = 0;
  for (int i = 0; i < Rules::kN && k < kSpecialisedMaxRules; i++)
    if (Rules::kT[i].n_new <= kSpecialisedMaxNew) {
      m |= 1ull << i;
      k++;
    }
  return m;
}
template <class Rules, int I>
__host__ __device__ constexpr bool specialised() {
  return I < Rules::kN && ((spec_mask<Rules>() >> I) & 1ull);
}
#define INET_UNI_CASE(I)                                                                                   \
  case I:                                                                                                  \
    if constexpr (specialised<Rules, I>()) {                                                               \
      if constexpr (chain_rule<Rules, I>()) {                                                              \
        if (lone && lone_slots<Rules, I>(S))                                                               \
          return lone_chain<kTrack, Rules, I>(d, tab, hist, W, S, valid, a, b, ra, rb, net, live);         \
      }                                                                                                    \
      return uni_interact<kTrack, Rules, I>(d, tab, hist, W, S, valid, vmask, a, b, ra, rb, net, live, quiet); \
    }                                                                                                      \
    break;

// One interaction per lane whose `valid` is set (warp-collective).  The new
// active pairs are left in W.out[0..return)[lane]; a pair that cannot be
// reduced (no rule, corrupt state) is dropped and returns 0.  Lane 0's
// `live` collects the change of live agents.  With a specialised rule set,
// a warp whose lanes all reduce the same rule takes that rule's own code;
// any other warp (and the general kernel always) interprets the templates
// in shared memory.
template <bool kTrack, class Rules>
__device__ __forceinline__ uint32_t async_interact(const Dev& d, const AsyncTpl* tmpl, const int16_t* tab,
                                                   uint32_t* hist, WarpMem& W, WarpStacks& S, bool valid,
                                                   uint32_t a, uint32_t b, long long& live, bool pre,
                                                   int4 pra, int4 prb, bool lone, bool quiet) {
  const int lane = threadIdx.x & 31;
  Ctrl* c = d.ctrl;
  uint32_t net = 0, ti = 0;
  int4 ra = make_int4(0, 0, 0, 0), rb = ra;
  if (valid && (a >= d.cap_agents || b >= d.cap_agents)) {
    set_error(c, INET_ERR_STATE, 2);
    valid = false;
  }
  if (valid) {
    if (pre) {
      ra = pra;
      rb = prb;
    } else {
      ra = ld_node(d.node + a);
      rb = ld_node(d.node + b);
    }
    const uint32_t la = (uint32_t)ra.x & 0xFFu, lb = (uint32_t)rb.x & 0xFFu;
    const int e = (la < d.n_labels && lb < d.n_labels) ? tab[la * d.n_labels + lb] : -1;
    net = (uint32_t)ra.x >> 8;
    if (net >= d.max_nets) {
      set_error(c, INET_ERR_STATE, 3);
      valid = false;
    } else if (e < 0) {
      valid = false;
      atomicCAS(d.netstat + net, 0, INET_ERR_NO_RULE);
      set_error(c, INET_ERR_NO_RULE, net);
      atomicAdd(d.netctr + net, (unsigned long long)(-(1ll << kNetPairShift)));
    } else {
      if (e & 1) {
        int4 t = ra; ra = rb; rb = t;
        uint32_t u = a; a = b; b = u;
      }
      ti = (uint32_t)e >> 1;
    }
  }
  if constexpr (Rules::kN > 0) {
    const unsigned vmask = __ballot_sync(kFull, valid);
    const uint32_t lead = __shfl_sync(kFull, ti, vmask ? __ffs(vmask) - 1 : 0);
    if (vmask && ((spec_mask<Rules>() >> lead) & 1ull) && __all_sync(kFull, !valid || ti == lead)) {
      switch (lead) {
        INET_UNI_CASE(0) INET_UNI_CASE(1) INET_UNI_CASE(2) INET_UNI_CASE(3) INET_UNI_CASE(4) INET_UNI_CASE(5)
        INET_UNI_CASE(6) INET_UNI_CASE(7) INET_UNI_CASE(8) INET_UNI_CASE(9) INET_UNI_CASE(10) INET_UNI_CASE(11)
        INET_UNI_CASE(12) INET_UNI_CASE(13) INET_UNI_CASE(14) INET_UNI_CASE(15) INET_UNI_CASE(16) INET_UNI_CASE(17)
        INET_UNI_CASE(18) INET_UNI_CASE(19) INET_UNI_CASE(20) INET_UNI_CASE(21) INET_UNI_CASE(22) INET_UNI_CASE(23)
        INET_UNI_CASE(24) INET_UNI_CASE(25) INET_UNI_CASE(26) INET_UNI_CASE(27) INET_UNI_CASE(28) INET_UNI_CASE(29)
        INET_UNI_CASE(30) INET_UNI_CASE(31) INET_UNI_CASE(32) INET_UNI_CASE(33) INET_UNI_CASE(34) INET_UNI_CASE(35)
        INET_UNI_CASE(36) INET_UNI_CASE(37) INET_UNI_CASE(38) INET_UNI_CASE(39) INET_UNI_CASE(40) INET_UNI_CASE(41)
        INET_UNI_CASE(42) INET_UNI_CASE(43) INET_UNI_CASE(44) INET_UNI_CASE(45) INET_UNI_CASE(46) INET_UNI_CASE(47)
        INET_UNI_CASE(48) INET_UNI_CASE(49) INET_UNI_CASE(50) INET_UNI_CASE(51) INET_UNI_CASE(52) INET_UNI_CASE(53)
        INET_UNI_CASE(54) INET_UNI_CASE(55) INET_UNI_CASE(56) INET_UNI_CASE(57) INET_UNI_CASE(58) INET_UNI_CASE(59)
        INET_UNI_CASE(60) INET_UNI_CASE(61) INET_UNI_CASE(62) INET_UNI_CASE(63)
        default: break;
      }
    }
  }
  static_assert(INET_MAX_RULES == 64, "one case per rule");
  const AsyncTpl& T = tmpl[ti];
  const uint32_t hdr = valid ? T.hdr : 0u;
  const uint32_t n_new = hdr & 0xFFu, n_fresh = (hdr >> 8) & 0xFFu, n_link = (hdr >> 16) & 0xFFu;
  const uint32_t need_a = n_new > 2 ? n_new - 2 : 0u;
  const uint32_t free_a = valid && n_new < 2 ? 2 - n_new : 0u;
  // a3: offsets of this lane among the warp's needs (10 bits per field;
  // a warp needs at most 32 x 8)
  const uint32_t packed = need_a | (n_fresh << 10) | (free_a << 20);
  uint32_t inc = packed;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += t;
  }
  const uint32_t tot = __shfl_sync(kFull, inc, 31), ex = inc - packed;
  const uint32_t Ka = tot & 1023u, Kv = (tot >> 10) & 1023u, Fa = tot >> 20;
  const uint32_t oa = ex & 1023u, ov = (ex >> 10) & 1023u, of = ex >> 20;
  PopPlan P;
  if (!warp_pop(d, S, Ka, Kv, lane, P)) return 0u;
  if (lane == 0) live += (long long)Ka - (long long)Fa;
  if (valid) {
    W.vals[kValExt + 0][lane] = (uint32_t)ra.y;
    W.vals[kValExt + 1][lane] = (uint32_t)ra.z;
    W.vals[kValExt + 2][lane] = (uint32_t)ra.w;
    W.vals[kValExt + 3][lane] = (uint32_t)rb.y;
    W.vals[kValExt + 4][lane] = (uint32_t)rb.z;
    W.vals[kValExt + 5][lane] = (uint32_t)rb.w;
    bool in_range = true;
    if (n_new > 0) W.vals[kValNew + 0][lane] = mk_agent(a);
    if (n_new > 1) W.vals[kValNew + 1][lane] = mk_agent(b);
    for (uint32_t j = 2; j < n_new; j++) {
      const uint32_t sl = plan_agent(d, W, P, oa + j - 2);
      if (sl >= d.cap_agents) in_range = false;
      W.vals[kValNew + j][lane] = mk_agent(sl);
    }
    for (uint32_t v = 0; v < n_fresh; v++) {
      const uint32_t x = plan_var(d, W, P, ov + v);
      if (x >= d.cap_vars) {
        in_range = false;
      } else {
        __stcg(d.var + x, kEmpty);  // a fresh name starts empty; published by this lane's fence
        if constexpr (kTrack) __stcg(d.vown + x, net);
      }
      W.vals[kValFresh + v][lane] = mk_var(x);
    }
    if (!in_range) {
      set_error(c, INET_ERR_STATE, 4);
      valid = false;
    }
  }
  __syncwarp();  // every taken stack entry has been read
  warp_settle<kTrack>(d, W, S, P, Fa, free_a, of, n_new == 0, a, b, lane);
  // a2: the new agents' records
  uint32_t np = 0;
  if (valid) {
    const uint32_t head_net = net << 8;
    for (uint32_t j = 0; j < n_new; j++) {
      const uint32_t w = T.agent[j];
      int4 rec;
      rec.x = (int32_t)(head_net | (w & 0xFFu));
      rec.y = port_val(W, (w >> 8) & 0xFFu, lane);
      rec.z = port_val(W, (w >> 16) & 0xFFu, lane);
      rec.w = port_val(W, w >> 24, lane);
      st_node(d.node + idx_of(W.vals[kValNew + j][lane]), rec);
    }
    // a4: link
    if (n_link)
      np = link_lane<kTrack, -1>(d, W, n_link, [&](uint32_t k, int s) {
        const uint32_t lk = T.link[k];
        return W.vals[s ? lk >> 8 : lk & 0xFFu][lane];
      }, lane);
  }
  flush_vstage(d, W, S, lane);
  if (valid) count_interaction<kTrack>(d, hist, net, hdr >> 24, np, n_new);
  return valid ? np : 0u;
}
#undef INET_UNI_CASE

// Writes a pair back to the exit frontier (other buffer).
__device__ __forceinline__ void exit_pair(const Dev& d, Pair p) {
  const uint32_t k = atomicAdd(&d.ctrl->aexit, 1u);
  if (k < d.cap_pairs) {
    __stcg(reinterpret_cast<unsigned long long*>(d.front[d.qcur ^ 1u] + k), *reinterpret_cast<unsigned long long*>(&p));
  } else {
    set_error(d.ctrl, INET_ERR_ARENA_FULL, 5);
  }
}

// A lane that claimed a ticket takes its pair as soon as it is published
// and frees the cell for the next lap.  Every wait of the asynchronous loop
// does this too, so a producer waiting for a cell never waits on a lane
// that is itself waiting.
__device__ __forceinline__ void poll_ticket(const Dev& d, const Pair* Q, bool& have, unsigned long long& ticket,
                                            unsigned long long tslot, uint32_t& pa, uint32_t& pb) {
  if (!have && ticket != kNoTicket) {
    unsigned long long* sq = d.qseq + tslot;
    if (ld_acquire64(sq) == ticket + 1) {
      const unsigned long long v = __ldcg(reinterpret_cast<const unsigned long long*>(Q + tslot));
      st_release64(sq, ticket + d.cap_pairs);
      pa = (uint32_t)v;
      pb = (uint32_t)(v >> 32);
      have = true;
      ticket = kNoTicket;
    }
  }
}

// Bounded wait for ticket t's pair (when no producer runs any more);
// returns false on timeout.
__device__ __forceinline__ bool wait_ticket(const Dev& d, const Pair* Q, unsigned long long t, Pair* out) {
  const unsigned long long s = t % d.cap_pairs;
  const unsigned long long t0 = globaltimer();
  for (uint32_t spin = 0;; spin++) {
    if (ld_acquire64(d.qseq + s) == t + 1) {
      const unsigned long long v = __ldcg(reinterpret_cast<const unsigned long long*>(Q + s));
      *out = Pair{(uint32_t)v, (uint32_t)(v >> 32)};
      return true;
    }
    __nanosleep(64);
    if ((spin & 63) == 63 && globaltimer() - t0 > d.timeout_ns) {
      set_error(d.ctrl, INET_ERR_TIMEOUT, 6);
      return false;
    }
  }
}

template <bool kTrack, class Rules = NoRules>
__global__ void __launch_bounds__(256, 2) k_async(Dev d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  size_t off = 0;
  auto take = [&](size_t n) { off = (off + 15) / 16 * 16; unsigned char* p = smem_raw + off; off += n; return p; };
  AsyncTpl* tmpl = reinterpret_cast<AsyncTpl*>(take(sizeof(AsyncTpl) * (d.n_tmpl ? d.n_tmpl : 1)));
  WarpMem* wm = reinterpret_cast<WarpMem*>(take(sizeof(WarpMem) * (blockDim.x / 32)));
  uint32_t* hist = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * INET_MAX_RULES));
  int16_t* tab = reinterpret_cast<int16_t*>(take(sizeof(int16_t) * d.n_labels * d.n_labels));
  for (uint32_t i = threadIdx.x; i < d.n_tmpl; i += blockDim.x) tmpl[i] = pack_template(d.tmpl[i]);
  for (uint32_t i = threadIdx.x; i < d.n_labels * d.n_labels; i += blockDim.x) tab[i] = d.table[i];
  for (uint32_t i = threadIdx.x; i < INET_MAX_RULES; i += blockDim.x) hist[i] = 0;
  if constexpr (Rules::kN > 0) {
    // a specialised kernel runs only on the rule set it was built for (the
    // check sits after the carve-up of shared memory: at the top of the
    // kernel it cost the loop 6 more registers)
    if (d.rules_key != Rules::kKey || d.n_tmpl != (uint32_t)Rules::kN) {
      if (threadIdx.x == 0 && blockIdx.x == 0) set_error(d.ctrl, INET_ERR_STATE, 10);
      return;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpMem& W = wm[wid];
  if (lane == 0) W.vstage_n = 0;
  WarpStacks S{0, 0};
  __syncthreads();
  Ctrl* c = d.ctrl;
  Pair* Q = d.front[d.qcur];
  const unsigned long long cap = d.cap_pairs;
  const uint32_t total_warps = gridDim.x * (blockDim.x / 32);
  bool have = false;
  uint32_t pa = 0, pb = 0;
  unsigned long long ticket = kNoTicket, tslot = 0;
  long long live = 0;
  uint32_t nap = 0;
  bool stop = false, finished = false, check_now = false;
  bool pre = false;
  bool qseen = false;  // the queue held pairs when this warp last looked
  int4 pra = make_int4(0, 0, 0, 0), prb = pra;
  unsigned long long t_start = 0;
  if (lane == 0) {
    const unsigned long long now = globaltimer();
    atomicCAS(&c->slice_t0, 0ull, now);
    t_start = ld_volatile64(&c->slice_t0);
  }
  for (uint32_t it = 0;; it++) {
    // stop / slice checks every 16 iterations, and when a napping warp's
    // clock says the time slice is over
    if ((it & 15) == 15 || check_now) {
      check_now = false;
      uint32_t st = 0;
      if (lane == 0) {
        st = ld_volatile(&c->astop) | (ld_volatile((const uint32_t*)&c->fatal) ? 1u : 0u);
        if (!st && globaltimer() - t_start > d.slice_ns) {
          c->astop = 1;
          c->hit_slice = 1;
          st = 1;
        }
      }
      if (__shfl_sync(kFull, st, 0)) {
        stop = true;
        break;
      }
    }
    // claim tickets for lanes without work when the queue has unclaimed
    // pairs.  While the queue holds fewer pairs than there are warps, only a
    // warp with no work claims, and one ticket at a time: each queued pair,
    // and the chain of interactions it starts, gets a warp of its own (with
    // idle lanes for the pairs it hands on) instead of sharing one with up
    // to 31 others, whose divergent work would slow every lane (2048 Mul
    // nets: 14.5 -> 12.9 ms with the grid at full occupancy).  A longer
    // queue is drained by every warp, busy ones looking every 8th iteration.
    const unsigned want = __ballot_sync(kFull, !have && ticket == kNoTicket);
    const unsigned busy = __ballot_sync(kFull, have);
    if (want && (!busy || (it & 7) == 0)) {
      unsigned long long base = 0;
      uint32_t k = 0, qs = 0;
      if (lane == 0) {
        unsigned long long qh, qt;
        asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(qh), "=l"(qt) : "l"(&c->q_head) : "memory");
        const unsigned long long backlog = qt > qh ? qt - qh : 0ull;
        qs = backlog ? 1u : 0u;
        const bool deep = backlog > total_warps;
        if (backlog && (!busy || deep)) {
          k = (uint32_t)min(min((unsigned long long)__popc(want), backlog), deep ? 32ull : 1ull);
          base = atomicAdd(&c->q_head, (unsigned long long)k);
        }
      }
      k = __shfl_sync(kFull, k, 0);
      qseen = __shfl_sync(kFull, qs, 0) != 0;
      if (k) {
        unsigned long long bm = 0;
        if (lane == 0) bm = base % cap;
        base = __shfl_sync(kFull, base, 0);
        bm = __shfl_sync(kFull, bm, 0);
        const unsigned rank = __popc(want & lanemask_lt());
        if (((want >> lane) & 1u) && rank < k) {
          ticket = base + rank;
          tslot = bm + rank;
          if (tslot >= cap) tslot %= cap;
        }
      }
    }
    poll_ticket(d, Q, have, ticket, tslot, pa, pb);
    const unsigned act = __ballot_sync(kFull, have);
    if (!act) {
      // idle: the loop is over when no pair is left anywhere
      uint32_t fin = 0;
      if (lane == 0) fin = ld_volatile_s64(&c->inflight) == 0 ? 1u : 0u;
      if (__shfl_sync(kFull, fin, 0)) {
        finished = true;
        break;
      }
      // back off up to 16 us: with thousands of warps, most of them idle
      // in a narrow phase, shorter naps make their polling of the queue and
      // of the in-flight count contend with the warps doing the work (an
      // Ackermann batch 77 -> 63 ms, 2048 Mul nets 13.1 -> 12.7 ms).  The
      // slice's end is noticed from the clock, which needs no memory access.
      __nanosleep(nap);
      nap = nap < 16384 ? nap * 2 + 32 : 16384;
      {
        uint32_t late = 0;
        if (lane == 0) late = globaltimer() - t_start > d.slice_ns ? 1u : 0u;
        check_now = __shfl_sync(kFull, late, 0) != 0;
      }
      continue;
    }
    nap = 0;
    // no lane waits for a ticket and the queue was empty when the warp last
    // looked: chains may run without the warp's loop (queued work is left to
    // the loop, whose idle lanes claim it); lone: one lane holds a pair
    const bool quiet = !qseen && __ballot_sync(kFull, ticket != kNoTicket) == 0;
    const bool lone = quiet && __popc(act) == 1;
    const uint32_t np = async_interact<kTrack, Rules>(d, tmpl, tab, hist, W, S, have, pa, pb, live, pre, pra, prb,
                                                      lone, quiet);
    // keep the first new pair and start loading its records now, so the
    // load overlaps the rest of this iteration
    const bool had = have;
    have = np > 0;
    pre = false;
    if (have) {
      const Pair p0 = W.out[0][lane];
      pa = p0.a;
      pb = p0.b;
      if (pa < d.cap_agents && pb < d.cap_agents) {
        pra = ld_node(d.node + pa);
        prb = ld_node(d.node + pb);
        pre = true;
      }
    }
    const uint32_t extra = np > 1 ? np - 1 : 0u;
    // pairs in flight: each new pair beyond a lane's own next one joins
    // before it is published to another warp (lane 0 waits until the
    // increment is performed, so no consumer's decrement can overtake it);
    // each pair that produced nothing leaves afterwards.  When every new
    // pair stays in this warp the increment need not be waited for: only
    // this warp's lane 0 can later count those pairs out, and its atomics on
    // the counter are performed in program order, while the producing
    // lane's own next pair keeps the count above zero meanwhile.  At most
    // cap pairs may be in flight, the capacity of the frontier that a stop
    // drains them to; beyond it the arena is full (checked whenever pairs
    // go to the queue).  Under that bound the queue slot a producer needs
    // is held by a claimed ticket whenever it is still occupied: an
    // unclaimed one would put every later ticket, and so more than cap
    // pairs, in flight.
    const long long grow = (long long)__reduce_add_sync(kFull, extra);
    const long long shrink = -(long long)__reduce_add_sync(kFull, had && np == 0 ? 1u : 0u);
    if (grow) {
      // extra pairs go first to idle lanes of this warp (through shared
      // memory), the rest to the ticket queue
      unsigned inc = extra;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
      }
      const unsigned totx = __shfl_sync(kFull, inc, 31);
      if (totx) {
        for (uint32_t j = 0; j < extra; j++) W.xl[inc - extra + j] = W.out[1 + j][lane];
        const unsigned idle = __ballot_sync(kFull, !have && ticket == kNoTicket);
        const unsigned nidle = __popc(idle);
        __syncwarp();
        const unsigned local = min(nidle, totx);
        if (lane == 0) {
          unsigned long long* ifl = reinterpret_cast<unsigned long long*>(&c->inflight);
          if (totx > local) {
            const long long r = (long long)atomicAdd(ifl, (unsigned long long)grow);
            if (r + grow > (long long)cap) set_error(c, INET_ERR_ARENA_FULL, 9);
          } else {
            atomicAdd(ifl, (unsigned long long)grow);
          }
        }
        __syncwarp();
        if ((idle >> lane) & 1u) {
          const unsigned r = __popc(idle & lanemask_lt());
          if (r < local) {
            const Pair p = W.xl[r];
            pa = p.a;
            pb = p.b;
            have = true;
            if (pa < d.cap_agents && pb < d.cap_agents) {
              pra = ld_node(d.node + pa);
              prb = ld_node(d.node + pb);
              pre = true;
            }
          }
        }
        const unsigned toq = totx - local;
        if (toq) {
          unsigned long long qb = 0, qm = 0;
          if (lane == 0) {
            qb = atomicAdd(&c->q_tail, (unsigned long long)toq);
            qm = qb % cap;
          }
          qb = __shfl_sync(kFull, qb, 0);
          qm = __shfl_sync(kFull, qm, 0);
          for (unsigned j0 = 0; j0 < toq; j0 += 32) {
            const unsigned j = j0 + (unsigned)lane;
            bool pend = j < toq;
            const unsigned long long tk = qb + j;
            unsigned long long si = qm + j;
            if (si >= cap) si %= cap;
            const Pair p = pend ? W.xl[local + j] : Pair{0, 0};
            const unsigned long long t0 = globaltimer();
            for (uint32_t spin = 0;; spin++) {
              // written once the cell's previous pair (ticket tk - cap) is taken
              if (pend && ld_acquire64(d.qseq + si) == tk) {
                __stcg(reinterpret_cast<unsigned long long*>(Q + si),
                       (unsigned long long)p.a | ((unsigned long long)p.b << 32));
                st_release64(d.qseq + si, tk + 1);
                pend = false;
              }
              poll_ticket(d, Q, have, ticket, tslot, pa, pb);
              if (!__any_sync(kFull, pend)) break;
              __nanosleep(64);
              if ((spin & 15) == 15) {
                // after a fatal error (the arena is poisoned) or the time
                // limit, pairs not yet written are given up
                uint32_t give = 0;
                if (lane == 0) {
                  if (ld_volatile((const uint32_t*)&c->fatal)) {
                    give = 1;
                  } else if (globaltimer() - t0 > d.timeout_ns) {
                    set_error(c, INET_ERR_TIMEOUT, 7);
                    give = 1;
                  }
                }
                if (__shfl_sync(kFull, give, 0)) break;
              }
            }
          }
        }
        __syncwarp();
      }
    }
    if (lane == 0 && shrink) atomicAdd(reinterpret_cast<unsigned long long*>(&c->inflight), (unsigned long long)shrink);
    __syncwarp();
  }
  // leaving: publish live agents; a stop drains every pair to the other buffer
  if (lane == 0 && live) atomicAdd(reinterpret_cast<unsigned long long*>(&c->live), (unsigned long long)live);
  if (finished && !stop) {
    if (lane == 0) {
      __threadfence();
      atomicAdd(&c->quiesce, 1u);
    }
  } else {
    uint32_t ok = 1;
    if (lane == 0) {
      __threadfence();
      atomicAdd(&c->quiesce, 1u);
    }
    __syncwarp();
    const unsigned long long t0 = globaltimer();
    for (;;) {
      poll_ticket(d, Q, have, ticket, tslot, pa, pb);  // producers still running may wait for this lane's slot
      uint32_t done = 0;
      if (lane == 0) {
        if (ld_volatile(&c->quiesce) >= total_warps) {
          done = 1;
        } else if (globaltimer() - t0 > d.timeout_ns) {
          set_error(c, INET_ERR_TIMEOUT, 8);
          ok = 0;
          done = 1;
        }
      }
      if (__shfl_sync(kFull, done, 0)) break;
      __nanosleep(256);
    }
    if (lane == 0) {
      __threadfence();
      if (ld_volatile((const uint32_t*)&c->fatal)) ok = 0;  // poisoned: nothing to keep
    }
    ok = __shfl_sync(kFull, ok, 0);
    if (ok) {
      const unsigned long long qt = ld_volatile64(&c->q_tail);
      if (!have && ticket != kNoTicket && ticket < qt) {
        Pair p;
        if (wait_ticket(d, Q, ticket, &p)) {
          pa = p.a;
          pb = p.b;
          have = true;
        }
      }
      if (have) exit_pair(d, Pair{pa, pb});
      // unclaimed tickets, shared among the warps
      const unsigned long long qh = ld_volatile64(&c->q_head);
      const uint32_t gw = blockIdx.x * (blockDim.x / 32) + (uint32_t)wid;
      for (unsigned long long tk = qh + (unsigned long long)gw * 32 + lane; tk < qt;
           tk += (unsigned long long)total_warps * 32) {
        Pair p;
        if (wait_ticket(d, Q, tk, &p)) exit_pair(d, p);
      }
    }
  }
  // free slots known only to this warp go back to the rings (when owners are
  // kept, marked free: a stack also holds slots fetched from the pools and
  // never used, which may come from the bump pointer with stale contents)
  __syncwarp();
  {
    unsigned long long ab = 0, vb = 0;
    if (lane == 0) {
      if (S.ac) ab = atomicAdd(&c->a_tail, (unsigned long long)S.ac);
      if (S.vc) vb = atomicAdd(&c->v_tail, (unsigned long long)S.vc);
    }
    ab = __shfl_sync(kFull, ab, 0);
    vb = __shfl_sync(kFull, vb, 0);
    for (int j = lane; j < S.ac; j += 32) {
      const uint32_t sl = W.astk[j];
      if constexpr (kTrack) {
        if (sl < d.cap_agents) __stcg(&d.node[sl].head, kFreeHead);
      }
      __stcg(d.afree + (ab + j) % d.cap_agents, sl);
    }
    for (int j = lane; j < S.vc; j += 32) {
      const uint32_t x = W.vstk[j];
      if constexpr (kTrack) {
        if (x < d.cap_vars) __stcg(d.vown + x, kNoNet);
      }
      __stcg(d.vfree + (vb + j) % d.cap_vars, x);
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < d.n_tmpl; i += blockDim.x)
    if (hist[i]) atomicAdd(&d.rule_hist[i], (unsigned long long)hist[i]);
}

// Before an asynchronous launch: the current frontier's pairs are tickets
// 0 .. n0-1, already written; every other cell waits for its first ticket.
// Only cells an earlier launch used are rewritten (all of them once after a
// reset), so a short launch does not pay, or flush L2 with, the whole ring.
__global__ void k_async_fill(Dev d) {
  const Ctrl* c = d.ctrl;
  const uint32_t n0 = min(c->fcount[d.qcur], d.cap_pairs);
  const unsigned long long lim =
      c->qinit ? max(min(c->qdirty, (unsigned long long)d.cap_pairs), (unsigned long long)n0) : d.cap_pairs;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < lim;
       i += (unsigned long long)gridDim.x * blockDim.x)
    d.qseq[i] = i < n0 ? i + 1 : i;
}

// Before an asynchronous launch (one thread): publish the rings, make the
// current frontier the ticket queue.
__global__ void k_async_prep(Dev d) {
  Ctrl* c = d.ctrl;
  const uint32_t n0 = min(c->fcount[d.qcur], d.cap_pairs);
  if (c->a_head > c->a_pub) c->a_head = c->a_pub;
  c->a_pub = c->a_tail;
  if (c->v_head > c->v_pub) c->v_head = c->v_pub;
  c->v_pub = c->v_tail;
  c->qinit = 1;  // the fill before this launch initialised the ring
  c->q_head = 0;
  c->q_tail = n0;
  c->inflight = n0;
  c->astop = 0;
  c->quiesce = 0;
  c->aexit = 0;
  c->slice_t0 = 0;
  c->hit_slice = 0;
  c->done = 0;
  __threadfence();
}

// After an asynchronous launch (one thread): the pairs written back become
// the frontier of the other buffer.
__global__ void k_async_post(Dev d) {
  Ctrl* c = d.ctrl;
  const uint32_t cur = d.qcur;
  const uint32_t n = min(c->aexit, d.cap_pairs);
  // pops that found the ring empty went to the bump pointer but advanced the head
  if (c->a_head > c->a_pub) c->a_head = c->a_pub;
  if (c->v_head > c->v_pub) c->v_head = c->v_pub;
  c->fcount[cur] = 0;
  c->fcount[cur ^ 1u] = n;
  // cells this launch wrote: tickets below the tail (any after a fatal error)
  c->qdirty = c->fatal ? (unsigned long long)d.cap_pairs : min(c->q_tail, (unsigned long long)d.cap_pairs);
  c->step = c->step + 1;
  c->done = n == 0 || c->fatal != 0 ? 1u : 0u;
  if (c->live > c->peak_live) c->peak_live = c->live;
  __threadfence();
}

}  // namespace inet
