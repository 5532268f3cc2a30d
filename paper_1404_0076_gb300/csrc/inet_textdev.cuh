// Text readback of a net's normal form on the device: ->col and ->sub
// (Sec. 2.2; Theorem 1 puts them after the reduction) by following name
// slots, and the rendering of the interface terms as text, without copying
// the arena to the host.
//
// The live agents of the net first get dense ids c = 0 .. n-1 (one pass
// over the arena, in no particular order: ids only name list elements).  The
// text of a term forest is a pre-order walk.  Agent c owns four elements of
// one linked list: OPEN(c) = 4c ("Label" and "(" when it has ports) and, for
// each auxiliary port i, AFTER(c, i) = 4c + 1 + i (the name at port i when
// the port leads to a name, then ", " or ")").  Interface root j owns
// ROOT(j) = 4n + j (its name when the root is a name, then ", " unless it
// is the last).  Successors:
//   OPEN(c)     -> FIRST(c, 0), or NEXT(c) for an agent without ports
//   AFTER(c, i) -> FIRST(c, i + 1), or NEXT(c) after the last port
//   ROOT(j)     -> the first element of root j + 1, or the end
// where FIRST(c, i) is OPEN(c') when port i leads (through name slots) to
// agent c' and AFTER(c, i) when it leads to a name, and NEXT(c) is the
// element that follows c's subterm: AFTER(p, i) when c hangs at port i of
// p, ROOT(j) when c is root j.  List ranking by pointer jumping gives every
// element the characters (without names) and the names that follow it; the
// names are then numbered in order of first occurrence (two scans), and
// every element writes its characters at its offset.
#pragma once

#include "inet_kernels.cuh"

namespace inet {

constexpr uint32_t kTxtEnd = 0xFFFFFFFEu;    // successor: the end of the text
constexpr uint32_t kTxtDead = 0xFFFFFFFFu;   // successor: not part of the text
constexpr uint32_t kTxtNone = 0xFFFFFFFFu;   // dense id or parent: none
// control words: [0] not a forest / a write outside the text, [1] rounds
// run, [2] head element, [3] agents the text reaches, [5] agents of the net,
// [8 + r] round r + 1 is needed
constexpr int kTxtCtl = 72;

// One list element: successor, names in the suffix, characters in the
// suffix (names not counted).
struct alignas(16) TxtElem {
  uint32_t succ;
  uint32_t names;
  unsigned long long chars;
};

// The word at the end of a chain of name slots that hold terms.
__device__ __forceinline__ uint32_t txt_resolve(const Dev& d, uint32_t w, uint32_t n_vars) {
  for (uint32_t hop = 0; hop <= n_vars && is_var(w) && idx_of(w) < n_vars; hop++) {
    const uint32_t v = __ldcg(d.var + idx_of(w));
    if (v == kEmpty) break;
    w = v;
  }
  return w;
}

// Marks the agent slots waiting in the free ring (between reductions every
// free slot is there): their records are stale.
__global__ void k_txt_free_marks(Dev d, uint32_t n_agents, uint8_t* dead) {
  const Ctrl* c = d.ctrl;
  const unsigned long long h = min(c->a_head, c->a_pub), t = c->a_tail;
  const unsigned long long n = t > h ? min(t - h, d.cap_agents) : 0ull;
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t s = __ldcg(d.afree + (h + k) % d.cap_agents);
    if (s < n_agents) dead[s] = 1;
  }
}

// Dense ids of the net's live agents: cid[a] for slot a (kTxtNone for the
// other slots, set before), slot[c] for id c; ctl[5] counts them.  Loops go
// by whole warps, so the ids are taken by one atomic per warp.
__global__ void k_txt_compact(Dev d, uint32_t net, uint32_t n_agents, const uint8_t* dead, uint32_t* cid,
                              uint32_t* slot, uint32_t* ctl) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  const uint32_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  for (uint32_t a0 = w * 32; a0 < n_agents; a0 += warps * 32) {
    const uint32_t a = a0 + (uint32_t)lane;
    bool mine = false;
    if (a < n_agents && !dead[a]) {
      const int32_t h = __ldcg(&d.node[a].head);
      mine = h != kFreeHead && ((uint32_t)h >> 8) == net;
    }
    const unsigned m = __ballot_sync(kFull, mine);
    if (!m) continue;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(ctl + 5, (uint32_t)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (mine) {
      const uint32_t c = base + (uint32_t)__popc(m & lanemask_lt());
      cid[a] = c;
      slot[c] = a;
    }
  }
}

// The dense id of the agent a resolved word leads to, kTxtNone for a name,
// and kTxtDead (ctl[0] set) for a word that is neither a live agent of the
// net nor a name slot in range: the host renders such a net.
__device__ __forceinline__ uint32_t txt_target(uint32_t w, uint32_t n_agents, uint32_t n_vars, const uint32_t* cid,
                                               uint32_t* ctl) {
  if (is_agent(w) && idx_of(w) < n_agents) {
    const uint32_t c = cid[idx_of(w)];
    if (c != kTxtNone) return c;
  } else if (is_var(w) && idx_of(w) < n_vars) {
    return kTxtNone;
  }
  atomicExch(ctl, 1u);
  return kTxtDead;
}

// parent[c] = the element that follows agent c's subterm, for every agent
// c that a port of an agent of the net, or an interface root, leads to.  A
// second claim on one agent (a shared subterm, or a cycle through the
// roots) sets ctl[0]: the caller renders such a net on the host instead.
__global__ void k_txt_parent(Dev d, uint32_t n_c, uint32_t n_agents, uint32_t n_vars, const uint32_t* slot,
                             const uint32_t* cid, const uint32_t* roots, uint32_t n_roots, const uint8_t* arity,
                             uint32_t* parent, uint32_t* ctl) {
  const uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (uint32_t j = i0; j < n_roots; j += stride) {
    const uint32_t c = txt_target(txt_resolve(d, roots[j], n_vars), n_agents, n_vars, cid, ctl);
    if (c < n_c && atomicCAS(parent + c, kTxtNone, 4 * n_c + j) != kTxtNone) atomicExch(ctl, 1u);
  }
  for (uint32_t c = i0; c < n_c; c += stride) {
    const int4 r = ld_node(d.node + slot[c]);
    const uint32_t lab = (uint32_t)r.x & 0xFFu, k = lab < d.n_labels ? min((uint32_t)arity[lab], 3u) : 0u;
    const uint32_t aux[3] = {(uint32_t)r.y, (uint32_t)r.z, (uint32_t)r.w};
    for (uint32_t i = 0; i < k; i++) {
      const uint32_t t = txt_target(txt_resolve(d, aux[i], n_vars), n_agents, n_vars, cid, ctl);
      if (t < n_c && atomicCAS(parent + t, kTxtNone, 4 * c + 1 + i) != kTxtNone) atomicExch(ctl, 1u);
    }
  }
}

// Successor and weights of every element (both buffers for the elements
// that are not part of any text: the rounds skip them).  lablen[l] =
// characters of label l.
__global__ void k_txt_init(Dev d, uint32_t n_c, uint32_t n_agents, uint32_t n_vars, const uint32_t* slot,
                           const uint32_t* cid, const uint32_t* roots, uint32_t n_roots, const uint8_t* arity,
                           const uint8_t* lablen, const uint32_t* parent, TxtElem* el, TxtElem* el2, uint32_t* ctl) {
  const uint32_t stride = gridDim.x * blockDim.x;
  // the element a resolved word starts at: OPEN(t) for agent t, else the
  // element that carries the name
  auto first = [&](uint32_t t, uint32_t name_elem) { return t < n_c ? 4 * t : name_elem; };
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n_c; c += stride) {
    TxtElem e[4];
    for (int t = 0; t < 4; t++) e[t] = TxtElem{kTxtDead, 0u, 0ull};
    const int4 r = ld_node(d.node + slot[c]);
    const uint32_t lab = (uint32_t)r.x & 0xFFu;
    const uint32_t k = lab < d.n_labels ? min((uint32_t)arity[lab], 3u) : 0u;
    const uint32_t nxt = parent[c] == kTxtNone ? kTxtDead : parent[c];
    const uint32_t aux[3] = {(uint32_t)r.y, (uint32_t)r.z, (uint32_t)r.w};
    uint32_t tgt[3] = {kTxtDead, kTxtDead, kTxtDead};
    for (uint32_t i = 0; i < k; i++) tgt[i] = txt_target(txt_resolve(d, aux[i], n_vars), n_agents, n_vars, cid, ctl);
    e[0].chars = (lab < d.n_labels ? lablen[lab] : 1u) + (k ? 1u : 0u);
    e[0].succ = k ? first(tgt[0], 4 * c + 1) : nxt;
    for (uint32_t i = 0; i < k; i++) {
      e[1 + i].names = tgt[i] == kTxtNone ? 1u : 0u;
      e[1 + i].chars = i + 1 < k ? 2u : 1u;
      e[1 + i].succ = i + 1 < k ? first(tgt[i + 1], 4 * c + 2 + i) : nxt;
    }
    for (int t = 0; t < 4; t++) {
      el[4 * c + t] = e[t];
      if (e[t].succ == kTxtDead) el2[4 * c + t] = e[t];
    }
  }
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n_roots; j += stride) {
    const uint32_t t = txt_target(txt_resolve(d, roots[j], n_vars), n_agents, n_vars, cid, ctl);
    TxtElem e;
    e.names = t == kTxtNone ? 1u : 0u;
    e.chars = j + 1 < n_roots ? 2u : 0u;
    e.succ = j + 1 < n_roots
                 ? first(txt_target(txt_resolve(d, roots[j + 1], n_vars), n_agents, n_vars, cid, ctl),
                         4 * n_c + j + 1)
                 : kTxtEnd;
    el[4 * n_c + j] = e;
  }
}

// The head of the list, root 0's first element, into ctl[2] (one thread).
__global__ void k_txt_head(Dev d, uint32_t n_c, uint32_t n_agents, uint32_t n_vars, const uint32_t* cid,
                           const uint32_t* roots, uint32_t* ctl) {
  const uint32_t t = txt_target(txt_resolve(d, roots[0], n_vars), n_agents, n_vars, cid, ctl);
  ctl[2] = t < n_c ? 4 * t : 4 * n_c;
}

// Pointer jumping, round r (buffer r % 2 to the other): every element adds
// its successor's sums and takes its successor's successor.  ctl[8 + r - 1]
// says whether round r is needed; ctl[1] = rounds run.  Elements that are
// not part of any text from the start (both buffers hold them) are skipped.
__global__ void k_txt_round(uint32_t n_el, uint32_t r, uint32_t* ctl, const TxtElem* b0, TxtElem* b1) {
  if (r > 0 && !ctl[8 + r - 1]) return;
  const TxtElem* in = (r & 1u) ? b1 : b0;
  TxtElem* out = (r & 1u) ? const_cast<TxtElem*>(b0) : b1;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += gridDim.x * blockDim.x) {
    TxtElem e = in[i];
    if (e.succ == kTxtDead) continue;
    if (e.succ < n_el) {
      const TxtElem q = in[e.succ];
      e.succ = q.succ;
      e.names += q.names;
      e.chars += q.chars;
    }
    out[i] = e;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl[1] = r + 1;
}

// After round r: is the head still short of the end?  (Every element of
// the head's list is then no further from its end than the head.)  One
// thread.
__global__ void k_txt_check_head(uint32_t n_el, uint32_t r, uint32_t* ctl, const TxtElem* b0, const TxtElem* b1) {
  if (ctl[1] != r + 1) return;
  const TxtElem* buf = ((r + 1) & 1u) ? b1 : b0;
  const uint32_t head = ctl[2];
  if (head < n_el && buf[head].succ < n_el) ctl[8 + r] = 1u;
}

// The head element after the last round that ran, to `dst` (one thread);
// its sums are the totals of the text.
__global__ void k_txt_copy_head(const uint32_t* ctl, const TxtElem* b0, const TxtElem* b1, TxtElem* dst) {
  const TxtElem* buf = (ctl[1] & 1u) ? b1 : b0;
  *dst = buf[ctl[2]];
}

// The name an element carries (its resolved word's name slot), or
// kTxtNone.
__device__ __forceinline__ uint32_t txt_name_of(const Dev& d, uint32_t e, uint32_t n_c, uint32_t n_vars,
                                                const uint32_t* roots, const uint32_t* slot) {
  uint32_t w;
  if (e >= 4 * n_c) {
    w = roots[e - 4 * n_c];
  } else {
    const uint32_t t = e & 3u;
    if (t == 0) return kTxtNone;
    const int4 r = ld_node(d.node + slot[e / 4]);
    w = t == 1 ? (uint32_t)r.y : t == 2 ? (uint32_t)r.z : (uint32_t)r.w;
  }
  w = txt_resolve(d, w, n_vars);
  return is_var(w) && idx_of(w) < n_vars ? idx_of(w) : kTxtNone;
}

// Names on the text, in order: an element that carries a name is occurrence
// L = total names - its suffix count (the suffix counts its own name);
// first[x] = the least L of name slot x, key[L] = x.
__global__ void k_txt_names(Dev d, uint32_t n_el, uint32_t n_c, uint32_t n_vars, const uint32_t* roots,
                            const uint32_t* slot, const TxtElem* fin, uint32_t total_names, uint32_t* first,
                            uint32_t* key) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += gridDim.x * blockDim.x) {
    const TxtElem e = fin[i];
    if (e.succ != kTxtEnd) continue;
    const uint32_t x = txt_name_of(d, i, n_c, n_vars, roots, slot);
    if (x == kTxtNone) continue;
    const uint32_t L = total_names - e.names;
    if (L < total_names) {
      key[L] = x;
      atomicMin(first + x, L);
    }
  }
}

// flag[L] = 1 when name occurrence L is the first of its name.
__global__ void k_txt_firsts(uint32_t n, const uint32_t* first, const uint32_t* key, uint32_t* flag) {
  const uint32_t L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L < n) flag[L] = first[key[L]] == L ? 1u : 0u;
}

__device__ __forceinline__ uint32_t txt_digits(uint32_t v) {
  uint32_t n = 1;
  while (v >= 10) {
    v /= 10;
    n++;
  }
  return n;
}

// num[L] = the canonical number of occurrence L's name (the first
// occurrences before its first one; `rank` is the exclusive scan of the
// flags), len[L] = the characters of "x<num>".
__global__ void k_txt_numbers(uint32_t n, const uint32_t* first, const uint32_t* key, const uint32_t* rank,
                              uint32_t* num, uint32_t* len) {
  const uint32_t L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= n) return;
  const uint32_t k = rank[first[key[L]]];
  num[L] = k;
  len[L] = 1 + txt_digits(k);
}

// Every element of the text writes its characters at: the characters
// (without names) before it, total - its suffix, plus the characters of the
// names before it, noff[L] (the exclusive scan of len; L = the first name
// occurrence at or after the element).  Label l's text is labels +
// laboff[l], lablen[l] characters.
__global__ void k_txt_scatter(Dev d, uint32_t n_el, uint32_t n_c, uint32_t n_vars, const uint32_t* roots,
                              const uint32_t* slot, uint32_t n_roots, const TxtElem* fin, unsigned long long total_chars,
                              uint32_t total_names, unsigned long long name_chars, const uint32_t* num,
                              const uint32_t* noff, const uint32_t* nlen, const uint8_t* arity, const char* labels,
                              const uint32_t* laboff, const uint8_t* lablen, char* out, unsigned long long cap,
                              uint32_t* ctl) {
  // every write is checked against the buffer; one outside it (which the
  // offsets rule out) is recorded in ctl[0] and skipped
  auto put = [&](unsigned long long p, char ch) {
    if (p < cap) out[p] = ch;
    else atomicExch(ctl, 1u);
  };
  // agents the text reaches (OPEN elements on it): per block, then ctl[3]
  __shared__ uint32_t reached;
  if (threadIdx.x == 0) reached = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += gridDim.x * blockDim.x) {
    const TxtElem e = fin[i];
    if (e.succ != kTxtEnd) continue;
    const uint32_t L = total_names - e.names;
    unsigned long long pos = (total_chars - e.chars) + (L < total_names ? noff[L] : name_chars);
    if (i < 4 * n_c && (i & 3u) == 0) {  // OPEN(c)
      atomicAdd(&reached, 1u);
      const int4 r = ld_node(d.node + slot[i / 4]);
      const uint32_t lab = (uint32_t)r.x & 0xFFu;
      if (lab < d.n_labels) {
        for (uint32_t c = 0; c < lablen[lab]; c++) put(pos + c, labels[laboff[lab] + c]);
        if (arity[lab]) put(pos + lablen[lab], '(');
      } else {
        put(pos, '?');
      }
      continue;
    }
    // AFTER(a, i) or ROOT(j): the name it carries, if any, then its separator
    if (txt_name_of(d, i, n_c, n_vars, roots, slot) != kTxtNone && L < total_names) {
      put(pos, 'x');
      uint32_t v = num[L];
      const uint32_t nd = nlen[L] - 1;
      for (uint32_t c = 0; c < nd; c++) {
        put(pos + nd - c, (char)('0' + v % 10));
        v /= 10;
      }
      pos += nlen[L];
    }
    bool last;
    if (i >= 4 * n_c) {
      last = i - 4 * n_c + 1 == n_roots;
      if (!last) {
        put(pos, ',');
        put(pos + 1, ' ');
      }
    } else {
      const int4 r = ld_node(d.node + slot[i / 4]);
      const uint32_t lab = (uint32_t)r.x & 0xFFu;
      const uint32_t k = lab < d.n_labels ? min((uint32_t)arity[lab], 3u) : 0u;
      last = (i & 3u) == k;
      if (last) {
        put(pos, ')');
      } else {
        put(pos, ',');
        put(pos + 1, ' ');
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && reached) atomicAdd(ctl + 3, reached);
}

}  // namespace inet
