// C ABI of the evaluator (include/inet.h): context, device workspace, net
// loading, the three drivers of the step loop (plain host loop, CUDA graph
// with a conditional WHILE node, persistent cooperative kernel) and readback.
#include <cuda_runtime.h>

#include <algorithm>
#include <thread>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "host_pool.h"
#include "inet.h"
#include "inet_async.cuh"
#include "inet_kernels.cuh"
#include "inet_micro.cuh"
#include "inet_control.cuh"
#include "inet_free.cuh"
#include "inet_jit.h"
#include "inet_paper.cuh"
#include "inet_readback.cuh"
#include "inet_textdev.cuh"
#include "inet_text.h"

using namespace inet;

namespace {

constexpr uint32_t kTraceCap = 1u << 20;
constexpr uint32_t kReadChunk = 1u << 16;  // nets per device walk of inet_readback_nats
constexpr uint32_t kWalkMin = 256;         // S agents one thread walks before its net's agents are ranked
constexpr uint64_t kDefaultAgents = 1ull << 22;
constexpr uint64_t kDefaultVars = 1ull << 22;
constexpr uint64_t kDefaultPairs = 1ull << 21;
constexpr uint32_t kDefaultNets = 1u << 16;
constexpr unsigned long long kDefaultTimeoutNs = 10ull * 1000 * 1000 * 1000;
constexpr unsigned long long kSliceNs = 2ull * 1000 * 1000 * 1000;
constexpr uint32_t kMaxSolo = 1024;
constexpr size_t kMaxSmem = 227 * 1024;

struct Layout {
  size_t ctrl, node, var, vown, front0, front1, qseq, afree, vfree, netctr, netstat, netrep, netmark, netlive,
      netquota, hist, table, tmpl, arity, trace_front, trace_live, rb_root, rb_val, fin_ids, fin_cnt, free_ids, free_st,
      stn_ids, stn_ctr, stn_live, rbmark, total;
};

inet_arena_cfg with_defaults(const inet_arena_cfg* in) {
  inet_arena_cfg c;
  memset(&c, 0, sizeof c);
  if (in) c = *in;
  if (!c.max_agents) c.max_agents = kDefaultAgents;
  if (!c.max_vars) c.max_vars = kDefaultVars;
  if (!c.max_pairs) c.max_pairs = kDefaultPairs;
  if (!c.max_nets) c.max_nets = kDefaultNets;
  return c;
}

bool valid_cfg(const inet_arena_cfg& c) {
  return c.max_agents <= kMaxIndex + 1ull && c.max_vars <= kMaxIndex + 1ull && c.max_pairs <= 0xFFFFFFFFull &&
         c.max_nets <= kMaxNetSlots && (c.flags & ~INET_ARENA_FREE_NETS) == 0;
}

Layout layout_of(const inet_arena_cfg& c) {
  Layout L;
  size_t b = 0;
  auto take = [&](size_t n) { b = (b + 255) / 256 * 256; size_t at = b; b += n; return at; };
  L.ctrl = take(sizeof(Ctrl));
  L.node = take(sizeof(Node) * c.max_agents);
  L.var = take(sizeof(uint32_t) * c.max_vars);
  L.vown = take((c.flags & INET_ARENA_FREE_NETS) ? sizeof(uint32_t) * c.max_vars : 0);
  L.front0 = take(sizeof(Pair) * c.max_pairs);
  L.front1 = take(sizeof(Pair) * c.max_pairs);
  L.qseq = take(sizeof(unsigned long long) * c.max_pairs);
  L.afree = take(sizeof(uint32_t) * c.max_agents);
  L.vfree = take(sizeof(uint32_t) * c.max_vars);
  L.netctr = take(sizeof(unsigned long long) * c.max_nets);
  L.netstat = take(sizeof(int32_t) * c.max_nets);
  L.netrep = take(sizeof(uint32_t) * c.max_nets);
  L.netmark = take(c.max_nets);
  L.netlive = take(sizeof(long long) * c.max_nets);
  L.netquota = take(sizeof(unsigned long long) * c.max_nets);
  L.hist = take(sizeof(unsigned long long) * INET_MAX_RULES);
  L.table = take(sizeof(int16_t) * kMaxLabels * kMaxLabels);
  L.tmpl = take(sizeof(Template) * INET_MAX_RULES);
  L.arity = take(kMaxLabels);
  L.trace_front = take(sizeof(long long) * kTraceCap);
  L.trace_live = take(sizeof(long long) * kTraceCap);
  L.rb_root = take(sizeof(uint32_t) * kReadChunk);
  L.rb_val = take(sizeof(unsigned long long) * kReadChunk);
  L.fin_ids = take(sizeof(int32_t) * kReadChunk);
  L.fin_cnt = take(sizeof(uint32_t));
  L.free_ids = take(sizeof(int32_t) * kReadChunk);
  L.free_st = take(sizeof(unsigned long long) * 4);
  L.stn_ids = take(sizeof(int32_t) * kReadChunk);
  L.stn_ctr = take(sizeof(unsigned long long) * kReadChunk);
  L.stn_live = take(sizeof(long long) * kReadChunk);
  L.rbmark = take(c.max_nets);
  L.total = take(0) + 256;
  return L;
}

struct NetRec {
  bool used = false;
  bool uploaded = false;          // its records and counter are on the device
  bool started = false;           // its pairs were handed to the device
  std::vector<uint32_t> iface;
  std::vector<Pair> pairs;        // initial active pairs, until started
};

}  // namespace

struct inet_ctx {
  int device = -1;
  bool host_only = true;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  inet_arena_cfg cfg{};
  Layout lay{};
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  bool ws_ready = false;
  Dev dev{};
  int num_sms = 0;
  // rules
  bool have_rules = false;
  CompiledRules rules;
  uint64_t rules_gen = 0;                   // counts rule sets loaded
  // rule-specialised asynchronous kernel (inet_jit.h): per owner tracking
  // (0: without, 1: with) for the loaded rules
  bool jit_on = true;
  int jit_state[2] = {0, 0};                // 0: not built yet, 1: built, -1: failed
  const void* jit_fn[2] = {nullptr, nullptr};
  double jit_ms = 0;                        // NVRTC time of the last build (0 from a cache)
  int jit_source = 0;                       // where the last build came from: 1 compiled, 2 disk, 3 process
  uint64_t jit_launches = 0;                // asynchronous launches that used it
  std::string jit_msg;
  // host mirrors of device counters
  uint64_t a_bump = 0, v_bump = 0;
  int64_t live = 0;
  uint32_t step = 0;
  uint32_t fcount[2] = {0, 0};
  // nets
  std::vector<NetRec> nets;
  // staged loads
  std::vector<Node> st_nodes;
  uint64_t st_a0 = 0;
  std::vector<uint32_t> st_vars;
  uint64_t st_v0 = 0;
  std::vector<uint32_t> st_vown;            // owning net of each staged name slot
  std::vector<unsigned long long> st_netctr;
  std::vector<int32_t> st_net_ids;          // ids of the staged nets, parallel to st_netctr
  std::vector<long long> st_netlive;        // their agents, parallel to st_netctr
  bool quotas_set = false;                  // some net has a quota (inet_set_quotas)
  std::vector<int32_t> free_net_ids;        // ids released by inet_free_nets, reused by loads
  // device-side per-net copies (after the last reduce)
  std::vector<unsigned long long> h_netctr;
  std::vector<int32_t> h_netstat;
  bool h_net_valid = true;  // false: the device changed them since the last copy
  // readback snapshot
  bool snap_valid = false;
  uint64_t snap_gen = 0;                    // counts snapshots taken
  // the text of the last inet_readback, so that a size query followed by
  // the copy walks the net once
  int32_t text_net = -1;
  uint64_t text_gen = 0;
  std::string text;
  uint64_t text_reached = 0;                // agents that walk reached
  std::vector<Node> snap_nodes;
  std::vector<uint32_t> snap_vars;
  std::vector<int64_t> snap_live;
  // graph
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  int g_block = 0, g_grid = 0;
  // trace of the last reduce
  std::vector<long long> tr_front, tr_live;
  bool poisoned = false;
  uint64_t h2d_bytes = 0, d2h_bytes = 0;  // host<->device bytes copied by this context
  // non-blocking numeral readback: one batch at a time on a second stream
  cudaStream_t rb_stream = nullptr;
  cudaEvent_t rb_ready = nullptr, rb_after = nullptr;
  uint32_t* rb_host_roots = nullptr;       // pinned, kReadChunk entries
  unsigned long long* rb_host_vals = nullptr;
  std::vector<uint64_t> rb_inter;           // interactions of the batch in flight
  std::vector<int32_t> rb_ids;              // its nets
  int32_t rb_n = -1;                        // nets of the batch in flight, -1: none
  // list-ranking scratch of the numeral readback: two buffers of
  // (successor, weight) per agent and name slot, and its control words
  uint2* jump_buf = nullptr;
  uint64_t jump_cap = 0;                    // elements per buffer
  uint32_t* jump_ctl = nullptr;
  // device text readback: grow-only scratch (inet_textdev.cuh), the label
  // table of the loaded rules, and the text of the last call
  struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
  };
  DevBuf txt_dead, txt_cid, txt_parent, txt_el, txt_roots, txt_first, txt_names, txt_out, txt_ctl, txt_labels;
  bool txt_labels_ok = false;
  uint64_t arena_gen = 0;                   // counts changes of the arena (loads, reductions, frees)
  int32_t dtext_net = -1;
  uint64_t dtext_gen = 0;
  uint64_t dtext_reached = 0;               // agents the text reaches
  int64_t dtext_live = -1;                  // the net's live agents when it was rendered
  uint64_t renders_device = 0, renders_host = 0;  // texts rendered on each side
  std::string dtext;
  std::string err;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

struct DeviceGuard {
  int prev = -1, want = -1;
  explicit DeviceGuard(int d) : want(d) {
    if (d < 0) return;
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    if (want >= 0 && prev >= 0 && prev != want) cudaSetDevice(prev);
  }
};

// Raises the dynamic shared-memory limit of a kernel on the current device
// to at least `bytes` and never lowers it: the attribute belongs to the
// kernel for the whole process, so lowering it for one context could make a
// concurrent launch of another context, which needs more, fail.  A fixed
// table (no allocation): kernel k on device d.
enum { kSmemStep = 0, kSmemPersistent = 2, kSmemAsync = 4, kSmemKernels = 6 };  // + 1: owners kept
std::mutex g_smem_mu;
size_t g_smem_set[kSmemKernels][256] = {};

cudaError_t raise_smem(int which, const void* func, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_smem_mu);
  size_t& cur = g_smem_set[which][dev];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// The same for kernels loaded at run time (the rule-specialised ones): a
// map by kernel and device.
std::mutex g_smem_dyn_mu;
std::map<std::pair<const void*, int>, size_t> g_smem_dyn;

cudaError_t raise_smem_dyn(const void* func, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_smem_dyn_mu);
  size_t& cur = g_smem_dyn[{func, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// The loop kernels a context launches: the instantiations that keep name
// owners and free marks when it was created with INET_ARENA_FREE_NETS.
using KernelFn = void (*)(Dev);
struct LoopKernels {
  KernelFn step, persistent, async;
  int track;
};
LoopKernels loop_kernels(bool track) {
  if (track) return {k_step<true>, k_persistent<true>, k_async<true>, 1};
  return {k_step<false>, k_persistent<false>, k_async<false>, 0};
}

inet_status fail(inet_ctx* c, inet_status code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

// The rule-specialised k_async (owner tracking: track) for the loaded rules,
// built on first use and kept; null when turned off or when it cannot be
// built (the general kernel then runs, and inet_jit_info says why).
const void* jit_kernel(inet_ctx* ctx, int track) {
  if (!ctx->jit_on || ctx->rules.tmpl.empty()) return nullptr;
  if (ctx->jit_state[track] == 1) return ctx->jit_fn[track];
  if (ctx->jit_state[track] == -1) return nullptr;
  int ma = 0, mi = 0;
  cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, ctx->device);
  cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, ctx->device);
  char arch[32];
  snprintf(arch, sizeof arch, "sm_%d%da", ma, mi);
  JitResult jr;
  std::string err;
  if (!jit_async(ctx->rules.tmpl.data(), ctx->rules.tmpl.size(), track != 0, arch, true, &jr, &err)) {
    ctx->jit_state[track] = -1;
    ctx->jit_msg = err;
    return nullptr;
  }
  ctx->jit_state[track] = 1;
  ctx->jit_fn[track] = jr.fn;
  ctx->jit_ms = jr.compile_ms;
  ctx->jit_source = jr.from_memory ? 3 : (jr.from_disk ? 2 : 1);
  ctx->jit_msg.clear();
  return jr.fn;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      ctx->poisoned = true;                                                               \
      return fail(ctx, INET_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                     \
  } while (0)

cudaError_t h2d(inet_ctx* ctx, void* dst, const void* src, size_t n) {
  ctx->h2d_bytes += n;
  return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, ctx->stream);
}
cudaError_t d2h(inet_ctx* ctx, void* dst, const void* src, size_t n) {
  ctx->d2h_bytes += n;
  return cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, ctx->stream);
}

template <class T>
T* at(inet_ctx* ctx, size_t off) {
  return reinterpret_cast<T*>(ctx->ws + off);
}

void fill_dev(inet_ctx* ctx) {
  Dev& d = ctx->dev;
  const Layout& L = ctx->lay;
  d.node = at<Node>(ctx, L.node);
  d.var = at<uint32_t>(ctx, L.var);
  d.front[0] = at<Pair>(ctx, L.front0);
  d.front[1] = at<Pair>(ctx, L.front1);
  d.qseq = at<unsigned long long>(ctx, L.qseq);
  d.afree = at<uint32_t>(ctx, L.afree);
  d.vfree = at<uint32_t>(ctx, L.vfree);
  d.vown = (ctx->cfg.flags & INET_ARENA_FREE_NETS) ? at<uint32_t>(ctx, L.vown) : nullptr;
  d.netctr = at<unsigned long long>(ctx, L.netctr);
  d.netstat = at<int32_t>(ctx, L.netstat);
  d.netrep = at<uint32_t>(ctx, L.netrep);
  const bool track = (ctx->cfg.flags & INET_ARENA_FREE_NETS) != 0;
  d.netlive = track ? at<long long>(ctx, L.netlive) : nullptr;
  d.netquota = track ? at<unsigned long long>(ctx, L.netquota) : nullptr;
  d.rule_hist = at<unsigned long long>(ctx, L.hist);
  d.ctrl = at<Ctrl>(ctx, L.ctrl);
  d.table = at<int16_t>(ctx, L.table);
  d.tmpl = at<Template>(ctx, L.tmpl);
  d.arity = at<uint8_t>(ctx, L.arity);
  d.trace_front = at<long long>(ctx, L.trace_front);
  d.trace_live = at<long long>(ctx, L.trace_live);
  d.cap_agents = ctx->cfg.max_agents;
  d.cap_vars = ctx->cfg.max_vars;
  d.cap_pairs = (uint32_t)ctx->cfg.max_pairs;
  d.trace_cap = kTraceCap;
  d.max_nets = ctx->cfg.max_nets;
  d.n_labels = (uint32_t)ctx->rules.n_labels();
  d.n_tmpl = (uint32_t)ctx->rules.tmpl.size();
  d.rules_key = rules_key(ctx->rules.tmpl.data(), ctx->rules.tmpl.size());
  d.timeout_ns = kDefaultTimeoutNs;
  d.slice_ns = kSliceNs;
  d.solo_max = 0;
  d.use_cond = 0;
  d.paper = 0;
  d.eq = nullptr;
  d.eq_n = nullptr;
  d.cap_eq = 0;
  d.eq_fix = nullptr;
  d.eq_fix_n = 0;
  d.cap_fix = 0;
  d.cond = 0;
}

inet_status upload_rules(inet_ctx* ctx) {
  if (!ctx->ws_ready || !ctx->have_rules) return INET_OK;
  const CompiledRules& r = ctx->rules;
  std::vector<uint8_t> ar(kMaxLabels, 0);
  for (size_t i = 0; i < r.arity.size(); i++) ar[i] = (uint8_t)r.arity[i];
  if (!r.table.empty())
    CK(h2d(ctx, ctx->ws + ctx->lay.table, r.table.data(), r.table.size() * sizeof(int16_t)));
  if (!r.tmpl.empty())
    CK(h2d(ctx, ctx->ws + ctx->lay.tmpl, r.tmpl.data(), r.tmpl.size() * sizeof(Template)));
  CK(h2d(ctx, ctx->ws + ctx->lay.arity, ar.data(), kMaxLabels));
  CK(cudaStreamSynchronize(ctx->stream));
  fill_dev(ctx);
  return INET_OK;
}

// Zeroes the control block and the per-net and name-slot arrays.
inet_status clear_device(inet_ctx* ctx) {
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.ctrl, 0, sizeof(Ctrl), ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.var, 0, sizeof(uint32_t) * ctx->cfg.max_vars, ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.netctr, 0, sizeof(unsigned long long) * ctx->cfg.max_nets, ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.netstat, 0, sizeof(int32_t) * ctx->cfg.max_nets, ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.netrep, 0, sizeof(uint32_t) * ctx->cfg.max_nets, ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.netmark, 0, ctx->cfg.max_nets, ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.rbmark, 0, ctx->cfg.max_nets, ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.netlive, 0, sizeof(long long) * ctx->cfg.max_nets, ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.netquota, 0, sizeof(unsigned long long) * ctx->cfg.max_nets, ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.hist, 0, sizeof(unsigned long long) * INET_MAX_RULES, ctx->stream));
  uint32_t never = 0xFFFFFFFFu;
  CK(h2d(ctx, &ctx->dev.ctrl->stop_step, &never, 4));
  CK(cudaStreamSynchronize(ctx->stream));
  return INET_OK;
}

inet_status ensure_workspace(inet_ctx* ctx) {
  if (ctx->ws_ready) return INET_OK;
  if (!ctx->ws) {
    void* p = nullptr;
    CK(cudaMalloc(&p, ctx->lay.total));
    ctx->ws = static_cast<unsigned char*>(p);
    ctx->ws_bytes = ctx->lay.total;
    ctx->own_ws = true;
  }
  ctx->ws_ready = true;
  fill_dev(ctx);
  inet_status s = clear_device(ctx);
  if (s) return s;
  return upload_rules(ctx);
}

// Copies staged nets to the device and the host-side counters to the
// control block, then places them: the uploaded range sits above the bump
// pointers, and its top part moves into slots the free rings hold (slots of
// consumed agents, finished names and freed nets), so that a context that
// frees nets reuses their memory (inet_free.cuh).  The host learns which
// slots were taken and rewrites the words it keeps: interfaces, and the
// initial pairs of nets not handed to the device yet.
inet_status upload_staged(inet_ctx* ctx) {
  const bool any = !ctx->st_nodes.empty() || !ctx->st_vars.empty() || !ctx->st_netctr.empty();
  if (!any) {
    ctx->st_a0 = ctx->a_bump;
    ctx->st_v0 = ctx->v_bump;
    return INET_OK;
  }
  const uint64_t a0 = ctx->st_a0, v0 = ctx->st_v0;
  const uint32_t ta = (uint32_t)ctx->st_nodes.size(), tv = (uint32_t)ctx->st_vars.size();
  if (a0 + ta != ctx->a_bump || v0 + tv != ctx->v_bump)
    return fail(ctx, INET_ERR_STATE, "staged nets do not end at the bump pointers");
  if (ta) CK(h2d(ctx, ctx->dev.node + a0, ctx->st_nodes.data(), (size_t)ta * sizeof(Node)));
  if (tv) {
    CK(h2d(ctx, ctx->dev.var + v0, ctx->st_vars.data(), (size_t)tv * sizeof(uint32_t)));
    if (ctx->dev.vown) CK(h2d(ctx, ctx->dev.vown + v0, ctx->st_vown.data(), (size_t)tv * sizeof(uint32_t)));
  }
  const size_t nn = ctx->st_netctr.size();
  if (nn) {
    bool run = true;  // ids id0, id0 + 1, ..: one copy and two clears
    for (size_t i = 1; i < nn && run; i++) run = ctx->st_net_ids[i] == ctx->st_net_ids[0] + (int32_t)i;
    if (run) {
      const int32_t id0 = ctx->st_net_ids[0];
      CK(h2d(ctx, ctx->dev.netctr + id0, ctx->st_netctr.data(), nn * sizeof(unsigned long long)));
      CK(cudaMemsetAsync(ctx->dev.netstat + id0, 0, nn * sizeof(int32_t), ctx->stream));
      CK(cudaMemsetAsync(ctx->dev.netrep + id0, 0, nn * sizeof(uint32_t), ctx->stream));
      if (ctx->dev.netlive) {
        CK(h2d(ctx, ctx->dev.netlive + id0, ctx->st_netlive.data(), nn * sizeof(long long)));
        CK(cudaMemsetAsync(ctx->dev.netquota + id0, 0, nn * sizeof(unsigned long long), ctx->stream));
      }
    } else {
      int32_t* dids = at<int32_t>(ctx, ctx->lay.stn_ids);
      unsigned long long* dctr = at<unsigned long long>(ctx, ctx->lay.stn_ctr);
      long long* dlive = at<long long>(ctx, ctx->lay.stn_live);
      for (size_t off = 0; off < nn; off += kReadChunk) {
        const uint32_t m = (uint32_t)std::min<size_t>(nn - off, kReadChunk);
        CK(h2d(ctx, dids, ctx->st_net_ids.data() + off, m * sizeof(int32_t)));
        CK(h2d(ctx, dctr, ctx->st_netctr.data() + off, m * sizeof(unsigned long long)));
        CK(h2d(ctx, dlive, ctx->st_netlive.data() + off, m * sizeof(long long)));
        k_net_ctr_scatter<<<(m + 255) / 256, 256, 0, ctx->stream>>>(ctx->dev, dids, dctr, dlive, m);
        CK(cudaGetLastError());
        if (off + m < nn) CK(cudaStreamSynchronize(ctx->stream));  // the id buffers are reused
      }
    }
  }
  static thread_local unsigned long long hb[2];
  static thread_local long long hl;
  static thread_local unsigned long long pl[4];
  hb[0] = ctx->a_bump;
  hb[1] = ctx->v_bump;
  hl = ctx->live;
  pl[0] = pl[1] = pl[2] = pl[3] = 0;
  CK(h2d(ctx, &ctx->dev.ctrl->a_bump, &hb[0], 8));
  CK(h2d(ctx, &ctx->dev.ctrl->v_bump, &hb[1], 8));
  CK(h2d(ctx, &ctx->dev.ctrl->live, &hl, 8));
  if (ta || tv) {
    const unsigned grid = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((std::max(ta, tv) + 255) / 256, 8ull * (uint64_t)std::max(ctx->num_sms, 1)));
    k_place_prep<<<1, 1, 0, ctx->stream>>>(ctx->dev, ta, tv);
    k_place<<<grid, 256, 0, ctx->stream>>>(ctx->dev, (uint32_t)a0, ta, (uint32_t)v0, tv);
    k_place_post<<<1, 1, 0, ctx->stream>>>(ctx->dev, (uint32_t)a0, ta, (uint32_t)v0, tv);
    CK(cudaGetLastError());
    CK(d2h(ctx, pl, &ctx->dev.ctrl->place_ka, sizeof pl));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  const uint32_t ka = (uint32_t)pl[0], kv = (uint32_t)pl[1];
  if (ka > ta || kv > tv) return fail(ctx, INET_ERR_STATE, "placement took more slots than were uploaded");
  if (ka || kv) {
    // the slots taken, in ring order
    std::vector<uint32_t> as(ka), vs(kv);
    auto seg = [&](std::vector<uint32_t>& out, const uint32_t* ring, uint64_t cap, uint64_t h) -> cudaError_t {
      const uint64_t k = out.size(), first = std::min<uint64_t>(k, cap - h);
      cudaError_t e = cudaSuccess;
      if (first) e = d2h(ctx, out.data(), ring + h, first * 4);
      if (e == cudaSuccess && k > first) e = d2h(ctx, out.data() + first, ring, (k - first) * 4);
      return e;
    };
    CK(seg(as, ctx->dev.afree, ctx->cfg.max_agents, pl[2]));
    CK(seg(vs, ctx->dev.vfree, ctx->cfg.max_vars, pl[3]));
    CK(cudaStreamSynchronize(ctx->stream));
    const uint64_t amov = a0 + ta - ka, vmov = v0 + tv - kv;
    auto ta_of = [&](uint32_t i) -> uint32_t { return i >= amov && i < a0 + ta ? as[i - amov] : i; };
    auto tr = [&](uint32_t w) -> uint32_t {
      if (is_agent(w)) return mk_agent(ta_of(idx_of(w)));
      if (is_var(w) && idx_of(w) >= vmov && idx_of(w) < v0 + tv) return mk_var(vs[idx_of(w) - vmov]);
      return w;
    };
    for (int32_t id : ctx->st_net_ids) {
      NetRec& nr = ctx->nets[(size_t)id];
      for (uint32_t& w : nr.iface) w = tr(w);
      for (Pair& p : nr.pairs) {
        p.a = ta_of(p.a);
        p.b = ta_of(p.b);
      }
    }
  }
  ctx->a_bump = a0 + ta - ka;
  ctx->v_bump = v0 + tv - kv;
  for (int32_t id : ctx->st_net_ids) ctx->nets[(size_t)id].uploaded = true;
  ctx->st_nodes.clear();
  ctx->st_vars.clear();
  ctx->st_vown.clear();
  ctx->st_netctr.clear();
  ctx->st_net_ids.clear();
  ctx->st_netlive.clear();
  ctx->st_a0 = ctx->a_bump;
  ctx->st_v0 = ctx->v_bump;
  ctx->snap_valid = false;
  ctx->arena_gen++;
  return INET_OK;
}

// Host copies of the per-net counters, refreshed from the device when a
// reduction changed them (nets not uploaded yet keep their host values).
inet_status ensure_net_counters(inet_ctx* ctx) {
  if (ctx->h_net_valid || ctx->host_only || !ctx->ws_ready) return INET_OK;
  const size_t nn = ctx->nets.size();
  if (nn) {
    CK(d2h(ctx, ctx->h_netctr.data(), ctx->dev.netctr, nn * sizeof(unsigned long long)));
    CK(d2h(ctx, ctx->h_netstat.data(), ctx->dev.netstat, nn * sizeof(int32_t)));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  for (size_t i = 0; i < ctx->st_net_ids.size(); i++) {
    ctx->h_netctr[(size_t)ctx->st_net_ids[i]] = ctx->st_netctr[i];
    ctx->h_netstat[(size_t)ctx->st_net_ids[i]] = 0;
  }
  ctx->h_net_valid = true;
  return INET_OK;
}

// Numerals of m nets whose interface words are at droot, into dval, queued
// on stream st: a bounded walk per net, then list ranking of
// the whole arena when some walk ran out (inet_readback.cuh).  The arena is
// quiescent for these nets (finished), so the slots below the host bump
// counters hold every element of their lists.  No readback may be in
// flight when the scratch grows.
inet_status read_nats_device(inet_ctx* ctx, cudaStream_t st, const uint32_t* droot, uint32_t m, int s_label,
                             int z_label, unsigned long long* dval) {
  const uint32_t na = (uint32_t)ctx->a_bump, nv = (uint32_t)ctx->v_bump;
  if (!ctx->jump_ctl) CK(cudaMalloc(&ctx->jump_ctl, sizeof(uint32_t) * kJumpCtl));
  if (na > ctx->jump_cap) {
    // (successor, weight) twice and the list, per agent slot in use
    const uint64_t want = std::min<uint64_t>(std::max<uint64_t>(na, 2 * ctx->jump_cap), ctx->cfg.max_agents);
    if (ctx->jump_buf) CK(cudaFree(ctx->jump_buf));
    ctx->jump_buf = nullptr;
    ctx->jump_cap = 0;
    CK(cudaMalloc(&ctx->jump_buf, (sizeof(uint2) * 2 + sizeof(uint32_t)) * want));
    ctx->jump_cap = want;
  }
  uint2* b0 = ctx->jump_buf;
  uint2* b1 = ctx->jump_buf + ctx->jump_cap;
  uint32_t* lst = reinterpret_cast<uint32_t*>(ctx->jump_buf + 2 * ctx->jump_cap);
  uint32_t* ctl = ctx->jump_ctl;
  uint32_t* cnt = ctl + kJumpCtl - 1;
  uint8_t* mark = at<uint8_t>(ctx, ctx->lay.rbmark);
  CK(cudaMemsetAsync(ctl, 0, sizeof(uint32_t) * kJumpCtl, st));
  const unsigned nb = (m + 255) / 256;
  // every net is walked for kWalkMin S agents; the rest of each longer
  // numeral is ranked on a list of its net's agents only
  k_nat_walk<<<nb, 256, 0, st>>>(ctx->dev, droot, m, na, nv, s_label, z_label, kWalkMin, dval, ctl);
  CK(cudaGetLastError());
  if (na == 0) return INET_OK;
  const unsigned grid = (unsigned)std::min<uint64_t>((na + 255) / 256, 8ull * (uint64_t)std::max(ctx->num_sms, 1));
  k_nat_mark<<<nb, 256, 0, st>>>(ctx->dev, dval, m, na, mark);
  k_nat_list<<<grid, 256, 0, st>>>(ctx->dev, na, nv, s_label, z_label, mark, ctl, lst, cnt, b0);
  CK(cudaGetLastError());
  // a list of L agents is ranked after ceil(log2 L) rounds, L <= na
  uint32_t rounds = 1;
  while ((1ull << rounds) < na && rounds < (uint32_t)kJumpCtl - 4) rounds++;
  for (uint32_t r = 0; r < rounds; r++) {
    k_nat_lround<<<grid, 256, 0, st>>>(na, r, ctl, lst, cnt, b0, b1);
    k_nat_jump_check<<<nb, 256, 0, st>>>(dval, m, na, r, ctl, b0, b1);
  }
  k_nat_unmark<<<nb, 256, 0, st>>>(ctx->dev, dval, m, na, mark);
  k_nat_jump_gather<<<nb, 256, 0, st>>>(dval, m, na, ctl, b0, b1);
  CK(cudaGetLastError());
  return INET_OK;
}

// A device buffer of at least `bytes` (grown, contents dropped).
cudaError_t dev_buf(inet_ctx::DevBuf& b, size_t bytes) {
  if (b.cap >= bytes) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  const size_t want = std::max(bytes, b.cap * 2);
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e == cudaSuccess) b.cap = want;
  return e;
}

// The text of net `id`'s interface after ->col and ->sub, rendered on the
// device (inet_textdev.cuh) and copied to `out`.  *ok = false when the net
// is not a forest (a subterm reached twice, or a cycle through the
// interface): the caller renders it on the host, whose walk bounds such
// terms.
inet_status read_text_device(inet_ctx* ctx, int32_t id, std::string& out, bool* ok, uint64_t* reached_out,
                             int64_t* live_out) {
  *ok = false;
  *reached_out = 0;
  *live_out = -1;
  const NetRec& nr = ctx->nets[(size_t)id];
  const uint32_t na = (uint32_t)ctx->a_bump, nv = (uint32_t)ctx->v_bump, nroots = (uint32_t)nr.iface.size();
  out.clear();
  if (nroots == 0) {
    *ok = true;
    return INET_OK;
  }
  const CompiledRules& R = ctx->rules;
  cudaStream_t st = ctx->stream;
  // the label table: lengths, offsets and the characters of every label
  if (!ctx->txt_labels_ok) {
    const size_t L = R.labels.size();
    std::vector<uint8_t> len(kMaxLabels, 0);
    std::vector<uint32_t> off(kMaxLabels, 0);
    std::string chars;
    for (size_t l = 0; l < L && l < kMaxLabels; l++) {
      off[l] = (uint32_t)chars.size();
      len[l] = (uint8_t)std::min<size_t>(R.labels[l].size(), 255);
      chars.append(R.labels[l], 0, len[l]);
    }
    const size_t bytes = kMaxLabels * (1 + 4) + chars.size() + 16;
    CK(dev_buf(ctx->txt_labels, bytes));
    unsigned char* tb = static_cast<unsigned char*>(ctx->txt_labels.p);
    CK(h2d(ctx, tb, len.data(), kMaxLabels));
    CK(h2d(ctx, tb + kMaxLabels, off.data(), kMaxLabels * 4));
    if (!chars.empty()) CK(h2d(ctx, tb + kMaxLabels * 5, chars.data(), chars.size()));
    CK(cudaStreamSynchronize(st));
    ctx->txt_labels_ok = true;
  }
  const uint8_t* lablen = static_cast<const uint8_t*>(ctx->txt_labels.p);
  const uint32_t* laboff = reinterpret_cast<const uint32_t*>(lablen + kMaxLabels);
  const char* labchars = reinterpret_cast<const char*>(lablen + kMaxLabels * 5);
  const unsigned blocks_max = 8u * (unsigned)std::max(ctx->num_sms, 1);
  auto grid_for = [&](uint64_t n) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, blocks_max));
  };
  // dense ids of the net's live agents
  CK(dev_buf(ctx->txt_dead, std::max<size_t>(na, 1)));
  CK(dev_buf(ctx->txt_cid, sizeof(uint32_t) * 2 * std::max<size_t>(na, 1)));
  CK(dev_buf(ctx->txt_roots, sizeof(uint32_t) * nroots));
  CK(dev_buf(ctx->txt_ctl, sizeof(uint32_t) * kTxtCtl + 2 * sizeof(TxtElem)));
  uint8_t* dead = static_cast<uint8_t*>(ctx->txt_dead.p);
  uint32_t* cid = static_cast<uint32_t*>(ctx->txt_cid.p);
  uint32_t* slot = cid + std::max<size_t>(na, 1);
  uint32_t* droots = static_cast<uint32_t*>(ctx->txt_roots.p);
  uint32_t* ctl = static_cast<uint32_t*>(ctx->txt_ctl.p);
  if (na) {
    CK(cudaMemsetAsync(dead, 0, na, st));
    CK(cudaMemsetAsync(cid, 0xFF, sizeof(uint32_t) * na, st));
  }
  CK(cudaMemsetAsync(ctl, 0, sizeof(uint32_t) * kTxtCtl, st));
  CK(h2d(ctx, droots, nr.iface.data(), sizeof(uint32_t) * nroots));
  const uint32_t net = (uint32_t)id;
  k_txt_free_marks<<<grid_for(na), 256, 0, st>>>(ctx->dev, na, dead);
  k_txt_compact<<<grid_for(na), 256, 0, st>>>(ctx->dev, net, na, dead, cid, slot, ctl);
  CK(cudaGetLastError());
  static thread_local uint32_t ncount;
  CK(d2h(ctx, &ncount, ctl + 5, sizeof ncount));
  CK(cudaStreamSynchronize(st));
  const uint32_t n_c = ncount;
  const uint64_t n_el64 = 4ull * n_c + nroots;
  if (n_c > na || n_el64 >= kTxtEnd) return INET_OK;  // host path
  const uint32_t n_el = (uint32_t)n_el64;
  CK(dev_buf(ctx->txt_parent, sizeof(uint32_t) * std::max<size_t>(n_c, 1)));
  CK(dev_buf(ctx->txt_el, sizeof(TxtElem) * 2 * (size_t)n_el));
  uint32_t* parent = static_cast<uint32_t*>(ctx->txt_parent.p);
  TxtElem* b0 = static_cast<TxtElem*>(ctx->txt_el.p);
  TxtElem* b1 = b0 + n_el;
  if (n_c) CK(cudaMemsetAsync(parent, 0xFF, sizeof(uint32_t) * n_c, st));
  const unsigned gel = grid_for(n_el);
  k_txt_parent<<<grid_for(std::max(n_c, nroots)), 256, 0, st>>>(ctx->dev, n_c, na, nv, slot, cid, droots, nroots,
                                                                ctx->dev.arity, parent, ctl);
  k_txt_init<<<grid_for(std::max(n_c, nroots)), 256, 0, st>>>(ctx->dev, n_c, na, nv, slot, cid, droots, nroots,
                                                              ctx->dev.arity, lablen, parent, b0, b1, ctl);
  // the head of the list (root 0's first element) into ctl[2]
  k_txt_head<<<1, 1, 0, st>>>(ctx->dev, n_c, na, nv, cid, droots, ctl);
  uint32_t rounds = 1;
  while (rounds < 64 && (1ull << rounds) < (uint64_t)n_el) rounds++;
  for (uint32_t r = 0; r < rounds && 8 + r < (uint32_t)kTxtCtl; r++) {
    k_txt_round<<<gel, 256, 0, st>>>(n_el, r, ctl, b0, b1);
    k_txt_check_head<<<1, 1, 0, st>>>(n_el, r, ctl, b0, b1);
  }
  k_txt_copy_head<<<1, 1, 0, st>>>(ctl, b0, b1, reinterpret_cast<TxtElem*>(ctl + kTxtCtl));
  CK(cudaGetLastError());
  static thread_local uint32_t hctl[kTxtCtl + 2 * sizeof(TxtElem) / 4];
  CK(d2h(ctx, hctl, ctl, sizeof(uint32_t) * kTxtCtl + sizeof(TxtElem)));
  CK(cudaStreamSynchronize(st));
  TxtElem he;
  memcpy(&he, hctl + kTxtCtl, sizeof he);
  if (hctl[0] || he.succ != kTxtEnd) return INET_OK;  // not a forest, or not ranked: host path
  const TxtElem* fin = (hctl[1] & 1u) ? b1 : b0;
  const unsigned long long total_chars = he.chars;
  const uint32_t total_names = he.names;
  unsigned long long name_chars = 0;
  uint32_t *num = nullptr, *noff = nullptr, *nlen = nullptr;
  if (total_names) {
    CK(dev_buf(ctx->txt_first, sizeof(uint32_t) * std::max<size_t>(nv, 1)));
    CK(dev_buf(ctx->txt_names, sizeof(uint32_t) * 5 * ((size_t)total_names + 1)));
    uint32_t* first = static_cast<uint32_t*>(ctx->txt_first.p);
    uint32_t* key = static_cast<uint32_t*>(ctx->txt_names.p);
    uint32_t* flag = key + (total_names + 1);
    num = flag + (total_names + 1);
    nlen = num + (total_names + 1);
    noff = nlen + (total_names + 1);
    CK(cudaMemsetAsync(first, 0xFF, sizeof(uint32_t) * std::max<size_t>(nv, 1), st));
    CK(cudaMemsetAsync(key, 0, sizeof(uint32_t) * (total_names + 1), st));
    CK(cudaMemsetAsync(flag, 0, sizeof(uint32_t) * (total_names + 1), st));
    const unsigned gn = (total_names + 255) / 256;
    k_txt_names<<<gel, 256, 0, st>>>(ctx->dev, n_el, n_c, nv, droots, slot, fin, total_names, first, key);
    k_txt_firsts<<<gn, 256, 0, st>>>(total_names, first, key, flag);
    k_rs_scan<<<1, 1024, 0, st>>>(flag, total_names + 1);  // exclusive: rank of each first occurrence
    k_txt_numbers<<<gn, 256, 0, st>>>(total_names, first, key, flag, num, nlen);
    CK(cudaMemsetAsync(nlen + total_names, 0, sizeof(uint32_t), st));
    CK(cudaMemcpyAsync(noff, nlen, sizeof(uint32_t) * (total_names + 1), cudaMemcpyDeviceToDevice, st));
    k_rs_scan<<<1, 1024, 0, st>>>(noff, total_names + 1);  // noff[total_names] = all name characters
    CK(cudaGetLastError());
    static thread_local uint32_t nc;
    CK(d2h(ctx, &nc, noff + total_names, sizeof nc));
    CK(cudaStreamSynchronize(st));
    name_chars = nc;
  }
  const size_t len = (size_t)(total_chars + name_chars);
  CK(dev_buf(ctx->txt_out, std::max<size_t>(len, 1)));
  char* dout = static_cast<char*>(ctx->txt_out.p);
  k_txt_scatter<<<gel, 256, 0, st>>>(ctx->dev, n_el, n_c, nv, droots, slot, nroots, fin, total_chars, total_names, name_chars,
                                     num, noff, nlen, ctx->dev.arity, labchars, laboff, lablen, dout,
                                     (unsigned long long)len, ctl);
  CK(cudaGetLastError());
  out.resize(len);
  if (len) CK(d2h(ctx, &out[0], dout, len));
  static thread_local uint32_t tail[4];
  CK(d2h(ctx, tail, ctl, sizeof tail));
  CK(cudaStreamSynchronize(st));
  *ok = tail[0] == 0;
  *reached_out = tail[3];
  *live_out = n_c;
  return INET_OK;
}

inet_status build_graph(inet_ctx* ctx, int block, int grid, size_t smem) {
  if (ctx->gexec && ctx->g_block == block && ctx->g_grid == grid) return INET_OK;
  if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
  if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
  CK(cudaGraphCreate(&ctx->graph, 0));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, ctx->graph, 1, cudaGraphCondAssignDefault));
  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  memset(cp_raw, 0, sizeof cp_raw);
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  CK(cudaGraphAddNode(&cn, ctx->graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  Dev d = ctx->dev;
  d.cond = h;
  d.use_cond = 1;
  void* args[] = {&d};
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof kp);
  kp.func = (void*)loop_kernels(ctx->dev.vown != nullptr).step;
  kp.gridDim = dim3((unsigned)grid);
  kp.blockDim = dim3((unsigned)block);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  cudaGraphNode_t kn;
  CK(cudaGraphAddKernelNode(&kn, body, nullptr, 0, &kp));
  CK(cudaGraphInstantiate(&ctx->gexec, ctx->graph, 0));
  ctx->g_block = block;
  ctx->g_grid = grid;
  return INET_OK;
}

void drop_graph(inet_ctx* ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->gexec = nullptr;
  ctx->graph = nullptr;
  ctx->g_block = ctx->g_grid = 0;
}

inet_status ensure_snapshot(inet_ctx* ctx) {
  if (ctx->snap_valid) return INET_OK;
  ctx->snap_nodes.resize(ctx->a_bump);
  ctx->snap_vars.resize(ctx->v_bump);
  if (ctx->a_bump)
    CK(d2h(ctx, ctx->snap_nodes.data(), ctx->dev.node, ctx->a_bump * sizeof(Node)));
  if (ctx->v_bump)
    CK(d2h(ctx, ctx->snap_vars.data(), ctx->dev.var, ctx->v_bump * sizeof(uint32_t)));
  Ctrl hc;
  CK(d2h(ctx, &hc, ctx->dev.ctrl, sizeof(Ctrl)));
  CK(cudaStreamSynchronize(ctx->stream));
  // free agent slots: ring entries [a_head, a_tail)
  std::vector<uint8_t> is_free(ctx->a_bump, 0);
  const uint64_t cap = ctx->cfg.max_agents;
  uint64_t nfree = hc.a_tail > hc.a_head ? std::min<uint64_t>(hc.a_tail - hc.a_head, cap) : 0;
  if (nfree) {
    std::vector<uint32_t> ring(nfree);
    uint64_t h = hc.a_head % cap;
    uint64_t first = std::min<uint64_t>(nfree, cap - h);
    CK(d2h(ctx, ring.data(), ctx->dev.afree + h, first * 4));
    if (nfree > first)
      CK(d2h(ctx, ring.data() + first, ctx->dev.afree, (nfree - first) * 4));
    CK(cudaStreamSynchronize(ctx->stream));
    for (uint32_t s : ring)
      if (s < ctx->a_bump) is_free[s] = 1;
  }
  ctx->snap_live.assign(ctx->nets.size(), 0);
  for (uint64_t i = 0; i < ctx->a_bump; i++) {
    if (is_free[i]) continue;
    uint32_t net = (uint32_t)ctx->snap_nodes[i].head >> 8;
    if (net < ctx->snap_live.size()) ctx->snap_live[net]++;
  }
  ctx->snap_valid = true;
  ctx->snap_gen++;
  return INET_OK;
}

inet_status check_net(inet_ctx* ctx, int32_t id) {
  if (id < 0 || (size_t)id >= ctx->nets.size() || !ctx->nets[(size_t)id].used)
    return fail(ctx, INET_ERR_INVALID_ARG, "unknown net id " + std::to_string(id));
  return INET_OK;
}

// Uploads staged nets and appends the initial active pairs of the listed
// nets to the current frontier on the device.
inet_status stage_nets(inet_ctx* ctx, const int32_t* net_ids, int32_t n) {
  for (int32_t i = 0; i < n; i++) {
    inet_status s = check_net(ctx, net_ids[i]);
    if (s) return s;
    if (ctx->nets[(size_t)net_ids[i]].started) return fail(ctx, INET_ERR_INVALID_ARG, "net already staged or reduced");
  }
  inet_status s = ensure_workspace(ctx);
  if (s) return s;
  s = upload_staged(ctx);
  if (s) return s;
  std::vector<Pair> add;
  for (int32_t i = 0; i < n; i++) {
    const NetRec& nr = ctx->nets[(size_t)net_ids[i]];
    add.insert(add.end(), nr.pairs.begin(), nr.pairs.end());
  }
  const uint32_t cur = ctx->step & 1u;
  if ((uint64_t)ctx->fcount[cur] + add.size() > ctx->cfg.max_pairs)
    return fail(ctx, INET_ERR_ARENA_FULL, "frontier capacity exceeded");
  for (int32_t i = 0; i < n; i++) {
    NetRec& nr = ctx->nets[(size_t)net_ids[i]];
    nr.pairs.clear();
    nr.pairs.shrink_to_fit();
    nr.started = true;
  }
  if (add.empty()) return INET_OK;
  CK(h2d(ctx, ctx->dev.front[cur] + ctx->fcount[cur], add.data(), add.size() * sizeof(Pair)));
  ctx->fcount[cur] += (uint32_t)add.size();
  CK(h2d(ctx, &ctx->dev.ctrl->fcount[cur], &ctx->fcount[cur], 4));
  CK(cudaStreamSynchronize(ctx->stream));
  return INET_OK;
}

// The id the k-th net of a load would get (k = 0, 1, ..): ids released by
// inet_free_nets first (most recent first), then never-used ones.  Nothing
// is committed; -1 when the context is out of net slots.
int32_t peek_net_id(const inet_ctx* ctx, size_t k) {
  const size_t nf = ctx->free_net_ids.size();
  if (k < nf) return ctx->free_net_ids[nf - 1 - k];
  const size_t fresh = ctx->nets.size() + (k - nf);
  return fresh < ctx->cfg.max_nets ? (int32_t)fresh : -1;
}

// Commits net `id` (the next id peek_net_id gave) with its record.
void commit_net(inet_ctx* ctx, int32_t id, NetRec&& nr, unsigned long long ctr, long long agents) {
  if (!ctx->free_net_ids.empty() && ctx->free_net_ids.back() == id) {
    ctx->free_net_ids.pop_back();
    ctx->nets[(size_t)id] = std::move(nr);
    ctx->h_netctr[(size_t)id] = ctr;
    ctx->h_netstat[(size_t)id] = 0;
  } else {
    ctx->nets.push_back(std::move(nr));
    ctx->h_netctr.push_back(ctr);
    ctx->h_netstat.push_back(0);
  }
  ctx->st_netctr.push_back(ctr);
  ctx->st_net_ids.push_back(id);
  ctx->st_netlive.push_back(agents);
}

// A batch of nets parsed and flattened on their own (agent and name slots
// from 0, net id 0), ready to be placed in a context (commit_batch).  Parsing
// reads only the compiled rules, so it may run on another thread while the
// context reduces.
}  // namespace

struct inet_parsed {
  std::vector<FlatNet> fns;
  std::vector<int> rcs;
  std::vector<std::string> errs;
  std::vector<uint8_t> taken;   // loaded into a context already
  uint64_t rules_gen = 0;       // the rule set it was parsed with
};

namespace {

void parse_batch(const CompiledRules& rules, uint64_t rules_gen, const char* buf, const uint64_t* offsets, int32_t n,
                 inet_parsed& pb) {
  pb.fns.assign((size_t)n, FlatNet());
  pb.rcs.assign((size_t)n, 0);
  pb.errs.assign((size_t)n, std::string());
  pb.taken.assign((size_t)n, 0);
  pb.rules_gen = rules_gen;
  // body(lo, hi) over [0, n) in ranges of 16 nets on the host pool
  HostPool::get().run(n, 16, [&](int32_t lo, int32_t hi) {
    for (int32_t i = lo; i < hi; i++)
      pb.rcs[(size_t)i] = flatten_net(std::string(buf + offsets[i], offsets[i + 1] - offsets[i]), rules, 0, 0, 0,
                                      pb.fns[(size_t)i], pb.errs[(size_t)i]);
  });
}

// Places nets [first, first + n) of a parsed batch: in order, ids first
// (released ones, then never-used ones); the first net that failed to parse
// or does not fit ends the batch, the nets before it stay loaded.  Each
// net's indices are shifted to its place and its net id written into its
// agent records, on the host pool, and the result appended to the staging
// vectors.
inet_status commit_batch(inet_ctx* ctx, inet_parsed& pb, int32_t first, int32_t n, int32_t* ids_out,
                         int32_t* n_loaded_out) {
  *n_loaded_out = 0;
  if (!ctx->host_only) {
    DeviceGuard g(ctx->device);
    inet_status s = ensure_workspace(ctx);
    if (s) return s;
  }
  std::vector<int32_t> pid((size_t)n);
  for (int32_t i = 0; i < n; i++) pid[(size_t)i] = peek_net_id(ctx, (size_t)i);
  FlatNet* fns = pb.fns.data() + first;
  const int* rcs = pb.rcs.data() + first;
  const std::string* errs = pb.errs.data() + first;
  auto on_threads = [](int32_t cnt, const HostPool::Body& body) { HostPool::get().run(cnt, 16, body); };
  std::vector<uint64_t> a_at((size_t)n + 1), v_at((size_t)n + 1);
  a_at[0] = ctx->a_bump;
  v_at[0] = ctx->v_bump;
  int32_t m = 0;
  inet_status stop = INET_OK;
  std::string stop_msg;
  for (; m < n; m++) {
    const FlatNet& fn = fns[(size_t)m];
    if (rcs[(size_t)m]) {
      stop = (inet_status)rcs[(size_t)m];
      stop_msg = errs[(size_t)m];
      break;
    }
    if (pid[(size_t)m] < 0) {
      stop = INET_ERR_ARENA_FULL;
      stop_msg = "no free net slot";
      break;
    }
    if (a_at[(size_t)m] + fn.nodes.size() > ctx->cfg.max_agents || v_at[(size_t)m] + fn.vars.size() > ctx->cfg.max_vars) {
      stop = INET_ERR_ARENA_FULL;
      stop_msg = "net does not fit the arena";
      break;
    }
    a_at[(size_t)m + 1] = a_at[(size_t)m] + fn.nodes.size();
    v_at[(size_t)m + 1] = v_at[(size_t)m] + fn.vars.size();
  }
  if (m > 0) {
    if (ctx->st_nodes.empty() && ctx->st_vars.empty() && ctx->st_netctr.empty()) {
      ctx->st_a0 = ctx->a_bump;
      ctx->st_v0 = ctx->v_bump;
    }
    // staged entries continue the staging vectors: slot a_at[i] is entry
    // a_at[i] - st_a0 (likewise for names)
    const size_t na0 = ctx->st_nodes.size(), nv0 = ctx->st_vars.size();
    ctx->st_nodes.resize(na0 + (size_t)(a_at[(size_t)m] - a_at[0]));
    ctx->st_vars.resize(nv0 + (size_t)(v_at[(size_t)m] - v_at[0]));
    ctx->st_vown.resize(nv0 + (size_t)(v_at[(size_t)m] - v_at[0]));
    Node* dn = ctx->st_nodes.data() + na0;
    uint32_t* dv = ctx->st_vars.data() + nv0;
    uint32_t* downer = ctx->st_vown.data() + nv0;
    on_threads(m, [&](int32_t lo, int32_t hi) {
      for (int32_t i = lo; i < hi; i++) {
        FlatNet& fn = fns[(size_t)i];
        const uint32_t ab = (uint32_t)a_at[(size_t)i], vb = (uint32_t)v_at[(size_t)i];
        auto shift = [ab, vb](uint32_t w) -> uint32_t {
          return is_agent(w) ? mk_agent(idx_of(w) + ab) : is_var(w) ? mk_var(idx_of(w) + vb) : w;
        };
        const int32_t head_net = pid[(size_t)i] << 8;
        Node* o = dn + (a_at[(size_t)i] - a_at[0]);
        for (const Node& nd : fn.nodes) {
          Node x = nd;
          x.head = (x.head & 0xFF) | head_net;
          for (uint32_t& w : x.aux) w = shift(w);
          *o++ = x;
        }
        uint32_t* ov = dv + (v_at[(size_t)i] - v_at[0]);
        for (uint32_t w : fn.vars) *ov++ = shift(w);
        std::fill_n(downer + (v_at[(size_t)i] - v_at[0]), fn.vars.size(), (uint32_t)pid[(size_t)i]);
        for (uint32_t& w : fn.iface) w = shift(w);
        for (Pair& p : fn.pairs) {
          p.a += ab;
          p.b += ab;
        }
      }
    });
    ctx->a_bump = a_at[(size_t)m];
    ctx->v_bump = v_at[(size_t)m];
    ctx->live += (int64_t)(a_at[(size_t)m] - a_at[0]);
    ctx->st_netctr.reserve(ctx->st_netctr.size() + (size_t)m);
    ctx->st_net_ids.reserve(ctx->st_net_ids.size() + (size_t)m);
    ctx->nets.reserve(ctx->nets.size() + (size_t)m);
    for (int32_t i = 0; i < m; i++) {
      FlatNet& fn = fns[(size_t)i];
      const unsigned long long ctr = (unsigned long long)fn.pairs.size() << kNetPairShift;
      NetRec nr;
      nr.used = true;
      nr.iface = std::move(fn.iface);
      nr.pairs = std::move(fn.pairs);
      commit_net(ctx, pid[(size_t)i], std::move(nr), ctr, (long long)fn.nodes.size());
      ids_out[i] = pid[(size_t)i];
      pb.taken[(size_t)(first + i)] = 1;
    }
    ctx->snap_valid = false;
    ctx->arena_gen++;
    *n_loaded_out = m;
  }
  if (stop) return fail(ctx, stop, stop_msg);
  return INET_OK;
}

// Device buffers of one control run, freed on every exit.
struct CtlBufs {
  std::vector<void*> p;
  template <class T>
  bool get(T** out, size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return false;
    p.push_back(q);
    *out = static_cast<T*>(q);
    return true;
  }
  ~CtlBufs() {
    for (void* q : p) cudaFree(q);
  }
};

}  // namespace

extern "C" {

inet_status inet_workspace_bytes(const inet_arena_cfg* cfg, size_t* bytes_out) {
  if (!bytes_out) return INET_ERR_INVALID_ARG;
  inet_arena_cfg c = with_defaults(cfg);
  if (!valid_cfg(c)) return INET_ERR_INVALID_ARG;
  *bytes_out = layout_of(c).total;
  return INET_OK;
}

inet_status inet_create(inet_ctx** out, int device, void* stream, const inet_arena_cfg* cfg) {
  if (!out) return INET_ERR_INVALID_ARG;
  *out = nullptr;
  inet_arena_cfg c = with_defaults(cfg);
  if (!valid_cfg(c)) return INET_ERR_INVALID_ARG;
  inet_ctx* ctx = new inet_ctx();
  ctx->cfg = c;
  ctx->lay = layout_of(c);
  ctx->device = device;
  ctx->host_only = device < 0;
  if (const char* e = getenv("INET_JIT")) ctx->jit_on = strcmp(e, "0") != 0;
  if (!ctx->host_only) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device >= n) {
      delete ctx;
      return INET_ERR_NO_DEVICE;
    }
    DeviceGuard g(device);
    if (stream) {
      ctx->stream = static_cast<cudaStream_t>(stream);
    } else if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) == cudaSuccess) {
      ctx->own_stream = true;
    } else {
      delete ctx;
      return INET_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
      delete ctx;
      return INET_ERR_CUDA;
    }
  }
  *out = ctx;
  return INET_OK;
}

inet_status inet_attach_workspace(inet_ctx* ctx, void* dptr, size_t bytes) {
  if (!ctx || !dptr) return INET_ERR_INVALID_ARG;
  if (ctx->host_only) return fail(ctx, INET_ERR_NO_DEVICE, "host-only context");
  if (ctx->ws) return fail(ctx, INET_ERR_STATE, "workspace already set");
  if (bytes < ctx->lay.total || (reinterpret_cast<uintptr_t>(dptr) & 255))
    return fail(ctx, INET_ERR_INVALID_ARG, "workspace too small or not 256-byte aligned");
  DeviceGuard g(ctx->device);
  ctx->ws = static_cast<unsigned char*>(dptr);
  ctx->ws_bytes = bytes;
  ctx->own_ws = false;
  return ensure_workspace(ctx);
}

void inet_destroy(inet_ctx* ctx) {
  if (!ctx) return;
  if (!ctx->host_only) {
    DeviceGuard g(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->rb_stream) {
      cudaStreamSynchronize(ctx->rb_stream);
      cudaStreamDestroy(ctx->rb_stream);
    }
    if (ctx->rb_ready) cudaEventDestroy(ctx->rb_ready);
    if (ctx->rb_after) cudaEventDestroy(ctx->rb_after);
    if (ctx->rb_host_roots) cudaFreeHost(ctx->rb_host_roots);
    if (ctx->rb_host_vals) cudaFreeHost(ctx->rb_host_vals);
    if (ctx->jump_buf) cudaFree(ctx->jump_buf);
    if (ctx->jump_ctl) cudaFree(ctx->jump_ctl);
    for (auto* b : {&ctx->txt_dead, &ctx->txt_cid, &ctx->txt_parent, &ctx->txt_el, &ctx->txt_roots, &ctx->txt_first,
                    &ctx->txt_names, &ctx->txt_out, &ctx->txt_ctl, &ctx->txt_labels})
      if (b->p) cudaFree(b->p);
    drop_graph(ctx);
    if (ctx->own_ws && ctx->ws) cudaFree(ctx->ws);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  }
  delete ctx;
}

inet_status inet_load_rules(inet_ctx* ctx, const char* text, size_t len) {
  if (!ctx || (!text && len)) return INET_ERR_INVALID_ARG;
  for (auto& n : ctx->nets)
    if (n.used) return fail(ctx, INET_ERR_STATE, "rules cannot change while nets are loaded (inet_reset first)");
  CompiledRules r;
  std::string err;
  int rc = compile_rules(std::string(text ? text : "", len), r, err);
  if (rc) return fail(ctx, rc, err);
  ctx->rules = std::move(r);
  ctx->have_rules = true;
  ctx->rules_gen++;
  ctx->txt_labels_ok = false;
  ctx->jit_state[0] = ctx->jit_state[1] = 0;
  ctx->jit_fn[0] = ctx->jit_fn[1] = nullptr;
  ctx->jit_msg.clear();
  if (ctx->host_only) return INET_OK;
  DeviceGuard g(ctx->device);
  drop_graph(ctx);
  return upload_rules(ctx);
}

inet_status inet_set_jit(inet_ctx* ctx, int32_t enable) {
  if (!ctx || (enable != 0 && enable != 1)) return INET_ERR_INVALID_ARG;
  ctx->jit_on = enable != 0;
  return INET_OK;
}

inet_status inet_jit_info(const inet_ctx* ctx, inet_jit_info_t* out) {
  if (!ctx || !out) return INET_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  const int track = (ctx->cfg.flags & INET_ARENA_FREE_NETS) ? 1 : 0;
  out->enabled = ctx->jit_on ? 1 : 0;
  out->state = ctx->jit_state[track];
  out->source = ctx->jit_source;
  out->compile_ms = ctx->jit_ms;
  out->launches = ctx->jit_launches;
  snprintf(out->msg, sizeof out->msg, "%s", ctx->jit_msg.c_str());
  return INET_OK;
}

inet_status inet_jit_build(inet_ctx* ctx, int32_t track) {
  if (!ctx || track < -1 || track > 1) return INET_ERR_INVALID_ARG;
  if (track < 0) track = (ctx->cfg.flags & INET_ARENA_FREE_NETS) ? 1 : 0;
  if (!ctx->have_rules || ctx->rules.tmpl.empty()) return fail(ctx, INET_ERR_STATE, "no rules loaded");
  if (ctx->host_only) {
    JitResult jr;
    std::string err;
    if (!jit_async(ctx->rules.tmpl.data(), ctx->rules.tmpl.size(), track != 0, "sm_103a", false, &jr, &err))
      return fail(ctx, INET_ERR_CUDA, err);
    ctx->jit_ms = jr.compile_ms;
    ctx->jit_source = jr.from_memory ? 3 : (jr.from_disk ? 2 : 1);
    return INET_OK;
  }
  DeviceGuard g(ctx->device);
  const bool was_on = ctx->jit_on;
  ctx->jit_on = true;
  const void* f = jit_kernel(ctx, track);
  ctx->jit_on = was_on;
  return f ? INET_OK : fail(ctx, INET_ERR_CUDA, ctx->jit_msg);
}

inet_status inet_rule_count(const inet_ctx* ctx, int32_t* n_out) {
  if (!ctx || !n_out) return INET_ERR_INVALID_ARG;
  *n_out = (int32_t)ctx->rules.tmpl.size();
  return INET_OK;
}

inet_status inet_rule_info(const inet_ctx* ctx, int32_t rule, inet_rule_desc* out) {
  if (!ctx || !out || rule < 0 || (size_t)rule >= ctx->rules.tmpl.size()) return INET_ERR_INVALID_ARG;
  const CompiledRules& r = ctx->rules;
  const Template& t = r.tmpl[(size_t)rule];
  memset(out, 0, sizeof *out);
  snprintf(out->name, sizeof out->name, "%s", r.rule_names[(size_t)rule].c_str());
  // the LHS symbols are the two labels whose table entry points at this rule
  int L = r.n_labels();
  for (int i = 0; i < L; i++)
    for (int j = 0; j < L; j++)
      if (r.table[(size_t)i * L + j] == (int16_t)(rule << 1)) {
        out->arity_alpha = r.arity[(size_t)i];
        out->arity_beta = r.arity[(size_t)j];
      }
  out->n_new = t.n_new;
  for (int j = 0; j < t.n_new; j++) out->new_ports += r.arity[t.lab[j]];
  out->n_fresh = t.n_fresh;
  out->n_link = t.n_link;
  return INET_OK;
}

inet_status inet_load_net(inet_ctx* ctx, const char* text, size_t len, int32_t* net_id_out) {
  if (!ctx || (!text && len) || !net_id_out) return INET_ERR_INVALID_ARG;
  if (!ctx->have_rules) return fail(ctx, INET_ERR_STATE, "load rules first");
  if (ctx->poisoned) return fail(ctx, INET_ERR_STATE, "context needs inet_reset after a fatal error");
  const int32_t id = peek_net_id(ctx, 0);
  if (id < 0) return fail(ctx, INET_ERR_ARENA_FULL, "no free net slot");
  if (!ctx->host_only) {
    DeviceGuard g(ctx->device);
    inet_status s = ensure_workspace(ctx);
    if (s) return s;
  }
  const uint32_t slot = (uint32_t)id;
  FlatNet fn;
  std::string err;
  int rc = flatten_net(std::string(text ? text : "", len), ctx->rules, slot, (uint32_t)ctx->a_bump,
                       (uint32_t)ctx->v_bump, fn, err);
  if (rc) return fail(ctx, rc, err);
  if (ctx->a_bump + fn.nodes.size() > ctx->cfg.max_agents || ctx->v_bump + fn.vars.size() > ctx->cfg.max_vars)
    return fail(ctx, INET_ERR_ARENA_FULL, "net does not fit the arena");
  if (ctx->st_nodes.empty() && ctx->st_vars.empty() && ctx->st_netctr.empty()) {
    ctx->st_a0 = ctx->a_bump;
    ctx->st_v0 = ctx->v_bump;
  }
  ctx->st_nodes.insert(ctx->st_nodes.end(), fn.nodes.begin(), fn.nodes.end());
  ctx->st_vars.insert(ctx->st_vars.end(), fn.vars.begin(), fn.vars.end());
  ctx->st_vown.insert(ctx->st_vown.end(), fn.vars.size(), slot);
  ctx->a_bump += fn.nodes.size();
  ctx->v_bump += fn.vars.size();
  ctx->live += (int64_t)fn.nodes.size();
  NetRec nr;
  nr.used = true;
  nr.iface = std::move(fn.iface);
  const unsigned long long ctr = (unsigned long long)fn.pairs.size() << kNetPairShift;
  nr.pairs = std::move(fn.pairs);
  commit_net(ctx, id, std::move(nr), ctr, (long long)fn.nodes.size());
  ctx->snap_valid = false;
  ctx->arena_gen++;
  *net_id_out = id;
  return INET_OK;
}

inet_status inet_load_nets(inet_ctx* ctx, const char* buf, const uint64_t* offsets, int32_t n, int32_t* ids_out,
                           int32_t* n_loaded_out) {
  if (!ctx || n < 0 || !n_loaded_out || (n > 0 && (!buf || !offsets || !ids_out))) return INET_ERR_INVALID_ARG;
  *n_loaded_out = 0;
  if (!ctx->have_rules) return fail(ctx, INET_ERR_STATE, "load rules first");
  if (ctx->poisoned) return fail(ctx, INET_ERR_STATE, "context needs inet_reset after a fatal error");
  for (int32_t i = 0; i < n; i++)
    if (offsets[i + 1] < offsets[i]) return INET_ERR_INVALID_ARG;
  inet_parsed pb;
  parse_batch(ctx->rules, ctx->rules_gen, buf, offsets, n, pb);
  return commit_batch(ctx, pb, 0, n, ids_out, n_loaded_out);
}

inet_status inet_parse_nets(const inet_ctx* ctx, const char* buf, const uint64_t* offsets, int32_t n,
                            inet_parsed** out) {
  if (!ctx || !out || n < 0 || (n > 0 && (!buf || !offsets))) return INET_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctx->have_rules) return INET_ERR_STATE;
  for (int32_t i = 0; i < n; i++)
    if (offsets[i + 1] < offsets[i]) return INET_ERR_INVALID_ARG;
  inet_parsed* pb = new inet_parsed();
  parse_batch(ctx->rules, ctx->rules_gen, buf, offsets, n, *pb);
  *out = pb;
  return INET_OK;
}

inet_status inet_parsed_info(const inet_parsed* p, int32_t* n_out, uint64_t* agents_out) {
  if (!p) return INET_ERR_INVALID_ARG;
  if (n_out) *n_out = (int32_t)p->fns.size();
  if (agents_out) {
    uint64_t a = 0;
    for (const FlatNet& fn : p->fns) a += fn.nodes.size();
    *agents_out = a;
  }
  return INET_OK;
}

inet_status inet_load_parsed(inet_ctx* ctx, inet_parsed* p, int32_t first, int32_t n, int32_t* ids_out,
                             int32_t* n_loaded_out) {
  if (!ctx || !p || !n_loaded_out || first < 0 || n < 0 || (n > 0 && !ids_out) ||
      (uint64_t)first + (uint64_t)n > p->fns.size())
    return INET_ERR_INVALID_ARG;
  *n_loaded_out = 0;
  if (!ctx->have_rules) return fail(ctx, INET_ERR_STATE, "load rules first");
  if (ctx->poisoned) return fail(ctx, INET_ERR_STATE, "context needs inet_reset after a fatal error");
  if (p->rules_gen != ctx->rules_gen) return fail(ctx, INET_ERR_STATE, "parsed under another rule set");
  for (int32_t i = first; i < first + n; i++)
    if (p->taken[(size_t)i]) return fail(ctx, INET_ERR_INVALID_ARG, "net of the parsed batch already loaded");
  return commit_batch(ctx, *p, first, n, ids_out, n_loaded_out);
}

void inet_parsed_free(inet_parsed* p) { delete p; }

inet_status inet_reduce(inet_ctx* ctx, const int32_t* net_ids, int32_t n, const inet_reduce_opts* opts,
                        inet_reduce_stats* stats) {
  if (!ctx || n < 0 || (n > 0 && !net_ids)) return INET_ERR_INVALID_ARG;
  if (ctx->host_only) return fail(ctx, INET_ERR_NO_DEVICE, "host-only context cannot reduce");
  if (ctx->poisoned) return fail(ctx, INET_ERR_STATE, "context needs inet_reset after a fatal error");
  if (!ctx->have_rules) return fail(ctx, INET_ERR_STATE, "load rules first");
  inet_reduce_opts o;
  memset(&o, 0, sizeof o);
  if (opts) o = *opts;
  const int B = o.block ? o.block : 256;
  if (o.mode < INET_MODE_PLAIN || o.mode > INET_MODE_PAPER) return fail(ctx, INET_ERR_INVALID_ARG, "bad mode");
  if (o.mode == INET_MODE_ASYNC) {
    if (B < 32 || B > 256 || B % 32) return fail(ctx, INET_ERR_INVALID_ARG, "ASYNC block must be a multiple of 32 in [32, 256]");
    if (o.max_steps) return fail(ctx, INET_ERR_INVALID_ARG, "ASYNC has no steps; bound a call with slice_us");
  } else if (B < 64 || B > 512 || B % 32) {
    return fail(ctx, INET_ERR_INVALID_ARG, "block must be a multiple of 32 in [64, 512]");
  }
  DeviceGuard g(ctx->device);
  inet_status s = stage_nets(ctx, net_ids, n);
  if (s) return s;
  const uint32_t cur = ctx->step & 1u;
  // per-call control fields
  struct {
    uint32_t step, done;
    int32_t error;
    uint32_t error_info, stop_step, hit_limit, trace_on, call_step0;
    int32_t fatal;
    uint32_t hit_slice;
    unsigned long long max_frontier;
    long long peak_live;
    unsigned long long slice_t0;
  } head;
  static_assert(sizeof(head) == offsetof(Ctrl, pad0), "control head layout");
  memset(&head, 0, sizeof head);
  head.step = ctx->step;
  head.stop_step = o.max_steps ? (uint32_t)std::min<uint64_t>(0xFFFFFFFEull, ctx->step + o.max_steps) : 0xFFFFFFFFu;
  head.trace_on = o.trace ? 1u : 0u;
  head.call_step0 = ctx->step;
  head.peak_live = ctx->live;
  const uint32_t fc[2] = {ctx->fcount[0], ctx->fcount[1]};
  CK(h2d(ctx, ctx->dev.ctrl, &head, sizeof head));
  CK(cudaMemsetAsync(ctx->dev.rule_hist, 0, sizeof(unsigned long long) * INET_MAX_RULES, ctx->stream));
  Dev d = ctx->dev;
  d.timeout_ns = o.timeout_ns ? o.timeout_ns : kDefaultTimeoutNs;
  // persistent kernel: frontiers of at most solo_max pairs run on block 0
  // with the frontier in shared memory (8 slots per pair, two buffers)
  d.solo_max = o.solo_max < 0 ? 0u : (o.solo_max == 0 ? (uint32_t)B : (uint32_t)o.solo_max);
  if (d.solo_max > kMaxSolo) return fail(ctx, INET_ERR_INVALID_ARG, "solo_max may not exceed 1024");
  const size_t smem = smem_bytes((uint32_t)B, d.n_labels, d.n_tmpl, 0);
  const size_t smem_p = smem_bytes((uint32_t)B, d.n_labels, d.n_tmpl, d.solo_max);
  if (smem_p > kMaxSmem) return fail(ctx, INET_ERR_INVALID_ARG, "block size and solo_max need too much shared memory");
  const LoopKernels K = loop_kernels(d.vown != nullptr);
  CK(raise_smem(kSmemStep + K.track, (const void*)K.step, smem));
  CK(raise_smem(kSmemPersistent + K.track, (const void*)K.persistent, smem_p));
  CK(cudaEventRecord(ctx->ev0, ctx->stream));
  uint64_t launches = 0;
  bool async_paused = false;
  if (fc[cur] > 0 && o.mode == INET_MODE_ASYNC) {
    const size_t smem_a = async_smem_bytes((uint32_t)B, d.n_labels, d.n_tmpl);
    // the kernel specialised for the rule set when it can be had
    const void* jf = jit_kernel(ctx, K.track);
    const void* afn = jf ? jf : (const void*)K.async;
    if (jf) CK(raise_smem_dyn(afn, smem_a));
    else CK(raise_smem(kSmemAsync + K.track, afn, smem_a));
    int per = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, afn, B, smem_a));
    const int maxg = std::max(1, per) * ctx->num_sms;
    // default: one block per SM (more warps mostly add idle polling)
    const int grid = o.grid > 0 ? std::min(o.grid, maxg) : maxg;
    if (o.slice_us > 0) d.slice_ns = (unsigned long long)o.slice_us * 1000ull;
    uint32_t q = cur;
    for (;;) {
      d.qcur = q;
      const uint32_t fill_blocks =
          (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((ctx->cfg.max_pairs + 255) / 256, 8ull * ctx->num_sms));
      k_async_fill<<<fill_blocks, 256, 0, ctx->stream>>>(d);
      k_async_prep<<<1, 1, 0, ctx->stream>>>(d);
      void* args[] = {&d};
      CK(cudaLaunchCooperativeKernel(afn, dim3((unsigned)grid), dim3((unsigned)B), args, smem_a, ctx->stream));
      if (jf) ctx->jit_launches++;
      k_async_post<<<1, 1, 0, ctx->stream>>>(d);
      CK(cudaGetLastError());
      launches += 4;
      CK(cudaEventRecord(ctx->ev1, ctx->stream));
      uint32_t st[10];  // step, done, error, error_info, stop_step, hit_limit, trace_on, call_step0, fatal, hit_slice
      CK(d2h(ctx, st, ctx->dev.ctrl, sizeof st));
      CK(cudaStreamSynchronize(ctx->stream));
      q ^= 1u;
      if (st[1]) break;
      if (o.slice_us > 0) {
        async_paused = true;
        break;
      }
    }
  } else if (fc[cur] > 0 && o.mode == INET_MODE_PAPER) {
    // the paper's loop (Sec. 3.6): an interaction phase whose name equations
    // are collected, then one communication pass (Sec. 3.5: sort by name,
    // fold adjacent pairs), until neither produced anything
    const uint64_t cap_eq64 = std::min<uint64_t>(2 * ctx->cfg.max_vars + 1024, 0x7FFFFF00ull);
    const uint32_t cap_eq = (uint32_t)cap_eq64;
    const uint32_t tiles_max = (cap_eq + kRsTile - 1) / kRsTile;
    // n result slots per active pair (Sec. 3.4): the most equations of any
    // right-hand side
    uint32_t nfix = 1;
    for (const Template& t : ctx->rules.tmpl) nfix = std::max<uint32_t>(nfix, t.n_link);
    const uint64_t cap_fix = (uint64_t)ctx->cfg.max_pairs * nfix;
    const uint32_t fix_tiles_max = (uint32_t)((cap_fix + kCpTile - 1) / kCpTile);
    CtlBufs bufs;
    unsigned long long *eq = nullptr, *v0 = nullptr, *v1 = nullptr, *fix = nullptr;
    uint32_t *k0 = nullptr, *k1 = nullptr, *counts = nullptr, *pc = nullptr, *fcounts = nullptr;
    if (!bufs.get(&eq, cap_eq) || !bufs.get(&v0, cap_eq) || !bufs.get(&v1, cap_eq) || !bufs.get(&k0, cap_eq) ||
        !bufs.get(&k1, cap_eq) || !bufs.get(&counts, (size_t)256 * tiles_max) || !bufs.get(&pc, 4) ||
        !bufs.get(&fix, (size_t)cap_fix) || !bufs.get(&fcounts, fix_tiles_max))
      return fail(ctx, INET_ERR_CUDA, "no device memory for the equation arrays of the paper's form");
    Dev dp = d;
    dp.paper = 1;
    dp.eq = eq;
    dp.eq_n = pc;
    dp.cap_eq = cap_eq;
    dp.eq_fix = fix;
    dp.eq_fix_n = nfix;
    dp.cap_fix = cap_fix;
    CK(cudaMemsetAsync(pc, 0, 4 * sizeof(uint32_t), ctx->stream));
    CK(cudaEventRecord(ctx->ev0, ctx->stream));  // the arrays are set up outside the measured time
    const uint64_t nv = ctx->v_bump;
    if (nv) k_paper_collect<<<(unsigned)((nv + 255) / 256), 256, 0, ctx->stream>>>(dp, nv);
    int bits = 1;
    while (bits < 32 && (ctx->cfg.max_vars >> bits)) bits++;
    uint32_t pending = fc[cur];
    for (;;) {
      if (pending) {
        k_paper_prep<<<1, 1, 0, ctx->stream>>>(dp);
        const uint32_t grid = std::max<uint32_t>(1, (pending + (uint32_t)B - 1) / (uint32_t)B);
        K.step<<<grid, B, smem, ctx->stream>>>(dp);
        // the dummies out, the equations after those already in the array
        const uint64_t mf = (uint64_t)pending * nfix;
        const uint32_t ft = (uint32_t)((mf + kCpTile - 1) / kCpTile);
        k_paper_compact_count<<<ft, kCpThreads, 0, ctx->stream>>>(fix, mf, fcounts);
        k_rs_scan<<<1, 1024, 0, ctx->stream>>>(fcounts, ft);
        k_paper_compact_scatter<<<ft, kCpThreads, 0, ctx->stream>>>(dp, fix, mf, fcounts, pc + 2);
        k_paper_compact_done<<<1, 1, 0, ctx->stream>>>(dp, pc + 2);
        launches += 6;
      }
      CK(cudaMemsetAsync(pc + 1, 0, sizeof(uint32_t), ctx->stream));
      uint32_t m = 0;
      CK(d2h(ctx, &m, pc, 4));
      CK(cudaStreamSynchronize(ctx->stream));
      if (m > cap_eq) return fail(ctx, INET_ERR_ARENA_FULL, "equation array of the paper's form is full");
      if (m) {
        const uint32_t t = (m + kRsTile - 1) / kRsTile;
        k_paper_orient<<<(m + 255) / 256, 256, 0, ctx->stream>>>(dp, m, k0, v0);
        uint32_t *ks = k0, *kd = k1;
        unsigned long long *vs = v0, *vd = v1;
        for (int shift = 0; shift < bits; shift += 8) {
          k_rs_upsweep<<<t, kRsThreads, 0, ctx->stream>>>(ks, m, shift, counts);
          k_rs_scan<<<1, 1024, 0, ctx->stream>>>(counts, 256 * t);
          k_rs_downsweep<<<t, kRsThreads, 0, ctx->stream>>>(ks, vs, m, shift, counts, kd, vd);
          std::swap(ks, kd);
          std::swap(vs, vd);
          launches += 3;
        }
        CK(cudaMemsetAsync(pc, 0, sizeof(uint32_t), ctx->stream));  // results compact from 0
        k_paper_merge<<<(m + 255) / 256, 256, 0, ctx->stream>>>(dp, ks, vs, m, pc + 1);
        launches += 2;
      }
      uint32_t hp[2] = {0, 0}, hs[2] = {0, 0}, fcn[2] = {0, 0};
      int32_t fat = 0;
      CK(d2h(ctx, hp, pc, 8));
      CK(d2h(ctx, hs, &ctx->dev.ctrl->step, 4));
      CK(d2h(ctx, fcn, ctx->dev.ctrl->fcount, 8));
      CK(d2h(ctx, &fat, &ctx->dev.ctrl->fatal, 4));
      CK(cudaStreamSynchronize(ctx->stream));
      pending = std::min<uint32_t>(fcn[hs[0] & 1u], (uint32_t)ctx->cfg.max_pairs);
      if (fat) break;
      if (pending == 0 && hp[1] == 0) break;  // no interaction and no communication: done
    }
    // what is left binds its names, as ->com's first arrivals would
    uint32_t left = 0;
    CK(d2h(ctx, &left, pc, 4));
    CK(cudaStreamSynchronize(ctx->stream));
    left = std::min(left, cap_eq);
    if (left) k_paper_deposit<<<(left + 255) / 256, 256, 0, ctx->stream>>>(dp, left);
    CK(cudaGetLastError());
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else if (fc[cur] > 0) {
    if (o.mode == INET_MODE_PLAIN) {
      // one launch and one 16-byte read of the frontier size per step
      uint32_t pending = fc[cur];
      for (;;) {
        const uint32_t grid = std::max<uint32_t>(1, (pending + (uint32_t)B - 1) / (uint32_t)B);
        K.step<<<grid, B, smem, ctx->stream>>>(d);
        CK(cudaGetLastError());
        launches++;
        CK(cudaEventRecord(ctx->ev1, ctx->stream));
        uint32_t st[4];  // step, done, error, error_info
        uint32_t fcn[2];
        CK(d2h(ctx, st, ctx->dev.ctrl, sizeof st));
        CK(d2h(ctx, fcn, ctx->dev.ctrl->fcount, sizeof fcn));
        CK(cudaStreamSynchronize(ctx->stream));
        if (st[1]) break;
        pending = fcn[st[0] & 1u];
        if (pending == 0) break;
      }
    } else {
      // GRAPH and PERSISTENT run many steps per launch; a launch also ends
      // when its time slice is over (hit_slice), and is then relaunched.
      int grid = o.grid;
      if (o.mode == INET_MODE_GRAPH) {
        if (grid <= 0) {
          int per = 0;
          CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K.step, B, smem));
          grid = std::max(1, per) * ctx->num_sms;
        }
        s = build_graph(ctx, B, grid, smem);
        if (s) return s;
      } else {
        int per = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K.persistent, B, smem_p));
        const int maxg = std::max(1, per) * ctx->num_sms;
        grid = grid > 0 ? std::min(grid, maxg) : maxg;
        // the step word the blocks start from
        const unsigned long long word = pack_word(fc[cur], 0, cur, 0);
        static const uint32_t zero4 = 0;
        CK(h2d(ctx, &ctx->dev.ctrl->bar_word, &word, 8));
        CK(h2d(ctx, &ctx->dev.ctrl->bar_count, &zero4, 4));
      }
      for (;;) {
        if (o.mode == INET_MODE_GRAPH) {
          CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
        } else {
          void* args[] = {&d};
          CK(cudaLaunchCooperativeKernel((const void*)K.persistent, dim3((unsigned)grid), dim3((unsigned)B), args,
                                         smem_p, ctx->stream));
        }
        launches++;
        CK(cudaEventRecord(ctx->ev1, ctx->stream));
        uint32_t hit = 0;
        CK(d2h(ctx, &hit, &ctx->dev.ctrl->hit_slice, 4));
        CK(cudaStreamSynchronize(ctx->stream));
        if (!hit) break;
        static const unsigned long long zero8 = 0;
        CK(h2d(ctx, &ctx->dev.ctrl->done, &zero8, 4));
        CK(h2d(ctx, &ctx->dev.ctrl->hit_slice, &zero8, 4));
        CK(h2d(ctx, &ctx->dev.ctrl->slice_t0, &zero8, 8));
        if (o.mode == INET_MODE_PERSISTENT) {
          uint32_t stp = 0, fcn[2] = {0, 0};
          CK(d2h(ctx, &stp, &ctx->dev.ctrl->step, 4));
          CK(d2h(ctx, fcn, ctx->dev.ctrl->fcount, 8));
          CK(cudaStreamSynchronize(ctx->stream));
          const unsigned long long word = pack_word(fcn[stp & 1u], 0, stp & 1u, 0);
          CK(h2d(ctx, &ctx->dev.ctrl->bar_word, &word, 8));
          CK(h2d(ctx, &ctx->dev.ctrl->bar_count, &zero8, 4));
        }
      }
    }
  }
  if (!launches) CK(cudaEventRecord(ctx->ev1, ctx->stream));
  // quotas (inet_set_quotas): a net holding more live agents than its quota
  // stops here with INET_ERR_ARENA_FULL, its pairs leave the frontier, and
  // the other nets go on as if it had never run
  if (ctx->quotas_set && d.netquota) {
    uint8_t* mark = at<uint8_t>(ctx, ctx->lay.netmark);
    unsigned long long* hit = at<unsigned long long>(ctx, ctx->lay.free_st) + 3;
    const uint32_t nn = (uint32_t)ctx->nets.size();
    CK(cudaMemsetAsync(hit, 0, sizeof *hit, ctx->stream));
    k_quota_check<<<(unsigned)std::max<uint32_t>(1, std::min<uint32_t>((nn + 255) / 256, 1024)), 256, 0, ctx->stream>>>(
        d, nn, mark, hit);
    k_quota_purge<<<1, 1024, 0, ctx->stream>>>(d, mark, nn, hit);
    CK(cudaGetLastError());
  }
  // results
  Ctrl hc;
  CK(d2h(ctx, &hc, ctx->dev.ctrl, sizeof(Ctrl)));
  std::vector<unsigned long long> hist(INET_MAX_RULES);
  CK(d2h(ctx, hist.data(), ctx->dev.rule_hist, sizeof(unsigned long long) * INET_MAX_RULES));
  const size_t nn = ctx->nets.size();
  ctx->h_net_valid = nn == 0;  // per-net counters are copied when asked for
  CK(cudaStreamSynchronize(ctx->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  const uint32_t steps = hc.step - ctx->step;
  ctx->tr_front.clear();
  ctx->tr_live.clear();
  if (o.trace && steps) {
    const uint32_t k = std::min(steps, kTraceCap);
    ctx->tr_front.resize(k);
    ctx->tr_live.resize(k);
    CK(d2h(ctx, ctx->tr_front.data(), ctx->dev.trace_front, k * sizeof(long long)));
    CK(d2h(ctx, ctx->tr_live.data(), ctx->dev.trace_live, k * sizeof(long long)));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  ctx->step = hc.step;
  ctx->fcount[0] = hc.fcount[0];
  ctx->fcount[1] = hc.fcount[1];
  ctx->a_bump = hc.a_bump;
  ctx->v_bump = hc.v_bump;
  ctx->live = hc.live;
  ctx->st_a0 = ctx->a_bump;
  ctx->st_v0 = ctx->v_bump;
  ctx->snap_valid = false;
  ctx->arena_gen++;
  if (stats) {
    memset(stats, 0, sizeof *stats);
    uint64_t tot = 0;
    for (size_t r = 0; r < ctx->rules.tmpl.size(); r++) {
      stats->per_rule[r] = hist[r];
      tot += hist[r];
    }
    stats->interactions = tot;
    stats->steps = steps;
    stats->max_frontier = hc.max_frontier;
    stats->live_agents = hc.live;
    stats->peak_live_agents = std::max<long long>(hc.peak_live, hc.live);
    stats->pending_pairs = hc.fcount[hc.step & 1u];
    stats->device_ms = ms;
    stats->n_rules = (uint32_t)ctx->rules.tmpl.size();
    // the graph body launches the step kernel once per step
    if (o.mode == INET_MODE_GRAPH) launches = steps + launches;
    stats->launches = (uint32_t)std::min<uint64_t>(launches, 0xFFFFFFFFull);
  }
  if (hc.fatal) {
    ctx->poisoned = true;
    const char* what = hc.fatal == INET_ERR_ARENA_FULL ? "arena, frontier or name capacity exhausted"
                     : hc.fatal == INET_ERR_TIMEOUT    ? "a device-side wait timed out"
                                                       : "inconsistent device state";
    return fail(ctx, hc.fatal, std::string(what) + " (context needs inet_reset)");
  }
  if (hc.error == INET_ERR_NO_RULE)
    return fail(ctx, INET_ERR_NO_RULE, "active pair without a rule in net " + std::to_string(hc.error_info));
  if (hc.hit_limit || async_paused)
    return fail(ctx, INET_ERR_STEP_LIMIT, "step limit reached; call inet_reduce again to continue");
  return INET_OK;
}

inet_status inet_stage(inet_ctx* ctx, const int32_t* net_ids, int32_t n) {
  if (!ctx || n < 0 || (n > 0 && !net_ids)) return INET_ERR_INVALID_ARG;
  if (ctx->host_only) return fail(ctx, INET_ERR_NO_DEVICE, "host-only context");
  if (ctx->poisoned) return fail(ctx, INET_ERR_STATE, "context needs inet_reset after a fatal error");
  DeviceGuard g(ctx->device);
  return stage_nets(ctx, net_ids, n);
}

inet_status inet_transfer_bytes(const inet_ctx* ctx, uint64_t* h2d_out, uint64_t* d2h_out) {
  if (!ctx) return INET_ERR_INVALID_ARG;
  if (h2d_out) *h2d_out = ctx->h2d_bytes;
  if (d2h_out) *d2h_out = ctx->d2h_bytes;
  return INET_OK;
}

inet_status inet_readback(inet_ctx* ctx, int32_t net_id, char* buf, size_t cap, size_t* needed_out) {
  if (!ctx) return INET_ERR_INVALID_ARG;
  inet_status s = check_net(ctx, net_id);
  if (s) return s;
  if (ctx->host_only) return fail(ctx, INET_ERR_NO_DEVICE, "host-only context");
  DeviceGuard g(ctx->device);
  if ((s = ensure_workspace(ctx)) || (s = upload_staged(ctx))) return s;
  // rendered on the device; a net that is not a forest of terms (a
  // subterm reached twice, a cycle) is rendered on the host, whose walk
  // bounds it
  if (ctx->dtext_net != net_id || ctx->dtext_gen != ctx->arena_gen) {
    bool ok = false;
    if ((s = read_text_device(ctx, net_id, ctx->dtext, &ok, &ctx->dtext_reached, &ctx->dtext_live))) return s;
    if (ok) ctx->renders_device++;
    else ctx->renders_host++;
    if (!ok) {
      if ((s = ensure_snapshot(ctx))) return s;
      Readback rb;
      read_net_text(ctx->snap_nodes.data(), ctx->snap_nodes.size(), ctx->snap_vars.data(), ctx->snap_vars.size(),
                    ctx->nets[(size_t)net_id].iface, ctx->rules, rb);
      ctx->dtext = std::move(rb.text);
      ctx->dtext_reached = (uint64_t)rb.reached;
      ctx->dtext_live = (size_t)net_id < ctx->snap_live.size() ? ctx->snap_live[(size_t)net_id] : 0;
    }
    ctx->dtext_net = net_id;
    ctx->dtext_gen = ctx->arena_gen;
  }
  const std::string& text = ctx->dtext;
  if (needed_out) *needed_out = text.size() + 1;
  if (!buf || cap < text.size() + 1) return fail(ctx, INET_ERR_INVALID_ARG, "buffer too small");
  memcpy(buf, text.c_str(), text.size() + 1);
  return INET_OK;
}

inet_status inet_readback_counts(const inet_ctx* ctx, uint64_t* device_out, uint64_t* host_out) {
  if (!ctx) return INET_ERR_INVALID_ARG;
  if (device_out) *device_out = ctx->renders_device;
  if (host_out) *host_out = ctx->renders_host;
  return INET_OK;
}

inet_status inet_readback_nat(inet_ctx* ctx, int32_t net_id, uint64_t* value_out, uint64_t* interactions_out) {
  if (!ctx || !value_out) return INET_ERR_INVALID_ARG;
  inet_status s = check_net(ctx, net_id);
  if (s) return s;
  if (ctx->host_only) return fail(ctx, INET_ERR_NO_DEVICE, "host-only context");
  DeviceGuard g(ctx->device);
  if ((s = ensure_workspace(ctx)) || (s = upload_staged(ctx)) || (s = ensure_snapshot(ctx)) ||
      (s = ensure_net_counters(ctx)))
    return s;
  Readback rb;
  read_net(ctx->snap_nodes.data(), ctx->snap_nodes.size(), ctx->snap_vars.data(), ctx->snap_vars.size(),
           ctx->nets[(size_t)net_id].iface, ctx->rules, 0, false, rb);
  if (interactions_out) *interactions_out = ctx->h_netctr[(size_t)net_id] & kNetIntMask;
  if (rb.nat < 0) return fail(ctx, INET_ERR_INVALID_ARG, "interface is not a numeral S^k(Z)");
  *value_out = (uint64_t)rb.nat;
  return INET_OK;
}

inet_status inet_net_pending(inet_ctx* ctx, const int32_t* net_ids, int32_t n, uint64_t* pending_out) {
  if (!ctx || n < 0 || (n > 0 && (!net_ids || !pending_out))) return INET_ERR_INVALID_ARG;
  if (!ctx->host_only) {
    DeviceGuard g(ctx->device);
    const inet_status s = ensure_net_counters(ctx);
    if (s) return s;
  }
  for (int32_t i = 0; i < n; i++) {
    const int32_t id = net_ids[i];
    if (id < 0 || (size_t)id >= ctx->nets.size() || !ctx->nets[(size_t)id].used) return INET_ERR_INVALID_ARG;
    const NetRec& nr = ctx->nets[(size_t)id];
    pending_out[i] = nr.started ? (ctx->h_netctr[(size_t)id] >> kNetPairShift) : nr.pairs.size();
  }
  return INET_OK;
}

inet_status inet_readback_nats(inet_ctx* ctx, const int32_t* net_ids, int32_t n, uint64_t* values_out,
                               uint64_t* interactions_out) {
  if (!ctx || n < 0 || (n > 0 && (!net_ids || !values_out))) return INET_ERR_INVALID_ARG;
  if (ctx->host_only) return fail(ctx, INET_ERR_NO_DEVICE, "host-only context");
  if (ctx->rb_n >= 0) return fail(ctx, INET_ERR_STATE, "a non-blocking readback is in flight");
  if (n == 0) return INET_OK;
  DeviceGuard g(ctx->device);
  inet_status s = ensure_workspace(ctx);
  if (s) return s;
  if ((s = upload_staged(ctx)) || (s = ensure_net_counters(ctx))) return s;
  std::vector<uint32_t> roots((size_t)n);
  for (int32_t i = 0; i < n; i++) {
    if ((s = check_net(ctx, net_ids[i]))) return s;
    const NetRec& nr = ctx->nets[(size_t)net_ids[i]];
    roots[(size_t)i] = nr.iface.size() == 1 ? nr.iface[0] : kEmpty;
    if (interactions_out) interactions_out[i] = ctx->h_netctr[(size_t)net_ids[i]] & kNetIntMask;
  }
  auto si = ctx->rules.index.find("S");
  auto zi = ctx->rules.index.find("Z");
  if (si == ctx->rules.index.end() || zi == ctx->rules.index.end()) {
    for (int32_t i = 0; i < n; i++) values_out[i] = ~0ull;
    return INET_OK;
  }
  // roots in, values out, kReadChunk nets at a time
  for (int32_t off = 0; off < n; off += (int32_t)kReadChunk) {
    const int32_t m = std::min<int32_t>(n - off, (int32_t)kReadChunk);
    uint32_t* droot = at<uint32_t>(ctx, ctx->lay.rb_root);
    unsigned long long* dval = at<unsigned long long>(ctx, ctx->lay.rb_val);
    CK(h2d(ctx, droot, roots.data() + off, sizeof(uint32_t) * (size_t)m));
    if ((s = read_nats_device(ctx, ctx->stream, droot, (uint32_t)m, si->second, zi->second, dval))) return s;
    CK(d2h(ctx, values_out + off, dval, sizeof(unsigned long long) * (size_t)m));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return INET_OK;
}

inet_status inet_readback_nats_begin(inet_ctx* ctx, const int32_t* net_ids, int32_t n) {
  if (!ctx || n < 0 || (uint32_t)n > kReadChunk || (n > 0 && !net_ids)) return INET_ERR_INVALID_ARG;
  if (ctx->host_only) return fail(ctx, INET_ERR_NO_DEVICE, "host-only context");
  if (ctx->poisoned) return fail(ctx, INET_ERR_STATE, "context needs inet_reset after a fatal error");
  if (ctx->rb_n >= 0) return fail(ctx, INET_ERR_STATE, "a non-blocking readback is already in flight");
  DeviceGuard g(ctx->device);
  inet_status s = ensure_workspace(ctx);
  if (s) return s;
  if ((s = upload_staged(ctx)) || (s = ensure_net_counters(ctx))) return s;
  if (!ctx->rb_stream) {
    CK(cudaStreamCreateWithFlags(&ctx->rb_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->rb_ready, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->rb_after, cudaEventDisableTiming));
    CK(cudaHostAlloc(reinterpret_cast<void**>(&ctx->rb_host_roots), sizeof(uint32_t) * kReadChunk, 0));
    CK(cudaHostAlloc(reinterpret_cast<void**>(&ctx->rb_host_vals), sizeof(unsigned long long) * kReadChunk, 0));
  }
  ctx->rb_inter.assign((size_t)n, 0);
  ctx->rb_ids.assign(net_ids, net_ids + n);
  for (int32_t i = 0; i < n; i++) {
    if ((s = check_net(ctx, net_ids[i]))) return s;
    const NetRec& nr = ctx->nets[(size_t)net_ids[i]];
    ctx->rb_host_roots[i] = nr.iface.size() == 1 ? nr.iface[0] : kEmpty;
    ctx->rb_inter[(size_t)i] = ctx->h_netctr[(size_t)net_ids[i]] & kNetIntMask;
  }
  auto si = ctx->rules.index.find("S");
  auto zi = ctx->rules.index.find("Z");
  if (si == ctx->rules.index.end() || zi == ctx->rules.index.end()) {
    for (int32_t i = 0; i < n; i++) ctx->rb_host_vals[i] = ~0ull;
    CK(cudaEventRecord(ctx->rb_ready, ctx->rb_stream));
  } else if (n > 0) {
    // after everything queued on the main stream so far (the reduction that
    // finished these nets); later reductions of other nets run alongside
    uint32_t* droot = at<uint32_t>(ctx, ctx->lay.rb_root);
    unsigned long long* dval = at<unsigned long long>(ctx, ctx->lay.rb_val);
    CK(cudaEventRecord(ctx->rb_after, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->rb_stream, ctx->rb_after, 0));
    CK(cudaMemcpyAsync(droot, ctx->rb_host_roots, sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice,
                       ctx->rb_stream));
    if ((s = read_nats_device(ctx, ctx->rb_stream, droot, (uint32_t)n, si->second, zi->second, dval))) return s;
    CK(cudaMemcpyAsync(ctx->rb_host_vals, dval, sizeof(unsigned long long) * (size_t)n, cudaMemcpyDeviceToHost,
                       ctx->rb_stream));
    CK(cudaEventRecord(ctx->rb_ready, ctx->rb_stream));
    ctx->h2d_bytes += sizeof(uint32_t) * (size_t)n;
    ctx->d2h_bytes += sizeof(unsigned long long) * (size_t)n;
  } else {
    CK(cudaEventRecord(ctx->rb_ready, ctx->rb_stream));
  }
  ctx->rb_n = n;
  return INET_OK;
}

inet_status inet_readback_nats_end(inet_ctx* ctx, int32_t wait, uint64_t* values_out, uint64_t* interactions_out,
                                   int32_t cap, int32_t* n_out) {
  if (!ctx || !n_out || cap < 0 || (cap > 0 && !values_out)) return INET_ERR_INVALID_ARG;
  *n_out = -1;
  if (ctx->rb_n < 0) return fail(ctx, INET_ERR_STATE, "no non-blocking readback in flight");
  if (cap < ctx->rb_n) return fail(ctx, INET_ERR_INVALID_ARG, "output arrays shorter than the batch");
  DeviceGuard g(ctx->device);
  if (wait) {
    CK(cudaEventSynchronize(ctx->rb_ready));
  } else {
    const cudaError_t e = cudaEventQuery(ctx->rb_ready);
    if (e == cudaErrorNotReady) return INET_OK;
    CK(e);
  }
  for (int32_t i = 0; i < ctx->rb_n; i++) {
    values_out[i] = ctx->rb_host_vals[i];
    if (interactions_out) interactions_out[i] = ctx->rb_inter[(size_t)i];
  }
  *n_out = ctx->rb_n;
  ctx->rb_n = -1;
  ctx->rb_ids.clear();
  return INET_OK;
}

inet_status inet_net_finished(inet_ctx* ctx, int32_t* ids_out, int32_t cap, int32_t* n_out) {
  if (!ctx || !n_out || cap < 0 || (cap > 0 && !ids_out)) return INET_ERR_INVALID_ARG;
  *n_out = 0;
  if (ctx->host_only) return fail(ctx, INET_ERR_NO_DEVICE, "host-only context");
  DeviceGuard g(ctx->device);
  inet_status s = ensure_workspace(ctx);
  if (s) return s;
  if ((s = upload_staged(ctx))) return s;
  const uint32_t nn = (uint32_t)ctx->nets.size();
  if (nn == 0 || cap == 0) return INET_OK;
  const uint32_t c = (uint32_t)std::min<int32_t>(cap, (int32_t)kReadChunk);
  int32_t* dids = at<int32_t>(ctx, ctx->lay.fin_ids);
  uint32_t* dcnt = at<uint32_t>(ctx, ctx->lay.fin_cnt);
  static thread_local uint32_t cnt;
  CK(cudaMemsetAsync(dcnt, 0, 4, ctx->stream));
  k_net_finished<<<(nn + 255) / 256, 256, 0, ctx->stream>>>(ctx->dev, nn, dids, c, dcnt);
  CK(cudaGetLastError());
  CK(d2h(ctx, &cnt, dcnt, 4));
  CK(cudaStreamSynchronize(ctx->stream));
  const uint32_t k = std::min(cnt, c);
  if (k) {
    CK(d2h(ctx, ids_out, dids, sizeof(int32_t) * k));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  *n_out = (int32_t)k;
  return INET_OK;
}

inet_status inet_free_nets(inet_ctx* ctx, const int32_t* net_ids, int32_t n) {
  if (!ctx || n < 0 || (uint32_t)n > kReadChunk || (n > 0 && !net_ids)) return INET_ERR_INVALID_ARG;
  if (ctx->host_only) return fail(ctx, INET_ERR_NO_DEVICE, "host-only context");
  if (ctx->poisoned) return fail(ctx, INET_ERR_STATE, "context needs inet_reset after a fatal error");
  if (!(ctx->cfg.flags & INET_ARENA_FREE_NETS))
    return fail(ctx, INET_ERR_STATE, "the context keeps no name owners: create it with INET_ARENA_FREE_NETS");
  if (n == 0) return INET_OK;
  std::vector<uint8_t> listed(ctx->nets.size(), 0);
  for (int32_t i = 0; i < n; i++) {
    inet_status s = check_net(ctx, net_ids[i]);
    if (s) return s;
    if (listed[(size_t)net_ids[i]]) return fail(ctx, INET_ERR_INVALID_ARG, "net listed twice");
    listed[(size_t)net_ids[i]] = 1;
    if (!ctx->nets[(size_t)net_ids[i]].started)
      return fail(ctx, INET_ERR_STATE, "net " + std::to_string(net_ids[i]) + " was never staged or reduced");
  }
  if (ctx->rb_n >= 0)
    for (int32_t id : ctx->rb_ids)
      if (listed[(size_t)id]) return fail(ctx, INET_ERR_STATE, "a readback of this net is in flight");
  DeviceGuard g(ctx->device);
  inet_status s = ensure_workspace(ctx);
  if (s) return s;
  // every record below the host's bump pointer must be on the device
  if ((s = upload_staged(ctx))) return s;
  int32_t* dids = at<int32_t>(ctx, ctx->lay.free_ids);
  unsigned long long* dst = at<unsigned long long>(ctx, ctx->lay.free_st);
  uint8_t* mark = at<uint8_t>(ctx, ctx->lay.netmark);
  CK(h2d(ctx, dids, net_ids, sizeof(int32_t) * (size_t)n));
  k_free_check<<<1, 1024, 0, ctx->stream>>>(ctx->dev, dids, (uint32_t)n, mark, dst);
  const uint64_t span = std::max(ctx->a_bump, ctx->v_bump);
  const unsigned grid = (unsigned)std::max<uint64_t>(
      1, std::min<uint64_t>((span + 255) / 256, 8ull * (uint64_t)std::max(ctx->num_sms, 1)));
  k_free_scan<<<grid, 256, 0, ctx->stream>>>(ctx->dev, (uint32_t)ctx->a_bump, (uint32_t)ctx->v_bump, mark, dst);
  k_free_unmark<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->dev, dids, (uint32_t)n, mark, dst);
  CK(cudaGetLastError());
  static thread_local unsigned long long hs[3];
  CK(d2h(ctx, hs, dst, sizeof hs));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hs[0]) return fail(ctx, INET_ERR_STATE, "a listed net still has active pairs; nothing was freed");
  for (int32_t i = 0; i < n; i++) {
    const size_t id = (size_t)net_ids[i];
    ctx->nets[id] = NetRec();
    ctx->h_netctr[id] = 0;
    ctx->h_netstat[id] = 0;
    ctx->free_net_ids.push_back(net_ids[i]);
  }
  ctx->live -= (int64_t)hs[1];
  ctx->snap_valid = false;
  ctx->arena_gen++;
  ctx->text_net = -1;
  return INET_OK;
}

inet_status inet_free_net(inet_ctx* ctx, int32_t net_id) { return inet_free_nets(ctx, &net_id, 1); }

inet_status inet_set_quotas(inet_ctx* ctx, const int32_t* net_ids, const uint64_t* quotas, int32_t n) {
  if (!ctx || n < 0 || (uint32_t)n > kReadChunk || (n > 0 && (!net_ids || !quotas))) return INET_ERR_INVALID_ARG;
  if (ctx->host_only) return fail(ctx, INET_ERR_NO_DEVICE, "host-only context");
  if (!(ctx->cfg.flags & INET_ARENA_FREE_NETS))
    return fail(ctx, INET_ERR_STATE, "quotas need the live agents of each net: create the context with INET_ARENA_FREE_NETS");
  for (int32_t i = 0; i < n; i++) {
    inet_status s = check_net(ctx, net_ids[i]);
    if (s) return s;
  }
  if (n == 0) return INET_OK;
  DeviceGuard g(ctx->device);
  inet_status s = ensure_workspace(ctx);
  if (s) return s;
  if ((s = upload_staged(ctx))) return s;  // a net's quota slot is reset when it is uploaded
  int32_t* dids = at<int32_t>(ctx, ctx->lay.stn_ids);
  unsigned long long* dq = at<unsigned long long>(ctx, ctx->lay.stn_ctr);
  CK(h2d(ctx, dids, net_ids, sizeof(int32_t) * (size_t)n));
  CK(h2d(ctx, dq, quotas, sizeof(uint64_t) * (size_t)n));
  k_net_set_quota<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->dev, dids, dq, (uint32_t)n);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  for (int32_t i = 0; i < n; i++) ctx->quotas_set = ctx->quotas_set || quotas[i] != 0;
  return INET_OK;
}

inet_status inet_net_status(inet_ctx* ctx, const int32_t* net_ids, int32_t n, int32_t* status_out) {
  if (!ctx || n < 0 || (n > 0 && (!net_ids || !status_out))) return INET_ERR_INVALID_ARG;
  if (!ctx->host_only) {
    DeviceGuard g(ctx->device);
    const inet_status s = ensure_net_counters(ctx);
    if (s) return s;
  }
  for (int32_t i = 0; i < n; i++) {
    const int32_t id = net_ids[i];
    if (id < 0 || (size_t)id >= ctx->nets.size() || !ctx->nets[(size_t)id].used) return INET_ERR_INVALID_ARG;
    status_out[i] = ctx->h_netstat[(size_t)id];
  }
  return INET_OK;
}

inet_status inet_arena_usage(inet_ctx* ctx, inet_arena_usage_t* out) {
  if (!ctx || !out) return INET_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  if (!ctx->host_only && ctx->ws_ready) {
    DeviceGuard g(ctx->device);
    inet_status s = upload_staged(ctx);
    if (s) return s;
    static thread_local unsigned long long hr[6];  // a_head, a_tail, a_pub, v_head, v_tail, v_pub
    CK(d2h(ctx, &hr[0], &ctx->dev.ctrl->a_head, 8));
    CK(d2h(ctx, &hr[1], &ctx->dev.ctrl->a_tail, 8));
    CK(d2h(ctx, &hr[2], &ctx->dev.ctrl->a_pub, 8));
    CK(d2h(ctx, &hr[3], &ctx->dev.ctrl->v_head, 8));
    CK(d2h(ctx, &hr[4], &ctx->dev.ctrl->v_tail, 8));
    CK(d2h(ctx, &hr[5], &ctx->dev.ctrl->v_pub, 8));
    CK(cudaStreamSynchronize(ctx->stream));
    // a pop that found the ring empty advanced the head past the published end
    out->free_agent_slots = hr[1] - std::min(hr[0], hr[2]);
    out->free_name_slots = hr[4] - std::min(hr[3], hr[5]);
  }
  out->agent_slots = ctx->a_bump;
  out->name_slots = ctx->v_bump;
  out->live_agents = ctx->live;
  out->nets = (uint32_t)(ctx->nets.size() - ctx->free_net_ids.size());
  out->free_net_ids = (uint32_t)ctx->free_net_ids.size();
  return INET_OK;
}

inet_status inet_net_info(inet_ctx* ctx, int32_t net_id, inet_net_stats* out) {
  if (!ctx || !out) return INET_ERR_INVALID_ARG;
  inet_status s = check_net(ctx, net_id);
  if (s) return s;
  memset(out, 0, sizeof *out);
  const NetRec& nr = ctx->nets[(size_t)net_id];
  if (ctx->host_only) {
    out->pending_pairs = nr.pairs.size();
    return INET_OK;
  }
  DeviceGuard g(ctx->device);
  if ((s = ensure_workspace(ctx)) || (s = upload_staged(ctx)) || (s = ensure_net_counters(ctx))) return s;
  const unsigned long long v = ctx->h_netctr[(size_t)net_id];
  out->status = ctx->h_netstat[(size_t)net_id];
  out->interactions = v & kNetIntMask;
  out->pending_pairs = v >> kNetPairShift;
  out->reduced = nr.started && out->pending_pairs == 0 ? 1 : 0;
  if (ctx->dtext_net == net_id && ctx->dtext_gen == ctx->arena_gen && ctx->dtext_live >= 0) {
    // the text rendered from the current arena counted both on the device
    out->live_agents = ctx->dtext_live;
    out->residual_agents = ctx->dtext_live - (int64_t)ctx->dtext_reached;
    return INET_OK;
  }
  if ((s = ensure_snapshot(ctx))) return s;
  uint64_t reached = ctx->text_reached;
  if (ctx->text_net != net_id || ctx->text_gen != ctx->snap_gen) {  // no text walk of this snapshot to reuse
    Readback rb;
    read_net(ctx->snap_nodes.data(), ctx->snap_nodes.size(), ctx->snap_vars.data(), ctx->snap_vars.size(), nr.iface,
             ctx->rules, 0, false, rb);
    reached = rb.reached;
  }
  out->live_agents = (size_t)net_id < ctx->snap_live.size() ? ctx->snap_live[(size_t)net_id] : 0;
  out->residual_agents = out->live_agents - reached;
  return INET_OK;
}

inet_status inet_trace(inet_ctx* ctx, int64_t* frontier, int64_t* live, size_t cap, size_t* n_out) {
  if (!ctx) return INET_ERR_INVALID_ARG;
  const size_t k = ctx->tr_front.size();
  if (n_out) *n_out = k;
  for (size_t i = 0; i < std::min(k, cap); i++) {
    if (frontier) frontier[i] = ctx->tr_front[i];
    if (live) live[i] = ctx->tr_live[i];
  }
  return INET_OK;
}

inet_status inet_reset(inet_ctx* ctx) {
  if (!ctx) return INET_ERR_INVALID_ARG;
  if (ctx->rb_n >= 0) {
    // a readback still walks this arena: let it end, drop its results
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->rb_stream);
    ctx->rb_n = -1;
  }
  ctx->nets.clear();
  ctx->h_netctr.clear();
  ctx->h_netstat.clear();
  ctx->st_nodes.clear();
  ctx->st_vars.clear();
  ctx->st_netctr.clear();
  ctx->st_vown.clear();
  ctx->st_net_ids.clear();
  ctx->st_netlive.clear();
  ctx->quotas_set = false;
  ctx->free_net_ids.clear();
  ctx->rb_ids.clear();
  ctx->a_bump = ctx->v_bump = 0;
  ctx->st_a0 = ctx->st_v0 = 0;
  ctx->live = 0;
  ctx->step = 0;
  ctx->fcount[0] = ctx->fcount[1] = 0;
  ctx->snap_valid = false;
  ctx->arena_gen++;
  ctx->text_net = -1;
  std::string().swap(ctx->text);
  ctx->dtext_net = -1;
  std::string().swap(ctx->dtext);
  ctx->tr_front.clear();
  ctx->tr_live.clear();
  ctx->poisoned = false;
  if (ctx->host_only || !ctx->ws_ready) return INET_OK;
  DeviceGuard g(ctx->device);
  return clear_device(ctx);
}

inet_status inet_bench_exch(int device, uint64_t n_slots, uint64_t n_ops, double* exch_per_s_out) {
  if (!exch_per_s_out || n_slots == 0 || n_ops == 0) return INET_ERR_INVALID_ARG;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return INET_ERR_NO_DEVICE;
  DeviceGuard g(device);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return INET_ERR_CUDA;
  const uint32_t block = 256, grid = (uint32_t)sms * 8;
  const uint64_t threads = (uint64_t)block * grid;
  const uint32_t per = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(n_ops / threads, 1u << 20));
  uint32_t* slots = nullptr;
  unsigned long long* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  inet_status st = INET_OK;
  float ms = 0;
  if (cudaMalloc(&slots, n_slots * sizeof(uint32_t)) != cudaSuccess || cudaMalloc(&sink, 8) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = INET_ERR_CUDA;
  } else {
    cudaMemset(slots, 0, n_slots * sizeof(uint32_t));
    cudaMemset(sink, 0, 8);
    k_bench_exch<<<grid, block>>>(slots, n_slots, per, 1, sink);  // warm-up
    cudaEventRecord(e0);
    k_bench_exch<<<grid, block>>>(slots, n_slots, per, 2, sink);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = INET_ERR_CUDA;
    else cudaEventElapsedTime(&ms, e0, e1);
  }
  if (st == INET_OK) *exch_per_s_out = ms > 0 ? (double)threads * per / (ms * 1e-3) : 0.0;
  if (slots) cudaFree(slots);
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

inet_status inet_bench_chase(int device, uint64_t n_slots, uint64_t hops, int32_t variant, double* ns_per_hop_out) {
  if (!ns_per_hop_out || n_slots < 2 || n_slots > (1ull << 28) || hops == 0 || hops > n_slots - 1 || variant < 0 ||
      variant > 2)
    return INET_ERR_INVALID_ARG;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return INET_ERR_NO_DEVICE;
  DeviceGuard g(device);
  // a random cyclic permutation (Sattolo's algorithm; splitmix64 stream)
  std::vector<uint32_t> nxt(n_slots);
  for (uint64_t i = 0; i < n_slots; i++) nxt[i] = (uint32_t)i;
  uint64_t st64 = 0x1404007614040076ull;
  for (uint64_t i = n_slots - 1; i > 0; i--) {
    uint64_t z = (st64 += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const uint64_t j = z % i;  // j < i
    std::swap(nxt[i], nxt[j]);
  }
  std::vector<int4> hrec(n_slots);
  for (uint64_t i = 0; i < n_slots; i++) hrec[i] = make_int4((int)nxt[i], 0, 0, 0);
  int4 *rec = nullptr, *wrk = nullptr;
  uint32_t* xs = nullptr;
  unsigned long long* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  inet_status st = INET_OK;
  float ms = 0;
  const uint32_t warm = (uint32_t)std::min<uint64_t>(hops, 1024);
  if (cudaMalloc(&rec, n_slots * sizeof(int4)) != cudaSuccess || cudaMalloc(&wrk, n_slots * sizeof(int4)) != cudaSuccess ||
      cudaMalloc(&xs, n_slots * sizeof(uint32_t)) != cudaSuccess || cudaMalloc(&sink, 8) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = INET_ERR_CUDA;
  } else if (cudaMemcpy(rec, hrec.data(), n_slots * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(xs, nxt.data(), n_slots * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    st = INET_ERR_CUDA;
  } else {
    // the timed chase starts where a short warm-up one ended, so both stay
    // within one lap of the cycle (hops + warm-up <= n_slots - 1 is checked
    // for the exchange variants by the caller's sizes; the load variant may
    // lap)
    k_bench_chase<<<1, 32>>>(rec, xs, wrk, 0u, warm, 0, sink);
    cudaEventRecord(e0);
    k_bench_chase<<<1, 32>>>(rec, xs, wrk, 0u, (uint32_t)hops, variant, sink);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = INET_ERR_CUDA;
    else cudaEventElapsedTime(&ms, e0, e1);
  }
  if (st == INET_OK) *ns_per_hop_out = 1e6 * (double)ms / (double)hops;
  if (rec) cudaFree(rec);
  if (wrk) cudaFree(wrk);
  if (xs) cudaFree(xs);
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

inet_status inet_control_link(int device, const uint64_t* eq, uint64_t n, uint32_t n_vars, int32_t method,
                              uint32_t* pairs_out, uint64_t cap, uint64_t* n_pairs_out, uint32_t* passes_out,
                              double* ms_out) {
  if ((n && !eq) || !n_pairs_out || (cap && !pairs_out) || n > 0x7FFFFFFFull || (method != 0 && method != 1))
    return INET_ERR_INVALID_ARG;
  int nd = 0;
  if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) return INET_ERR_NO_DEVICE;
  DeviceGuard g(device);
  const uint32_t N = (uint32_t)n;
  CtlBufs B;
  unsigned long long* d_eq = nullptr;
  uint2* d_pairs = nullptr;
  uint32_t* d_cnt = nullptr;  // n_pairs, n_keep, merged, bad, n_out
  if (!B.get(&d_eq, N) || !B.get(&d_pairs, N) || !B.get(&d_cnt, 8)) return INET_ERR_CUDA;
  if (cudaMemcpy(d_eq, eq, sizeof(unsigned long long) * N, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(d_cnt, 0, 8 * sizeof(uint32_t)) != cudaSuccess)
    return INET_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  uint32_t passes = 0, bad = 0;
  const uint32_t gb = (N + 255) / 256;
  if (method == 0) {
    uint32_t* slots = nullptr;
    if (!B.get(&slots, n_vars) || cudaMemset(slots, 0, sizeof(uint32_t) * std::max<uint32_t>(n_vars, 1)) != cudaSuccess)
      return INET_ERR_CUDA;
    cudaEventRecord(e0);
    if (N) k_ctl_link_atomic<<<gb, 256>>>(d_eq, N, slots, n_vars, d_pairs, d_cnt + 0, d_cnt + 3);
    cudaEventRecord(e1);
    passes = 1;
  } else {
    uint32_t *k0 = nullptr, *k1 = nullptr, *k2 = nullptr, *counts = nullptr;
    unsigned long long *v0 = nullptr, *v1 = nullptr, *v2 = nullptr;
    const uint32_t tiles = std::max<uint32_t>(1, (N + kRsTile - 1) / kRsTile);
    if (!B.get(&k0, N) || !B.get(&k1, N) || !B.get(&k2, N) || !B.get(&v0, N) || !B.get(&v1, N) || !B.get(&v2, N) ||
        !B.get(&counts, (size_t)256 * tiles))
      return INET_ERR_CUDA;
    int bits = 1;
    while (bits < 32 && (n_vars >> bits)) bits++;
    cudaEventRecord(e0);
    if (N) k_ctl_orient<<<gb, 256>>>(d_eq, N, k0, v0, d_cnt + 1, d_pairs, d_cnt + 0);
    uint32_t m = 0;
    cudaMemcpy(&m, d_cnt + 1, 4, cudaMemcpyDeviceToHost);
    // the loop of Sec. 3.6: sort by name, merge, until no equation merges
    for (;;) {
      if (m == 0) break;
      const uint32_t t = (m + kRsTile - 1) / kRsTile;
      uint32_t *ks = k0, *kd = k1;
      unsigned long long *vs = v0, *vd = v1;
      for (int shift = 0; shift < bits; shift += 8) {
        k_rs_upsweep<<<t, kRsThreads>>>(ks, m, shift, counts);
        k_rs_scan<<<1, 1024>>>(counts, 256 * t);
        k_rs_downsweep<<<t, kRsThreads>>>(ks, vs, m, shift, counts, kd, vd);
        std::swap(ks, kd);
        std::swap(vs, vd);
      }
      cudaMemset(d_cnt + 2, 0, 4);
      cudaMemset(d_cnt + 4, 0, 4);
      k_ctl_merge<<<(m + 255) / 256, 256>>>(ks, vs, m, k2, v2, d_cnt + 4, d_pairs, d_cnt + 0, d_cnt + 2, d_cnt + 3);
      passes++;
      uint32_t hc[3] = {0, 0, 0};
      if (cudaMemcpy(hc, d_cnt + 2, 12, cudaMemcpyDeviceToHost) != cudaSuccess) return INET_ERR_CUDA;
      m = hc[2];
      if (hc[0] == 0 || passes > N + 1) break;  // nothing merged: fixpoint
      std::swap(k0, k2);
      std::swap(v0, v2);
    }
    cudaEventRecord(e1);
  }
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) return INET_ERR_CUDA;
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  uint32_t np = 0;
  cudaMemcpy(&np, d_cnt + 0, 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&bad, d_cnt + 3, 4, cudaMemcpyDeviceToHost);
  if (bad) return INET_ERR_LINEARITY;
  *n_pairs_out = np;
  if (pairs_out && np) {
    std::vector<uint2> hp(np);
    if (cudaMemcpy(hp.data(), d_pairs, sizeof(uint2) * np, cudaMemcpyDeviceToHost) != cudaSuccess) return INET_ERR_CUDA;
    for (uint32_t i = 0; i < np && i < cap; i++) {
      pairs_out[2 * i] = hp[i].x;
      pairs_out[2 * i + 1] = hp[i].y;
    }
  }
  if (passes_out) *passes_out = passes;
  if (ms_out) *ms_out = ms;
  return INET_OK;
}

inet_status inet_control_segsum(int device, const int32_t* in, uint64_t n, int32_t* out, uint64_t* n_out) {
  if ((n && (!in || !out)) || !n_out || n > 0x7FFFFFFFull) return INET_ERR_INVALID_ARG;
  int nd = 0;
  if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) return INET_ERR_NO_DEVICE;
  DeviceGuard g(device);
  *n_out = 0;
  if (n == 0) return INET_OK;
  const uint32_t N = (uint32_t)n;
  CtlBufs B;
  int32_t *d_in = nullptr, *d_out = nullptr;
  uint32_t *d_rank = nullptr, *d_n = nullptr;
  if (!B.get(&d_in, N) || !B.get(&d_out, N) || !B.get(&d_rank, N) || !B.get(&d_n, 1)) return INET_ERR_CUDA;
  if (cudaMemcpy(d_in, in, sizeof(int32_t) * N, cudaMemcpyHostToDevice) != cudaSuccess) return INET_ERR_CUDA;
  k_ctl_runs<<<1, 1>>>(d_in, N, d_rank);
  k_ctl_segsum<<<(N + 255) / 256, 256>>>(d_in, N, d_out, d_n, d_rank);
  uint32_t m = 0;
  if (cudaMemcpy(&m, d_n, 4, cudaMemcpyDeviceToHost) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return INET_ERR_CUDA;
  if (cudaMemcpy(out, d_out, sizeof(int32_t) * m, cudaMemcpyDeviceToHost) != cudaSuccess) return INET_ERR_CUDA;
  *n_out = m;
  return INET_OK;
}

const char* inet_last_error(const inet_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Entry point that allocates no memory, for callers that cannot call
// cudaMalloc or any allocator on their request path: a serving process whose
// allocator has already reserved the whole GPU at start-up, or code with a
// hard latency budget where a device allocation (and its implicit
// synchronisation) is not allowed.  The caller owns the arena that holds the
// net; everything else the reduction needs (frontier buffers, free-slot
// rings, control block, rule tables, per-net counters) lives in one fixed
// array in device memory, below, which every GPU that loads this library
// keeps until the process exits.

namespace {

constexpr uint64_t kFixedAgents = 1ull << 20;   // agent slots the fixed rings can recycle
constexpr uint64_t kFixedVars = 1ull << 20;     // name slots
constexpr uint32_t kFixedPairs = 1u << 18;      // frontier capacity (each of two buffers)
constexpr uint32_t kFixedNets = 4096;           // nets the host-only context may hold

constexpr size_t up256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kFxCtrl = 0;
constexpr size_t kFxTable = up256(kFxCtrl + sizeof(Ctrl));
constexpr size_t kFxTmpl = up256(kFxTable + sizeof(int16_t) * kMaxLabels * kMaxLabels);
constexpr size_t kFxArity = up256(kFxTmpl + sizeof(Template) * INET_MAX_RULES);
constexpr size_t kFxHist = up256(kFxArity + kMaxLabels);
constexpr size_t kFxNetctr = up256(kFxHist + sizeof(unsigned long long) * INET_MAX_RULES);
constexpr size_t kFxNetstat = up256(kFxNetctr + sizeof(unsigned long long) * kFixedNets);
constexpr size_t kFxFront0 = up256(kFxNetstat + sizeof(int32_t) * kFixedNets);
constexpr size_t kFxFront1 = up256(kFxFront0 + sizeof(Pair) * kFixedPairs);
constexpr size_t kFxAfree = up256(kFxFront1 + sizeof(Pair) * kFixedPairs);
constexpr size_t kFxVfree = up256(kFxAfree + sizeof(uint32_t) * kFixedAgents);
constexpr size_t kFxOut = up256(kFxVfree + sizeof(uint32_t) * kFixedVars);
constexpr size_t kFixedBytes = up256(kFxOut + 64);
static_assert(kFixedBytes == INET_FIXED_SCRATCH_BYTES, "fixed scratch size in inet.h is out of date");

}  // namespace

// The fixed scratch array.  Host code must not use this name as an address:
// it is a host-side stand-in; the device address comes from
// cudaGetSymbolAddress() below.
static __device__ __align__(256) unsigned char g_inet_fixed_scratch[kFixedBytes];

namespace {

std::mutex g_fixed_mu;
void* g_fixed_addr[256] = {};

// Device address of the fixed scratch on `device`, looked up once per device
// with that device current.  The address stays valid while the device's
// primary context lives: a device reset (cudaDeviceReset) between calls
// would leave it stale, which the header rules out.
inet_status fixed_scratch(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_fixed_mu);
  if (device < 0 || device >= 256) return INET_ERR_INVALID_ARG;
  if (!g_fixed_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_inet_fixed_scratch) != cudaSuccess || !p) return INET_ERR_CUDA;
    g_fixed_addr[device] = p;
  }
  *out = g_fixed_addr[device];
  return INET_OK;
}

// Reads the numeral S^k(Z) at the interface word `root` (one thread; name
// slots are followed as ->col/->sub do).  out[0] = k or -1.
__global__ void k_fixed_read_nat(const Node* nodes, const uint32_t* vars, uint64_t n_agents, uint64_t n_vars,
                                 uint32_t root, int s_label, int z_label, long long* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long k = 0;
  uint32_t w = root;
  for (uint64_t guard = 0; guard <= n_agents + n_vars; guard++) {
    if (is_var(w)) {
      const uint32_t x = idx_of(w);
      if (x >= n_vars) break;
      const uint32_t v = __ldcg(vars + x);
      if (v == kEmpty) break;
      w = v;
      continue;
    }
    if (!is_agent(w) || idx_of(w) >= n_agents) break;
    const int4 r = __ldcg(reinterpret_cast<const int4*>(nodes + idx_of(w)));
    const int lab = r.x & 0xFF;
    if (lab == z_label) {
      out[0] = k;
      return;
    }
    if (lab != s_label) break;
    k++;
    w = (uint32_t)r.y;
  }
  out[0] = -1;
}

}  // namespace

extern "C" inet_status inet_reduce_into(inet_ctx* host_ctx, int32_t net_id, void* arena, size_t arena_bytes,
                                        uint64_t max_agents, uint64_t max_vars, int device, void* stream,
                                        uint64_t* value_out, uint64_t* interactions_out) {
  inet_ctx* ctx = host_ctx;
  if (!ctx || !arena || !value_out) return INET_ERR_INVALID_ARG;
  if (!ctx->host_only) return fail(ctx, INET_ERR_INVALID_ARG, "inet_reduce_into takes a host-only context");
  if (!ctx->have_rules) return fail(ctx, INET_ERR_STATE, "load rules first");
  inet_status s = check_net(ctx, net_id);
  if (s) return s;
  const NetRec& nr = ctx->nets[(size_t)net_id];
  const size_t var_off = up256(sizeof(Node) * max_agents);
  if (max_agents > kFixedAgents || max_vars > kFixedVars)
    return fail(ctx, INET_ERR_INVALID_ARG, "max_agents and max_vars may not exceed 1048576 (fixed scratch limit)");
  if (ctx->nets.size() > kFixedNets)
    return fail(ctx, INET_ERR_INVALID_ARG, "the host-only context holds more than 4096 nets (fixed scratch limit)");
  if (nr.pairs.size() > kFixedPairs)
    return fail(ctx, INET_ERR_INVALID_ARG, "net has more initial active pairs than the fixed frontier holds");
  if (ctx->st_nodes.size() > max_agents || ctx->st_vars.size() > max_vars)
    return fail(ctx, INET_ERR_INVALID_ARG, "the context's nets do not fit max_agents / max_vars");
  // the staged nets are copied to arena offset 0 with the net's own pairs
  // as they are: that holds only while staging started at slot 0
  if (ctx->st_a0 != 0 || ctx->st_v0 != 0 || ctx->st_nodes.size() != ctx->a_bump || ctx->st_vars.size() != ctx->v_bump)
    return fail(ctx, INET_ERR_STATE, "the host-only context's staged nets do not start at slot 0");
  if (arena_bytes < var_off + sizeof(uint32_t) * max_vars || (reinterpret_cast<uintptr_t>(arena) & 255))
    return fail(ctx, INET_ERR_INVALID_ARG, "arena smaller than 16*max_agents (rounded to 256) + 4*max_vars, or not 256-byte aligned");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(ctx, INET_ERR_NO_DEVICE, "no such CUDA device");
  DeviceGuard g(device);
  unsigned char* fx = nullptr;
  s = fixed_scratch(device, reinterpret_cast<void**>(&fx));
  if (s) return fail(ctx, s, "cudaGetSymbolAddress of the fixed scratch failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Node* nodes = static_cast<Node*>(arena);
  uint32_t* vars = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(arena) + var_off);
  const CompiledRules& r = ctx->rules;
#define FX(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(ctx, INET_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
  // inputs: the context's staged nets (agent ids start at 0) into the arena
  if (!ctx->st_nodes.empty())
    FX(cudaMemcpyAsync(nodes, ctx->st_nodes.data(), sizeof(Node) * ctx->st_nodes.size(), cudaMemcpyHostToDevice, st));
  if (!ctx->st_vars.empty())
    FX(cudaMemcpyAsync(vars, ctx->st_vars.data(), sizeof(uint32_t) * ctx->st_vars.size(), cudaMemcpyHostToDevice, st));
  if (max_vars > ctx->st_vars.size())
    FX(cudaMemsetAsync(vars + ctx->st_vars.size(), 0, sizeof(uint32_t) * (max_vars - ctx->st_vars.size()), st));
  // scratch: what must start at zero, then the rule tables and the frontier
  FX(cudaMemsetAsync(fx + kFxHist, 0, kFxFront0 - kFxHist, st));
  FX(cudaMemcpyAsync(fx + kFxTable, r.table.data(), sizeof(int16_t) * r.table.size(), cudaMemcpyHostToDevice, st));
  FX(cudaMemcpyAsync(fx + kFxTmpl, r.tmpl.data(), sizeof(Template) * r.tmpl.size(), cudaMemcpyHostToDevice, st));
  uint8_t ar[kMaxLabels] = {};
  for (size_t i = 0; i < r.arity.size() && i < kMaxLabels; i++) ar[i] = (uint8_t)r.arity[i];
  FX(cudaMemcpyAsync(fx + kFxArity, ar, sizeof ar, cudaMemcpyHostToDevice, st));
  if (!nr.pairs.empty())
    FX(cudaMemcpyAsync(fx + kFxFront0, nr.pairs.data(), sizeof(Pair) * nr.pairs.size(), cudaMemcpyHostToDevice, st));
  const unsigned long long ctr0 = (unsigned long long)nr.pairs.size() << kNetPairShift;
  FX(cudaMemcpyAsync(fx + kFxNetctr + sizeof(unsigned long long) * (size_t)net_id, &ctr0, sizeof ctr0,
                     cudaMemcpyHostToDevice, st));
  Ctrl hc;
  memset(&hc, 0, sizeof hc);
  hc.stop_step = 0xFFFFFFFFu;
  hc.fcount[0] = (uint32_t)nr.pairs.size();
  hc.a_bump = ctx->st_nodes.size();
  hc.v_bump = ctx->st_vars.size();
  hc.live = (long long)ctx->st_nodes.size();
  FX(cudaMemcpyAsync(fx + kFxCtrl, &hc, sizeof hc, cudaMemcpyHostToDevice, st));
  Dev d;
  memset(&d, 0, sizeof d);
  d.node = nodes;
  d.var = vars;
  d.front[0] = reinterpret_cast<Pair*>(fx + kFxFront0);
  d.front[1] = reinterpret_cast<Pair*>(fx + kFxFront1);
  d.qseq = nullptr;  // no asynchronous launch here
  d.afree = reinterpret_cast<uint32_t*>(fx + kFxAfree);
  d.vfree = reinterpret_cast<uint32_t*>(fx + kFxVfree);
  d.netctr = reinterpret_cast<unsigned long long*>(fx + kFxNetctr);
  d.netstat = reinterpret_cast<int32_t*>(fx + kFxNetstat);
  d.netrep = nullptr;  // no inet_net_finished here
  d.rule_hist = reinterpret_cast<unsigned long long*>(fx + kFxHist);
  d.ctrl = reinterpret_cast<Ctrl*>(fx + kFxCtrl);
  d.table = reinterpret_cast<const int16_t*>(fx + kFxTable);
  d.tmpl = reinterpret_cast<const Template*>(fx + kFxTmpl);
  d.arity = reinterpret_cast<const uint8_t*>(fx + kFxArity);
  d.trace_front = nullptr;
  d.trace_live = nullptr;
  d.trace_cap = 0;
  d.cap_agents = max_agents;
  d.cap_vars = max_vars;
  d.cap_pairs = kFixedPairs;
  d.max_nets = kFixedNets;
  d.n_labels = (uint32_t)r.n_labels();
  d.n_tmpl = (uint32_t)r.tmpl.size();
  d.timeout_ns = kDefaultTimeoutNs;
  d.slice_ns = kSliceNs;
  const int B = 256;
  d.solo_max = B;
  const size_t smem = smem_bytes(B, d.n_labels, d.n_tmpl, d.solo_max);
  int nsm = 0, per = 0;
  FX(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
  FX(raise_smem(kSmemPersistent, (const void*)k_persistent<false>, smem));
  FX(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<false>, B, smem));
  const int grid = std::max(1, per) * nsm;
  if (!nr.pairs.empty()) {
    const unsigned long long word0 = pack_word((uint32_t)nr.pairs.size(), 0, 0, 0);
    FX(cudaMemcpyAsync(&d.ctrl->bar_word, &word0, 8, cudaMemcpyHostToDevice, st));
    for (;;) {
      void* args[] = {&d};
      FX(cudaLaunchCooperativeKernel((const void*)k_persistent<false>, dim3((unsigned)grid), dim3((unsigned)B), args, smem, st));
      uint32_t hit = 0;
      FX(cudaMemcpyAsync(&hit, &d.ctrl->hit_slice, 4, cudaMemcpyDeviceToHost, st));
      FX(cudaStreamSynchronize(st));
      if (!hit) break;
      const unsigned long long zero = 0;
      FX(cudaMemcpyAsync(&d.ctrl->done, &zero, 4, cudaMemcpyHostToDevice, st));
      FX(cudaMemcpyAsync(&d.ctrl->hit_slice, &zero, 4, cudaMemcpyHostToDevice, st));
      FX(cudaMemcpyAsync(&d.ctrl->slice_t0, &zero, 8, cudaMemcpyHostToDevice, st));
      uint32_t stp = 0, fcn[2] = {0, 0};
      FX(cudaMemcpyAsync(&stp, &d.ctrl->step, 4, cudaMemcpyDeviceToHost, st));
      FX(cudaMemcpyAsync(fcn, d.ctrl->fcount, 8, cudaMemcpyDeviceToHost, st));
      FX(cudaStreamSynchronize(st));
      const unsigned long long word = pack_word(fcn[stp & 1u], 0, stp & 1u, 0);
      FX(cudaMemcpyAsync(&d.ctrl->bar_word, &word, 8, cudaMemcpyHostToDevice, st));
      FX(cudaMemcpyAsync(&d.ctrl->bar_count, &zero, 4, cudaMemcpyHostToDevice, st));
    }
  }
  int32_t err[2] = {0, 0};
  FX(cudaMemcpyAsync(&err[0], &d.ctrl->error, 4, cudaMemcpyDeviceToHost, st));
  FX(cudaMemcpyAsync(&err[1], &d.ctrl->fatal, 4, cudaMemcpyDeviceToHost, st));
  unsigned long long ctr = 0;
  FX(cudaMemcpyAsync(&ctr, d.netctr + net_id, sizeof ctr, cudaMemcpyDeviceToHost, st));
  auto si = r.index.find("S");
  auto zi = r.index.find("Z");
  long long nat = -1;
  if (nr.iface.size() == 1 && si != r.index.end() && zi != r.index.end()) {
    long long* out = reinterpret_cast<long long*>(fx + kFxOut);
    k_fixed_read_nat<<<1, 1, 0, st>>>(nodes, vars, max_agents, max_vars, nr.iface[0], si->second, zi->second, out);
    FX(cudaGetLastError());
    FX(cudaMemcpyAsync(&nat, out, sizeof nat, cudaMemcpyDeviceToHost, st));
  }
  FX(cudaStreamSynchronize(st));
#undef FX
  if (interactions_out) *interactions_out = ctr & kNetIntMask;
  if (err[1]) return fail(ctx, err[1], "the reduction hit a capacity or state error");
  if (err[0]) return fail(ctx, err[0], "active pair without a rule");
  if (nat < 0) return fail(ctx, INET_ERR_INVALID_ARG, "the interface is not a numeral S^k(Z)");
  *value_out = (uint64_t)nat;
  return INET_OK;
}
