/*
 * inet.h -- C ABI of the GB300 interaction-net evaluator.
 *
 * The library evaluates configurations < t.. | Delta > of the lightweight
 * interaction calculus (Sec. 2.2) under a set of interaction rules
 * alpha(x..) = beta(y..) -> Theta.  The hot loop is the data-parallel
 * reduction step of Sec. 3.3-3.5: every active pair of the current frontier
 * is rewritten by its rule (->int), the new agents and names are allocated,
 * and the new equations are linked (->com, with ->sub of auxiliary ports at
 * instantiation), until no active pair remains (Sec. 3.6, evaluate()).
 * ->col and the remaining ->sub steps are applied at readback (Theorem 1).
 *
 * Conventions (all entry points):
 *   - Every function returns an inet_status: INET_OK (0) or a negative code.
 *     Errors never abort the process; inet_last_error() gives a message.
 *   - The caller owns every host buffer it passes; the library copies what
 *     it needs during the call and keeps no caller pointer, except for the
 *     device workspace given to inet_attach_workspace().
 *   - Device work is ordered on the context's CUDA stream.  inet_reduce()
 *     returns when the requested reduction has finished on the device.
 *   - A context is used by one host thread at a time.
 *   - Text syntax: agent symbols start with an upper-case letter, names
 *     with a lower-case letter (Sec. 3.3).  A rule is
 *       Alpha(x1, .., xn) = Beta(y1, .., ym) -> t1 = u1, .., tk = uk;
 *     (an empty right-hand side is written "-> ;") and a net is
 *       < t1, .., tp | u1 = v1, .., uq = vq >
 *     '#' starts a comment.  Arity is fixed by first use (at most 3).
 */
#ifndef INET_H
#define INET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct inet_ctx inet_ctx;
typedef struct inet_parsed inet_parsed;
typedef int32_t inet_status;

enum {
  INET_OK = 0,
  INET_ERR_INVALID_ARG = -1, /* bad pointer, size, id or option; truncated readback */
  INET_ERR_PARSE = -2,       /* malformed text, unknown symbol, arity mismatch */
  INET_ERR_LINEARITY = -3,   /* a name occurs more than twice (Sec. 2.2, Configurations),
                                or a rule name is not bound linearly */
  INET_ERR_NO_RULE = -4,     /* an active pair has no rule (premise of the
                                Proposition on the correctness of evaluate(), Sec. 3.6) */
  INET_ERR_ARENA_FULL = -5,  /* agent, name, frontier or net capacity exhausted */
  INET_ERR_STEP_LIMIT = -6,  /* inet_reduce_opts.max_steps reached; resumable */
  INET_ERR_TIMEOUT = -7,     /* a device-side wait gave up (persistent form) */
  INET_ERR_CUDA = -8,        /* a CUDA runtime call failed */
  INET_ERR_NO_DEVICE = -9,   /* operation needs a GPU; context is host-only */
  INET_ERR_STATE = -10       /* call out of order, or context poisoned by an
                                earlier ARENA_FULL / TIMEOUT / CUDA error */
};

/* Capacities of the device arena.  Zero fields take defaults. */
typedef struct inet_arena_cfg {
  uint64_t max_agents; /* agent slots, 16 bytes each (default 1<<22) */
  uint64_t max_vars;   /* name slots, 4 bytes each (default 1<<22) */
  uint64_t max_pairs;  /* frontier capacity: active pairs at once (default 1<<21); two
                          buffers of 8 bytes per pair plus an 8-byte sequence number
                          per cell of the asynchronous driver's ticket queue */
  uint32_t max_nets;   /* independent nets held at once (default 1<<16) */
  uint32_t flags;      /* INET_ARENA_* bits (default 0) */
} inet_arena_cfg;

/* inet_arena_cfg.flags: keep the owning net of every name slot in use (4
 * bytes per name slot, and one store per name a reduction creates), which
 * inet_free_nets needs to find a net's names.  Without it inet_free_nets
 * returns INET_ERR_STATE; a batch that is reduced and read back once has no
 * use for it. */
#define INET_ARENA_FREE_NETS 1u

/* How the step loop of Sec. 3.6 (evaluate()) is driven. */
enum {
  INET_MODE_PLAIN = 0,      /* host loop: one kernel launch and one 16-byte
                               device-to-host read of the frontier size per step */
  INET_MODE_GRAPH = 1,      /* the step kernel inside a CUDA graph with a
                               conditional WHILE node; no host round trip */
  INET_MODE_PERSISTENT = 2, /* one cooperative launch; a grid barrier between
                               steps; narrow frontiers run on one block */
  INET_MODE_ASYNC = 3,      /* one cooperative launch without steps: every warp
                               reduces pairs as they appear (active pairs are
                               independent, Sec. 2.1); no per-step trace; more
                               than max_pairs pairs in flight at once is
                               INET_ERR_ARENA_FULL */
  INET_MODE_PAPER = 4       /* the paper's own loop (Sec. 3.6): each step writes
                               the name equations of every active pair to n
                               result slots of its own, dummies in the rest,
                               and a stream compaction removes the dummies
                               (Sec. 3.4); then one communication pass sorts
                               the equations by name and folds adjacent pairs
                               (Sec. 3.5), until neither produced anything; for
                               comparison.  Runs to the end (max_steps and
                               slice_us are ignored); needs 2 * max_vars
                               equations of scratch (36 bytes each) and n
                               slots of 8 bytes per frontier pair, allocated
                               per call; freed names return to the ring */
};

typedef struct inet_reduce_opts {
  int32_t mode;          /* INET_MODE_* */
  int32_t block;         /* threads per block, multiple of 32 in [64, 512] (ASYNC: [32, 256]); 0 = 256 */
  int32_t grid;          /* blocks for GRAPH / PERSISTENT / ASYNC; 0 = automatic
                            (ASYNC and PERSISTENT: as many as can be resident,
                            full occupancy) */
  int32_t solo_max;      /* PERSISTENT: frontier sizes <= solo_max run on block 0
                            alone; 0 = automatic, < 0 = never */
  uint64_t max_steps;    /* stop after this many steps of this call (0 = no limit);
                            returns INET_ERR_STEP_LIMIT, state stays resumable */
  uint64_t timeout_ns;   /* limit of any device-side wait (0 = 10 s) */
  int32_t trace;         /* 1 = record frontier size and live agents per step
                            (not in ASYNC mode, which has no steps) */
  int32_t slice_us;      /* ASYNC: if > 0 the call returns after about this many
                            microseconds with INET_ERR_STEP_LIMIT when pairs are
                            left (resumable); 0 = run to the end */
} inet_reduce_opts;

#define INET_MAX_RULES 64

typedef struct inet_reduce_stats {
  uint64_t interactions;        /* ->int steps performed by this call */
  uint64_t steps;               /* loop iterations of this call */
  uint64_t max_frontier;        /* largest frontier seen in this call */
  int64_t  live_agents;         /* agents alive after the call (all nets) */
  int64_t  peak_live_agents;    /* max of live agents at step boundaries */
  uint64_t pending_pairs;       /* active pairs left (non-zero after STEP_LIMIT) */
  double   device_ms;           /* device time of the step loop (CUDA events) */
  uint32_t n_rules;
  uint32_t launches;            /* kernel launches of this call (a graph's
                                   body counts once per step) */
  uint64_t per_rule[INET_MAX_RULES]; /* interactions by rule, rule-text order */
} inet_reduce_stats;

typedef struct inet_net_stats {
  int32_t  status;        /* INET_OK or the first error of this net */
  int32_t  reduced;       /* 1 once the net has no pending pair */
  uint64_t interactions;  /* ->int steps of this net so far */
  uint64_t pending_pairs; /* active pairs of this net in the frontier */
  int64_t  live_agents;   /* agents of this net alive (readback snapshot) */
  int64_t  residual_agents; /* live agents not reachable from the interface */
} inet_net_stats;

/* Shape of one compiled rule (for byte accounting and tools). */
typedef struct inet_rule_desc {
  char name[64];        /* "Alpha><Beta" */
  int32_t arity_alpha;  /* auxiliary ports of the two LHS agents */
  int32_t arity_beta;
  int32_t n_new;        /* agents of Theta */
  int32_t new_ports;    /* sum of the arities of the agents of Theta */
  int32_t n_fresh;      /* bound names of Theta joining two auxiliary ports */
  int32_t n_link;       /* equations of Theta' linked after instantiation */
} inet_rule_desc;

/* Number of rules of the loaded rule set. */
inet_status inet_rule_count(const inet_ctx* ctx, int32_t* n_out);

/* Shape of rule `rule` (text order, 0-based). */
inet_status inet_rule_info(const inet_ctx* ctx, int32_t rule, inet_rule_desc* out);

/* Workspace bytes the given capacities need (cfg may be NULL). */
inet_status inet_workspace_bytes(const inet_arena_cfg* cfg, size_t* bytes_out);

/* Creates a context on CUDA device `device` (device < 0: host-only context,
 * which parses and loads but cannot reduce: INET_ERR_NO_DEVICE).  `stream`
 * is a cudaStream_t or NULL for a stream the context creates.  `cfg` may be
 * NULL.  The device workspace is allocated at the first load unless one is
 * attached first. */
inet_status inet_create(inet_ctx** out, int device, void* stream, const inet_arena_cfg* cfg);

/* Uses caller-owned device memory (e.g. from a PyTorch allocator) as the
 * workspace.  `bytes` must be >= inet_workspace_bytes() for the context's
 * capacities and `dptr` 256-byte aligned.  The memory must stay valid until
 * inet_destroy().  Must be called before the first load. */
inet_status inet_attach_workspace(inet_ctx* ctx, void* dptr, size_t bytes);

void inet_destroy(inet_ctx* ctx);

/* Parses and compiles a rule set (Sec. 2.2, Interaction Rules): checks
 * arities and linearity (every LHS name occurs once in Theta, every other
 * name twice), stores each rule under the unordered pair {alpha, beta}
 * (t = s is s = t, Sec. 2.2) and compiles Theta into an instantiation
 * template.  Replaces any earlier rule set; allowed only while no net is
 * loaded. */
inet_status inet_load_rules(inet_ctx* ctx, const char* text, size_t len);

/* Parses one configuration < t.. | Delta > (Sec. 2.2, Configurations),
 * checks that every name occurs at most twice, flattens nested terms into
 * agent records (a subterm's principal port is linked to its parent's
 * auxiliary port), applies ->com to the initial equations, and stages the
 * result for the device.  Returns the net id. */
inet_status inet_load_net(inet_ctx* ctx, const char* text, size_t len, int32_t* net_id_out);

/* inet_load_net() for n nets in one call: net i is the text
 * buf[offsets[i] .. offsets[i+1]) (offsets has n + 1 entries).  The texts
 * are parsed and placed on a process-wide pool of host threads (started on
 * first use; a call made while another runs, or in a process forked after
 * the pool started, works on the calling thread) and staged in order;
 * ids_out[i] gets net i's id.  Stops at the first net that fails (its error
 * is returned) with *n_loaded_out = the number of nets loaded before it. */
inet_status inet_load_nets(inet_ctx* ctx, const char* buf, const uint64_t* offsets, int32_t n, int32_t* ids_out,
                           int32_t* n_loaded_out);

/* inet_load_nets() in two halves, so that parsing can overlap the device
 * work of the context: inet_parse_nets parses and flattens n nets (net i
 * is buf[offsets[i] .. offsets[i+1])) with the context's rule set only, on
 * the process-wide pool of host threads, into a new batch *out that the
 * caller frees with inet_parsed_free.  It reads nothing of the context but
 * its rules, so it may run on another host thread while the context is in
 * use (the rules must not change meanwhile).  Parse errors are kept per net
 * and reported when that net is loaded.  inet_load_parsed then places nets
 * [first, first + n) of the batch in the context like inet_load_nets (ids,
 * capacity checks, staging; the first net that fails stops it, with
 * *n_loaded_out the nets loaded before it); each net of a batch can be
 * loaded once (INET_ERR_INVALID_ARG otherwise), and only into a context
 * with the same rule set (INET_ERR_STATE otherwise).  inet_parsed_info
 * gives the nets in the batch and their agents in total (either pointer
 * may be NULL).  The paper has no counterpart. */
inet_status inet_parse_nets(const inet_ctx* ctx, const char* buf, const uint64_t* offsets, int32_t n,
                            inet_parsed** out);
inet_status inet_parsed_info(const inet_parsed* p, int32_t* n_out, uint64_t* agents_out);
inet_status inet_load_parsed(inet_ctx* ctx, inet_parsed* p, int32_t first, int32_t n, int32_t* ids_out,
                             int32_t* n_loaded_out);
void inet_parsed_free(inet_parsed* p);

/* Adds the active pairs of the listed nets (which must not have been
 * staged or reduced yet; n may be 0) to the frontier and runs the reduction loop of
 * Sec. 3.6 until no active pair remains in the whole context, an error
 * occurs, or opts->max_steps steps have run.  opts and stats may be NULL.
 * Per-net errors (NO_RULE) do not stop other nets; the first error is
 * returned. */
inet_status inet_reduce(inet_ctx* ctx, const int32_t* net_ids, int32_t n,
                        const inet_reduce_opts* opts, inet_reduce_stats* stats);

/* Admission without running: uploads loaded nets and adds the active pairs
 * of the listed nets (not yet staged or reduced) to the device frontier.
 * A later inet_reduce(ctx, NULL, 0, ...) reduces them together with any
 * pairs already in flight. */
inet_status inet_stage(inet_ctx* ctx, const int32_t* net_ids, int32_t n);

/* Total bytes this context has copied host-to-device and device-to-host
 * (either pointer may be NULL). */
inet_status inet_transfer_bytes(const inet_ctx* ctx, uint64_t* h2d_out, uint64_t* d2h_out);

/* Writes the net's interface after ->col and ->sub (Sec. 2.2; Theorem 1),
 * terms left to right, names renamed x0, x1, .. in order of first
 * occurrence, as a NUL-terminated string.  If cap is too small returns
 * INET_ERR_INVALID_ARG with *needed_out set (needed_out may be NULL).  The
 * text is rendered on the device: every agent of the net and every port
 * becomes an element of one list in text order, ranked by pointer jumping
 * (characters and names after each element), names numbered by first
 * occurrence, characters written at their offsets; only the text is copied
 * to the host.  A net whose interface does not unfold into a finite forest
 * (a subterm reached twice, a cycle) is rendered from a host snapshot of the
 * arena instead, by a walk with a bound.  The device scratch (48 bytes per
 * agent slot in use, 4 per name slot) is allocated with cudaMalloc on first
 * use and grown when needed.  The text is kept until the arena changes, so a
 * size query followed by the copy renders it once, and inet_net_info of the
 * same net then takes its live and residual agents from that render. */
inet_status inet_readback(inet_ctx* ctx, int32_t net_id, char* buf, size_t cap, size_t* needed_out);

/* How many texts inet_readback rendered on the device and how many on the
 * host (either pointer may be NULL).  The paper has no counterpart. */
inet_status inet_readback_counts(const inet_ctx* ctx, uint64_t* device_out, uint64_t* host_out);

/* If the net's interface is a single numeral S^k(Z), stores k.  Otherwise
 * INET_ERR_INVALID_ARG.  interactions_out (may be NULL) gets the net's
 * interaction count. */
inet_status inet_readback_nat(inet_ctx* ctx, int32_t net_id, uint64_t* value_out, uint64_t* interactions_out);

/* Pending active pairs of each listed net as of the end of the last
 * inet_reduce() (0 = the net is in normal form).  Host-only: no device work,
 * no copy. */
inet_status inet_net_pending(inet_ctx* ctx, const int32_t* net_ids, int32_t n, uint64_t* pending_out);

/* Nets finished since the last call: every net whose pending pairs are zero
 * (reduced to normal form, or stopped by INET_ERR_NO_RULE) and that no
 * earlier call reported, found by one device scan over the counters, so a
 * request loop learns of completions without copying every net's counter.
 * At most `cap` (<= 65536) ids go to ids_out, in no particular order; the
 * rest are reported by the next call.  *n_out gets the number written.  The
 * paper has no counterpart (Sec. 3.6 ends a whole evaluation). */
inet_status inet_net_finished(inet_ctx* ctx, int32_t* ids_out, int32_t cap, int32_t* n_out);

/* inet_readback_nat() for many nets at once, on the device, following name
 * slots as ->col/->sub do (Theorem 1): one thread walks each net for 256 S
 * agents; numerals that are longer are finished by list ranking: one scan
 * of the agent slots lists the agents of those nets (each record names its
 * net), and pointer jumping runs over that list only.  values_out[i] = k
 * when net i's interface is one numeral S^k(Z), else UINT64_MAX;
 * interactions_out (may be NULL) gets each net's interaction count.  Copies
 * only 16 bytes per net to the host.  The first call, and the first after
 * the arena has grown, allocates the ranking scratch (20 bytes per agent
 * slot in use) with cudaMalloc. */
inet_status inet_readback_nats(inet_ctx* ctx, const int32_t* net_ids, int32_t n, uint64_t* values_out,
                               uint64_t* interactions_out);

/* inet_readback_nats() without blocking the caller or the main stream: the
 * walk and the ranking run on a second stream of the context, after the work
 * queued so far on the main stream and alongside later inet_reduce() calls
 * (finished nets are never touched by the reduction of others, Sec. 2.1).
 * At most 65536 nets per batch and one batch in flight per context;
 * inet_reset() waits for it and drops its results.  The nets should be finished
 * (inet_net_pending() == 0); an unfinished net reads as not-a-numeral or as
 * a partial count.  The paper has no counterpart: it serves a request loop
 * that harvests results while the device keeps reducing. */
inet_status inet_readback_nats_begin(inet_ctx* ctx, const int32_t* net_ids, int32_t n);

/* Completes the batch begun last.  If it is done (wait != 0: once it is),
 * copies its n values (as inet_readback_nats()) and interaction counts
 * (interactions_out may be NULL) into arrays of at least `cap` entries, in
 * begin order, and sets *n_out = n; otherwise sets *n_out = -1 and returns
 * INET_OK.  INET_ERR_STATE when no batch is in flight. */
inet_status inet_readback_nats_end(inet_ctx* ctx, int32_t wait, uint64_t* values_out, uint64_t* interactions_out,
                                   int32_t cap, int32_t* n_out);

/* Returns every slot the listed nets still hold to the free rings: their
 * agents (found by the net id in each agent record) and their name slots
 * (found by the owner array), so that later loads and reductions reuse the
 * memory; the ids themselves are released too and handed out again by
 * later loads.  Nets are independent configurations (Sec. 2.2,
 * Configurations): nothing outside a net can reach its agents or names, so
 * once its result has been read back (->col / ->sub, Theorem 1) it can go.
 * The context must have been created with INET_ARENA_FREE_NETS (else
 * INET_ERR_STATE).  Every listed net must have been staged or reduced and must have no active
 * pair left (normal form, or stopped by INET_ERR_NO_RULE); otherwise
 * INET_ERR_STATE and nothing is freed.  A net listed twice is
 * INET_ERR_INVALID_ARG; a net in the non-blocking readback in flight is
 * INET_ERR_STATE.  At most 65536 nets per call.  One scan over every agent
 * and name slot in use (about 20 bytes of device traffic per slot), so a
 * request loop frees finished nets in batches.  After the call the ids are
 * unknown (INET_ERR_INVALID_ARG) until a load reuses them.  Loads place new
 * nets into freed slots before using never-used ones (inet_stage /
 * inet_reduce upload them above the bump pointers and move the top part
 * into slots the rings hold). */
inet_status inet_free_nets(inet_ctx* ctx, const int32_t* net_ids, int32_t n);

/* inet_free_nets() for one net. */
inet_status inet_free_net(inet_ctx* ctx, int32_t net_id);

/* Quotas: net net_ids[i] may hold at most quotas[i] live agents (0: no
 * limit).  After each launch of inet_reduce, a net that still has active
 * pairs and holds more agents than its quota gets INET_ERR_ARENA_FULL as its
 * own status (inet_net_status), its pairs leave the frontier, and it counts
 * as finished (inet_net_finished reports it; inet_free_nets can free it);
 * every other net is untouched.  A request loop that admits nets by an
 * estimate of their size gives each its estimate as quota, so a net that
 * outgrows its estimate stops alone instead of filling the arena that the
 * others share.  The arena must still hold what the nets can allocate within
 * one launch (a time slice, slice_us).  Needs INET_ARENA_FREE_NETS (the live
 * agents of each net are kept with the owners; else INET_ERR_STATE).  A
 * net's quota is reset when its id is loaded again.  At most 65536 nets per
 * call.  The paper has no counterpart. */
inet_status inet_set_quotas(inet_ctx* ctx, const int32_t* net_ids, const uint64_t* quotas, int32_t n);

/* The status of each listed net: INET_OK, INET_ERR_NO_RULE (an active pair
 * without a rule) or INET_ERR_ARENA_FULL (over its quota), as of the end of
 * the last inet_reduce.  The paper has no counterpart. */
inet_status inet_net_status(inet_ctx* ctx, const int32_t* net_ids, int32_t n, int32_t* status_out);

/* How much of the arena is in use (inet_arena_usage). */
typedef struct inet_arena_usage_t {
  uint64_t agent_slots;       /* agent bump pointer: slots handed out at least once since the
                                 last reset; each slot below it is live or waits in a free ring */
  uint64_t name_slots;        /* name bump pointer, likewise */
  uint64_t free_agent_slots;  /* agent slots waiting in the free ring */
  uint64_t free_name_slots;   /* name slots waiting in the free ring */
  int64_t live_agents;        /* agents alive in all nets */
  uint32_t nets;              /* net ids in use */
  uint32_t free_net_ids;      /* ids released by inet_free_nets, not reused yet */
} inet_arena_usage_t;

/* Fills *out.  Loaded nets are uploaded and placed first, so the figures
 * include them.  Between reductions every free slot is in a ring, so
 * agent_slots - free_agent_slots slots are held by nets (likewise for
 * names).  The paper has no counterpart: it lets a request loop see that
 * freed memory is reused. */
inet_status inet_arena_usage(inet_ctx* ctx, inet_arena_usage_t* out);

/* Per-net counters; live and residual agents come from the readback
 * snapshot. */
inet_status inet_net_info(inet_ctx* ctx, int32_t net_id, inet_net_stats* out);

/* Copies the per-step trace of the last inet_reduce() with opts->trace set:
 * frontier size and live agents after each step.  *n_out gets the number of
 * steps recorded (at most cap are copied; either array may be NULL). */
inet_status inet_trace(inet_ctx* ctx, int64_t* frontier, int64_t* live, size_t cap, size_t* n_out);

/* Drops every net and empties the arena (capacities and rules are kept).
 * Clears a poisoned state. */
inet_status inet_reset(inet_ctx* ctx);

/* ---- Rule-specialised asynchronous kernel ----------------------------------
 * INET_MODE_ASYNC interprets each rule's instantiation template (Sec. 2.2,
 * ->int: the agents of the right-hand side, their ports, the equations left
 * to ->com) from shared memory.  The rule set is fixed once loaded, so the
 * library also compiles, at the first asynchronous reduce of a rule set,
 * the same kernel with the templates as constants (NVRTC, with the device
 * headers the library was built from; a few seconds, then kept for the
 * process and cached on disk in $INET_JIT_CACHE, by default jit-cache beside
 * the library).  A warp whose lanes all reduce one rule whose right-hand side
 * has at most two agents (the rules that carry chains) then runs that rule's
 * own code, with no template reads and no scans; other warps run the general
 * code.  Results are identical either way.  When NVRTC is missing or fails
 * the general kernel runs and inet_jit_info says why.  On by default; the
 * environment variable INET_JIT=0 turns it off for new contexts, and
 * INET_NVRTC_LIB names the NVRTC library to open instead of searching. */
typedef struct inet_jit_info_t {
  int32_t enabled;     /* 1: asynchronous reduces use the specialised kernel */
  int32_t state;       /* for the loaded rules: 0 not built yet, 1 built, -1 failed */
  int32_t source;      /* the last build: 1 compiled, 2 on-disk cache, 3 already in this process */
  int32_t pad;
  double compile_ms;   /* NVRTC time of the last build (0 when from a cache) */
  uint64_t launches;   /* asynchronous launches of this context that used it */
  char msg[256];       /* why the last build failed ("" otherwise) */
} inet_jit_info_t;

/* Turns the specialised kernel on (1) or off (0) for this context. */
inet_status inet_set_jit(inet_ctx* ctx, int32_t enable);
/* State of the specialised kernel of this context. */
inet_status inet_jit_info(const inet_ctx* ctx, inet_jit_info_t* out);
/* Builds the specialised kernel for the loaded rules now (owner tracking:
 * track = 1; -1: the instantiation this context launches) instead of at the
 * first asynchronous reduce.  On a host-only
 * context (device < 0) it only compiles (or finds the cached cubin), which
 * needs no GPU.  INET_ERR_STATE without rules, INET_ERR_CUDA (message in
 * inet_last_error) when the build fails. */
inet_status inet_jit_build(inet_ctx* ctx, int32_t track);

/* Microbenchmark of the linker's primitive (->com, Sec. 2.2): random 32-bit
 * atomic exchanges that return the old value, over an array of n_slots
 * slots (allocated and freed here) on CUDA device `device`; about n_ops
 * exchanges are timed after one warm-up launch.  *exch_per_s_out gets
 * exchanges per second.  It gives the atomic-throughput bound on the
 * interaction rate beside the HBM roofline. */
inet_status inet_bench_exch(int device, uint64_t n_slots, uint64_t n_ops, double* exch_per_s_out);

/* Microbenchmark of the latency floor of a chain of interactions: one
 * thread follows a random cycle through an array of n_slots 16-byte records
 * (allocated and freed here; 16 MB at 2^20 slots stays in L2) for `hops`
 * dependent steps, each step one of
 *   variant 0: the load of the next record (a chain of interactions whose
 *              next pair is known from the record just read, as Add(y, r) =
 *              S(x) meets the S agent x next);
 *   variant 1: an atomic exchange whose result names the next record, then
 *              that record's load (->com finding an agent waiting in a name
 *              slot, Sec. 2.2);
 *   variant 2: a record store, a fence, the exchange and the load (one level
 *              of a chain of second arrivals: the new agent, its publication,
 *              ->com, and the found agent's record).
 * *ns_per_hop_out gets nanoseconds per step.  hops <= n_slots - 1 (the
 * exchange variants consume one slot per step).  The paper has no
 * counterpart: it gives the hardware floor that the measured time per level
 * of a batch is compared with. */
inet_status inet_bench_chase(int device, uint64_t n_slots, uint64_t hops, int32_t variant, double* ns_per_hop_out);

/* ---- Control: the paper's communication phase ------------------------------
 * Sec. 3.5 resolves ->com by sorting every name-headed equation x = t by the
 * name and folding adjacent equations x = t, x = s into s = t (reduce_by_key),
 * one ->com per name and pass, the whole loop repeated until nothing merges
 * (Sec. 3.6).  inet_control_link runs that method (method 1: stable radix
 * sort + merge passes, own kernels) or this evaluator's linker (method 0: one
 * launch of atomic exchanges on name slots, chains chased) on the same
 * equations, for comparison on one GPU.  Not on the reduction path.
 *   eq[i]      = t | (uint64_t)u << 32, term words (agent or name); every
 *                name index < n_vars occurs at most twice (linearity)
 *   pairs_out  = 2 * cap agent indices: the active pairs found (any order)
 *   *passes_out = merge passes (method 1) or 1; *ms_out = device time of the
 *                linking (host reads between passes included for method 1)
 * Device memory is allocated and freed inside.  INET_ERR_LINEARITY when a
 * name occurs more than twice or a chain does not end. */
inet_status inet_control_link(int device, const uint64_t* eq, uint64_t n, uint32_t n_vars, int32_t method,
                              uint32_t* pairs_out, uint64_t cap, uint64_t* n_pairs_out, uint32_t* passes_out,
                              double* ms_out);

/* reduce_by_key with equality of adjacent values and + as the fold, the
 * primitive Sec. 3.5 builds on (its example: 2 0 3 3 3 7 5 5 -> 2 0 9 7 10).
 * `out` holds at least n values; *n_out gets the number of runs. */
inet_status inet_control_segsum(int device, const int32_t* in, uint64_t n, int32_t* out, uint64_t* n_out);

/* ---- Reduction without any allocation ------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate on their request path: a serving process whose allocator
 * reserved all GPU memory at start-up, or code with a hard latency budget
 * where cudaMalloc (and the synchronisation it implies) is not allowed.
 *
 * It reduces net `net_id` of a HOST-ONLY context (inet_create with device
 * < 0, rules and nets loaded there ahead of time; that set-up may allocate)
 * on CUDA device `device`, on `stream` (NULL: the legacy default stream),
 * and calls no cudaMalloc, cudaFree or other allocating routine:
 *   - `arena` is caller-owned device memory, 256-byte aligned, of at least
 *     round_up(16 * max_agents, 256) + 4 * max_vars bytes: agent records
 *     first, then name slots.  Every net of the context is copied there at
 *     the start of the call (agent ids from 0); on return it holds the
 *     normal form.
 *   - The frontier, the free-slot rings, the control block, the rule tables
 *     and the per-net counters live in one fixed array of
 *     INET_FIXED_SCRATCH_BYTES in device memory, which every GPU that loads
 *     the library holds until the process exits.  Hence the limits:
 *     max_agents and max_vars <= 1048576, at most 262144 active pairs in a
 *     step, at most 4096 nets in the context.  Larger sizes are rejected
 *     with INET_ERR_INVALID_ARG before any device work.
 *   - The first call on a device looks the array's address up on that
 *     device (cudaGetSymbolAddress) and keeps it for the process; make that
 *     first call before any stream capture begins, and do not reset the
 *     device (cudaDeviceReset) between calls, which would leave the kept
 *     address stale.
 *   - All calls on a device share the array, and each call clears what must
 *     start at zero.  Calls that overlap on the GPU race: issue them one at
 *     a time (the call returns only after its device work is finished).
 *   - The numeral is read back by one device thread walking it (there is
 *     no room in the fixed array for the list ranking of
 *     inet_readback_nats): one dependent load per S agent and name slot on
 *     its path, about a microsecond each, so a numeral of a million
 *     elements costs about a second.
 *   - The context's nets must have been staged from slot 0 (every load of
 *     a host-only context is); otherwise INET_ERR_STATE.
 * On success *value_out is k when the net's interface is the numeral S^k(Z)
 * (otherwise INET_ERR_INVALID_ARG) and *interactions_out (may be NULL) the
 * number of interactions. */
#define INET_FIXED_SCRATCH_BYTES 12647680u
inet_status inet_reduce_into(inet_ctx* host_ctx, int32_t net_id, void* arena, size_t arena_bytes,
                             uint64_t max_agents, uint64_t max_vars, int device, void* stream,
                             uint64_t* value_out, uint64_t* interactions_out);

/* Message of the last failed call on this context (never NULL). */
const char* inet_last_error(const inet_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* INET_H */
