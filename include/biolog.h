/*
 * biolog.h -- C ABI of the GB300 candidate-search library for the biomass
 * logistics problem of M. G. Plessen, "GPU-accelerated Logistics Optimisation
 * for Biomass Production with Multiple Simultaneous Harvesters Tours, Fields
 * and Plants" (arXiv 1909.10286).
 *
 * The library runs Algorithm 1 (Sec. 2.5) on one GPU: every iteration draws n
 * candidate plans with counter-based Philox moves (Step 8), scores each one
 * exactly -- Eq. 2 demand check, Fig. 1 path-length cost (Sec. 2.2), HU and SU
 * assignment by local minimisation (Sec. 2.5, Eq. 6, Algorithm 2), and the
 * completion-time gate -- then takes the argmin and updates the best plan
 * (Steps 13-16). The whole iteration stays on the device.
 *
 * Conventions for every entry point:
 *   - plain C types only; no exceptions cross the ABI;
 *   - the return value is BL_OK (0) or a negative BL_E* code, and the message
 *     of the last failure is available from bl_last_error(handle) (or
 *     bl_global_error() when no handle exists yet);
 *   - "host" pointers are CPU memory, "device" pointers are CUDA global memory
 *     of the current device;
 *   - calls on one handle are not thread-safe; different handles are
 *     independent.
 *
 * Node numbering: node 0 is the HQ, nodes 1..B the BPs, nodes B+1..B+F the
 * fields. BP ids and field ids below are 0-based (BP b is node 1+b).
 *
 * Plan encoding (Sec. 2.4, decision variables (i)-(iv)), all int16:
 *   bp_order[B]    BP ids, tours concatenated in tour order, each tour's BPs
 *                  in visiting order;
 *   tour_cnt[T]    BPs per tour (0 = inactive tour);
 *   field_order[F] field ids grouped by BP id (BP 0's fields first), each
 *                  group in harvest order;
 *   bp_cnt[B]      fields per BP, indexed by BP id.
 * Decision variables (v)-(vi), the HUs and SUs per tour, are derived by the
 * scorer's local minimisation and reported by bl_best_plan.
 */
#ifndef BIOLOG_H
#define BIOLOG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BL_OK 0
#define BL_EINVAL (-1)               /* bad argument, size or value */
#define BL_EINFEASIBLE_INSTANCE (-2) /* total supply below total demand (Eq. 2 cannot hold) */
#define BL_ETOO_LARGE (-3)           /* beyond the int16 encoding or the kernel limits below */
#define BL_ECUDA (-4)                /* a CUDA runtime call failed */
#define BL_ETIMEOUT (-5)             /* a bounded device-side wait gave up */
#define BL_ESTATE (-6)               /* call out of order (e.g. a freed or failed handle) */

/* Limits of this build: tours <= 16, HUs <= 64, SUs <= 128, fields <= 32767,
   BPs <= 1024. The FP32 supplies, HU rates, SU capacities and SU fill areas
   of one instance must each span at most 2^(52 - 24 - log2(n+1)) in ratio so
   that their sums are exact in 64-bit fixed point and in FP64. */
#define BL_MAX_TOURS 16
#define BL_MAX_HU 64
#define BL_MAX_SU 128
#define BL_MAX_FIELDS 32767
#define BL_MAX_BPS 1024

/* One problem instance (Sec. 2.1, Table 1). Caller-owned, host memory,
   read only during bl_plan_init*, which copies what it needs. */
typedef struct bl_instance {
    int32_t n_fields, n_bps, n_tours, n_hu, n_su;
    const float *xy;           /* host, (1+B+F) x 2, km */
    const float *dist;         /* host, optional (1+B+F)^2 row-major km; NULL = straight
                                  lines from xy (Sec. 3.1), computed in FP64, stored FP32 */
    const float *area_ha;      /* host, F: field sizes h_f */
    const float *supply_t;     /* host, F: expected supplies (Eq. 3), > 0 */
    const float *demand_t;     /* host, B: minimum demands d_b (Eq. 2), > 0 */
    const float *hu_rate_ha_h; /* host, H: in-field working rate of each HU, > 0 */
    float hu_speed_kmh;        /* road speed of HUs */
    const float *su_cap_t;     /* host, S: loading capacity of each SU */
    const float *su_fill_ha;   /* host, S: hectares harvested while the SU fills */
    const float *su_speed_kmh; /* host, S: road speed of each SU */
} bl_instance;

/* Search parameters. */
typedef struct bl_params {
    float eps;               /* exploration rule, Eq. 5, in [0, 1] */
    float p_swap;            /* probability that a move is a swap of two same-type
                                vertices instead of a reinsert (0 = the paper's Step 8) */
    uint64_t seed;           /* Philox key */
    uint32_t inst_idx;       /* Philox counter word 2 of instance 0 (instance k uses inst_idx+k) */
    int32_t n_cand;          /* candidates per iteration per instance, >= 1 */
    int32_t fix_field_bp;    /* 1 = a removed field returns to its own BP (Sec. 2.6) */
    int32_t fix_resources;   /* 1 = keep the initial HU/SU dealing, no local minimisation (Case 2) */
    int32_t gate;            /* completion-time gate: 0 off, 1 discard Tmax > Tmax*,
                                2 discard Tmax >= Tmax* (literal reading) */
    int32_t block_threads;   /* 0 = autotuned; else threads per block of the scorer */
    int32_t blocks_per_sm;   /* 0 = autotuned; else resident blocks per SM to size the grid */
    int32_t tile;            /* 0 = autotuned; else candidates per work item */
    int32_t log_capacity;    /* iterations kept in the per-instance log (0 = 4096) */
    int32_t lanes_per_cand;  /* 0 or 1: one thread scores a candidate; 4, 8, 16 or 32: a group
                                of that many lanes of a warp scores it together, lane g holding
                                tour g (>= the largest tour count; 4 or 8 for <= 4 tours, 8 or
                                16 for <= 6, 16 or 32 above; else BL_EINVAL). Same results. */
    int32_t k_moves;         /* 0 or 1: one remove-and-reinsert move per candidate (Step 8);
                                2 or 3: Step 8 repeated, move j drawn on the plan the first j
                                moves made (Philox counter word 3 = 0, then j + 1); needs
                                lanes_per_cand <= 1 and no learned proposals (else BL_EINVAL) */
    uint32_t cand_offset;    /* candidate numbers (Philox counter word 0) of this handle:
                                cand_offset .. cand_offset + n_cand - 1 (0 = the whole range);
                                one slice of a split iteration (bl_search_score_slice) */
    void *workspace;         /* device, optional: caller-owned buffer of
                                bl_workspace_bytes() bytes, 256-byte aligned; NULL = the
                                library allocates and frees its own */
    size_t workspace_bytes;
} bl_params;

/* Report of one plan, filled by bl_best_plan. Caller-owned host buffers sized
   from the instance; any array pointer may be NULL. */
typedef struct bl_plan {
    int16_t *bp_order;     /* B */
    int16_t *tour_cnt;     /* T */
    int16_t *field_order;  /* F */
    int16_t *bp_cnt;       /* B */
    int16_t *hu_tour;      /* H: tour of each HU (-1 = none) */
    int16_t *su_tour;      /* S: tour of each SU (-1 = none) */
    float *tour_cost_km;   /* T: per-tour cost C(g) (Table 2 row "C") */
    float *tour_tcompl_h;  /* T: completion times (Table 2 row "T_compl") */
    float *tour_twait_h;   /* T: average HU waiting times (Table 2 row "T_wait") */
    int16_t *tour_n_hu;    /* T */
    int16_t *tour_n_su;    /* T */
    float cost_km;         /* C* (+inf if no feasible plan has been found) */
    float tmax_h;          /* Tmax* */
    uint32_t iter;         /* iterations run so far */
} bl_plan;

/* Search state of one instance (checkpoint / resume, host-driven loops).
   Host buffers, caller-owned, sized from the instance. */
typedef struct bl_state {
    int16_t *xold_bp_order, *xold_tour_cnt, *xold_field_order, *xold_bp_cnt;
    int16_t *xbest_bp_order, *xbest_tour_cnt, *xbest_field_order, *xbest_bp_cnt;
    float cstar, tmaxstar;
    uint32_t iter;
} bl_state;

typedef struct bl_handle bl_handle;
typedef struct bl_mlp bl_mlp;   /* learned move ranker, see bl_mlp_create */

/* Bytes of device workspace bl_plan_init_batch needs for these instances and
   parameters (to pass a caller-owned buffer in bl_params.workspace). */
int bl_workspace_bytes(const bl_instance *insts, int32_t n_inst, const bl_params *params, size_t *bytes);

/* Algorithm 1, Steps 1-4 (Sec. 2.5): validate and copy the instance, build the
   initial plan (nearest-neighbour BP chain cut into tours, fields to the
   closest BP still short of its demand, nearest-neighbour field order from
   the HQ), score it on the GPU (C*, Tmax*), set x_old = x* = x_init, and
   prepare the kernels. `cuda_stream` is a cudaStream_t (NULL = default
   stream); every later call on the handle is ordered on it. On success *out
   owns all device memory (or uses params->workspace). Errors: BL_EINVAL,
   BL_EINFEASIBLE_INSTANCE, BL_ETOO_LARGE, BL_ECUDA; *out is NULL then. */
int bl_plan_init(const bl_instance *inst, const bl_params *params, void *cuda_stream, bl_handle **out);

/* Same for n_inst independent instances of uneven size searched together:
   one persistent launch per iteration covers all of them (work items ordered
   largest instance first), each with its own x_old, x*, C*, Tmax* and
   Philox counter word inst_idx+k. The launch shape (threads per block, tour
   and unit capacity, distances in shared memory or read through L2) is the
   one the largest instance needs, for every instance of the handle. Small
   instances of an uneven batch run faster on a handle of their own: e.g.
   those with at most 4 tours and 32 HUs and SUs take the 256-thread shape.
   Handles on one stream run one after another. */
int bl_plan_init_batch(const bl_instance *insts, int32_t n_inst, const bl_params *params, void *cuda_stream,
                       bl_handle **out);

/* Algorithm 1, Steps 5-16, n_iters times, asynchronously on the handle's
   stream: per iteration the eps rule (Eq. 5), n_cand Philox moves and exact
   scores per instance, the argmin (ties to the lowest index) and the update
   of x_old, x*, C*, Tmax*. Launches are replayed from a CUDA graph. Device
   errors (BL_ETIMEOUT) surface at the next synchronising call. */
int bl_search_step(bl_handle *h, int32_t n_iters);

/* One iteration split over several handles -- on several GPUs, one process
   each (Sec. 2.5: the candidates of an iteration are independent). Every
   handle holds the same instance, parameters and state, and scores its own
   slice of the candidate numbers (params.cand_offset, params.n_cand).
   bl_search_score_slice runs Steps 9-12 on the slice and writes the slice's
   argmin key ((cost bits << 32) | i, the same order as bl_get_log's i*) to
   *d_key (device memory, caller-owned), without updating anything. The
   caller reduces the slices' keys to their minimum (an all-reduce-min of
   one 64-bit integer per iteration) and passes the result to
   bl_search_apply on every handle, which replays move i* on the handle's own
   copy of the base plan, recomputes Tmax_{i*} and runs Steps 13-16, so all
   handles keep identical states without exchanging plans. Both are
   asynchronous on the handle's stream; one instance per handle (BL_EINVAL
   otherwise). A key that does not score as candidate i* of this iteration
   makes the handle's next synchronising call return BL_ESTATE. */
int bl_search_score_slice(bl_handle *h, uint64_t *d_key);
int bl_search_apply(bl_handle *h, const uint64_t *d_key);

/* Inspection of the search kernel itself (Steps 9-12 of Algorithm 1, the
   three evaluation steps of Sec. 2.5): one iteration exactly as
   bl_search_step runs it -- the same kernel, launch shape and work items,
   with the argmin and the update of x_old, x*, C*, Tmax* -- that also writes
   each candidate's result where the kernel decides it: d_out[2 (k stride +
   i)] = C_i and d_out[2 (k stride + i) + 1] = Tmax_i for candidate i of
   instance k. An infeasible candidate (Eq. 2) gets {+inf, +inf}; one the
   completion-time gate discards {+inf, Tmax_i}; the rest {C_i, Tmax_i}.
   d_out is device memory owned by the caller, at least 8 n_inst stride
   bytes; stride >= the candidates per iteration. Asynchronous on the
   handle's stream; not for timing (the search never writes d_out).
   Errors: BL_EINVAL, BL_ESTATE, BL_ECUDA. */
int bl_search_step_inspect(bl_handle *h, float *d_out, int32_t stride);

/* Synchronise and report instance `inst`'s best plan x*, re-scored once for
   the per-tour table (Table 2's rows). */
int bl_best_plan(bl_handle *h, int32_t inst, bl_plan *out);

/* Synchronise and copy instance `inst`'s search state to host buffers. */
int bl_get_state(bl_handle *h, int32_t inst, bl_state *out);

/* Replace instance `inst`'s search state (resume from a checkpoint). The plans
   are validated; the copy is ordered on the handle's stream. */
int bl_set_state(bl_handle *h, int32_t inst, const bl_state *in);

/* The same for every instance of the handle at once, in one host<->device
   transfer each way through a pinned staging buffer the library allocates on
   first use (a host-driven loop's checkpoint of a batch). out / in point to
   n_inst states. bl_get_states synchronises; bl_set_states validates every
   plan first (nothing is written if one is invalid), copies the caller's
   buffers before it returns, and is asynchronous on the handle's stream.
   Errors as bl_get_state / bl_set_state, and BL_ETOO_LARGE if the packed
   states exceed the library's 8 MiB inspection scratch. */
int bl_get_states(bl_handle *h, bl_state *out);
int bl_set_states(bl_handle *h, const bl_state *in);

/* Per-iteration log of instance `inst` for iterations [first, first+n) that
   are still in the ring buffer: i*, C_{i*}, whether the base was x* (Eq. 5),
   C* after the update, and the indicator of Fig. 3 (0 no improvement,
   1 improved by a field move, 2 by a BP move). Host outputs, may be NULL. */
int bl_get_log(bl_handle *h, int32_t inst, uint32_t first, int32_t n, int32_t *istar, float *c_istar,
               int8_t *use_best, float *cstar, int8_t *indicator);

/* Inspection: score candidates i0..i0+n-1 of iteration `iter` drawn from
   base x* (use_best = 1) or x_old (0) of instance `inst`, without updating
   anything; tmax_star is the gate's reference (pass the state's Tmax*).
   Host outputs (any may be NULL): cost[n], tmax[n] (FP32; +inf when
   infeasible), moves[n x 4 k] (k = params.k_moves records {kind, vertex,
   a, b} per candidate, move j relative to the plan after the first j:
   kind 0 field reinsert (a = BP, b = slot), 1 BP reinsert (a = tour, b =
   slot), 2 field swap (a = other field), 3 BP swap (a = other BP)),
   n_hu[n x T], n_su[n x T],
   and the HU and SU assignments the two local minimisations of Sec. 2.5
   reach, hu_tour[n x H] and su_tour[n x S] (tour of each unit by id, -1
   when unassigned: infeasible candidates). */
int bl_score_candidates(bl_handle *h, int32_t inst, int32_t use_best, uint32_t iter, float tmax_star, int32_t i0,
                        int32_t n, float *cost, float *tmax, int16_t *moves, int16_t *n_hu, int16_t *n_su,
                        int16_t *hu_tour, int16_t *su_tour);

/* Inspection: the decoded candidate plans (Step 8 applied to the base) for
   candidate indices idx[0..n-1]; plans is a host buffer of n x (2B+T+F)
   int16, each row bp_order | tour_cnt | field_order | bp_cnt. */
int bl_decode_candidates(bl_handle *h, int32_t inst, int32_t use_best, uint32_t iter, const int32_t *idx, int32_t n,
                         int16_t *plans);

/* Argmin without allocation (the paper has no counterpart: this is a library
   convenience). Scores candidates i0..i0+n-1 of iteration `iter`, drawn from
   base x* (use_best = 1) or x_old (0) of instance `inst`, and writes the
   smallest key ((cost bits << 32) | i, as in bl_get_log's i*) to *d_key and
   the winner's maximum completion time to *d_tmax. d_key and d_tmax are
   device pointers owned by the caller; the call is asynchronous on the
   handle's stream. It is meant for callers that must not allocate device
   memory where they call it -- for example a latency-critical loop in which
   the device synchronisation of cudaMalloc/cudaFree is unacceptable, or a
   process whose device memory is entirely owned by another allocator.
   Nothing is allocated: the kernel's scratch (one partial result per block,
   at most 1024 blocks, and a completion counter; 16,640 bytes) is a static
   array in the library's device code that every GPU loading the library
   holds until the process exits. The current device must be the one the
   handle was created on (BL_EINVAL otherwise). The first call on a handle
   looks up that array's device address, so make it before any stream
   capture. All calls on a device share the array: the counter is cleared
   before each launch, and calls that overlap on the GPU (e.g. on two
   streams) race and must not be issued. If a block's bounded staging wait
   gives up, the outputs are still written but hold no result (*d_key =
   ~0, *d_tmax = NaN) and the handle's next synchronising call reports
   BL_ETIMEOUT. Errors: BL_ETOO_LARGE when n < 1, n > BL_NOALLOC_MAX_CAND,
   i0 < 0 or i0 + n > INT32_MAX (checked first, for any handle, NULL
   included), then BL_EINVAL, BL_ESTATE, BL_ECUDA. */
#define BL_NOALLOC_MAX_CAND (1 << 28)
int bl_argmin_noalloc(bl_handle *h, int32_t inst, int32_t use_best, uint32_t iter, float tmax_star, int32_t i0,
                      int32_t n, uint64_t *d_key, float *d_tmax);

/* ---- Learned move ranking (an extension; the paper draws moves uniformly) ----
   A small MLP in -> H -> H -> H -> 1 with ReLU scores candidate moves from
   per-move features (bl_features); its GEMMs run on the tensor cores in BF16
   with FP32 accumulation (tcgen05, accumulators in tensor memory); master
   weights are FP32; training minimises the mean squared error with Adam. All
   pointers named d_* are device memory owned by the caller; calls are
   asynchronous on the MLP's stream unless they return host values. */

/* Create an MLP with He-uniform initial weights drawn from `seed`. in_dim in
   [1, 256], hidden a multiple of 16 in [16, 256], max_batch the largest M of
   later calls. Owns its device memory. */
int bl_mlp_create(int32_t in_dim, int32_t hidden, int32_t max_batch, uint64_t seed, void *cuda_stream, bl_mlp **out);

/* y[M] = MLP(x[M x in_dim]), x BF16 row-major, asynchronously on the MLP's
   stream. When hidden is a multiple of 32 the three layers and the head run
   as one fused tensor-core kernel (activations stay on chip, rounded to BF16
   between layers like the layer-by-layer pass) and M is not bounded by
   max_batch; otherwise M <= max_batch. A bounded wait that gave up inside a
   kernel sets the MLP's error flag, reported as BL_ETIMEOUT by the next
   bl_mlp_grads / bl_mlp_train_step. */
int bl_mlp_forward(bl_mlp *m, const uint16_t *d_x, int32_t M, float *d_y);

/* Forward and backward pass of the loss mean_i (y_i - t_i)^2 without
   updating; the gradients are then readable with bl_mlp_get(which = 1).
   Synchronises; *h_loss (may be NULL) receives the loss. */
int bl_mlp_grads(bl_mlp *m, const uint16_t *d_x, const float *d_target, int32_t M, float *h_loss);

/* One Adam step (beta 0.9 / 0.999) with learning rate lr on that loss. */
int bl_mlp_train_step(bl_mlp *m, const uint16_t *d_x, const float *d_target, int32_t M, float lr, float *h_loss);

/* bl_mlp_train_step on a minibatch of `batch` rows (<= max_batch) drawn
   uniformly with replacement from the n_rows rows of d_X [n_rows x in_dim]
   (BF16) and d_T [n_rows], gathered in the library: row r of the minibatch of
   Adam step t is floor(z n_rows / 2^64) with z = SplitMix64(seed + (t batch
   + r) * 0x9E3779B97F4A7C15) (mod 2^64), so a run is reproducible from the
   seed. */
int bl_mlp_train_step_sampled(bl_mlp *m, const uint16_t *d_X, const float *d_T, int64_t n_rows, int32_t batch,
                              uint64_t seed, float lr, float *h_loss);

/* Copy parameters (which = 0) or the last gradients (which = 1) to host
   buffers: w1 [H x in], b1 [H], w2 [H x H], b2 [H], w3 [H x H], b3 [H],
   w4 [H], b4 [1]; NULL pointers are skipped. Synchronises. */
int bl_mlp_get(bl_mlp *m, int32_t which, float *w1, float *b1, float *w2, float *b2, float *w3, float *b3, float *w4,
               float *b4);

/* Replace the parameters (host buffers, same layout). */
int bl_mlp_set(bl_mlp *m, const float *w1, const float *b1, const float *w2, const float *b2, const float *w3,
               const float *b3, const float *w4, const float *b4);

int bl_mlp_free(bl_mlp *m);
const char *bl_mlp_last_error(const bl_mlp *m);

/* The tensor-core GEMM itself: C[M x N] = A[M x K] B[N x K]^T (+ bias[N])
   (ReLU if relu), A and B BF16 row-major, C as FP32 (d_cf) and/or BF16
   (d_cb); 1 <= N <= 256. *d_err becomes nonzero if a bounded wait on the
   tensor cores gave up. */
int bl_gemm_bf16(const uint16_t *d_a, const uint16_t *d_b, const float *d_bias, float *d_cf, uint16_t *d_cb, int32_t M,
                 int32_t N, int32_t K, int32_t relu, uint32_t *d_err, void *cuda_stream);

/* Features of candidates i0..i0+n-1 of iteration `iter` (base x* if use_best
   = 1, x_old if 0; use_best = -1 with iter = 0xFFFFFFFF takes the state's
   current iteration and Eq. 5 choice): d_feat receives n x 64 BF16 values per
   candidate (the move's kind, the distances around its removal and insertion
   slots and the resulting HU-route change, field-to-BP distances, supply,
   area, demand slack, completion-time slack of the tours involved, positions,
   coordinates), normalised per instance. *d_base_cost (may be NULL) receives
   the base plan's cost. Asynchronous on the handle's stream. */
int bl_features(bl_handle *h, int32_t inst, int32_t use_best, uint32_t iter, int32_t i0, int32_t n, uint16_t *d_feat,
                float *d_base_cost);

/* Algorithm 1 with learned proposals, n_iters times, for every instance of
   the handle (an extension; the paper draws moves uniformly): per iteration
   and instance the first `pool` Philox candidates are featurised and ranked
   by `mlp` (predicted cost change, lower is better) in one pass over all
   instances; about the n_keep best (threshold from a sample of 4096
   predictions) plus a fraction rand_frac of the others, drawn uniformly by
   Philox, are scored exactly by the same kernel as bl_search_step, which takes
   each instance's argmin and updates its state. Every accepted plan is thus
   judged by the exact score. pool <= n_cand of the handle; the MLP must have
   been created on the handle's stream, and pool x instances rows must be
   within its batch limit (see bl_mlp_forward). The first call allocates the
   pool buffers (pool x instances x 136 bytes). Asynchronous on the stream. */
int bl_search_step_learned(bl_handle *h, bl_mlp *mlp, int32_t n_iters, int32_t pool, int32_t n_keep, float rand_frac);

/* Self-test of the bounded device waits (plumbing; no counterpart in the
   paper). Every wait of the library's kernels on a barrier or a bulk copy
   gives up after a wall-clock limit, sets the handle's error flag and returns,
   so that a lost completion turns into BL_ETIMEOUT on the host instead of a
   hung GPU. This call runs one thread on `stream` that waits, with the limit
   limit_ns (0 < limit_ns <= 10 s), on a barrier that nothing completes (no
   copy or arrival is pending on it), and reports what happened: BL_ETIMEOUT
   (expected: the wait gave up) with *elapsed_ns (may be NULL) the time it
   waited, BL_OK if the wait unexpectedly completed, BL_EINVAL, BL_ECUDA.
   Synchronises the stream; the context stays usable. */
int bl_wait_selftest(void *stream, uint64_t limit_ns, uint64_t *elapsed_ns);

/* Kernel configuration in use: threads per block, grid blocks, candidates
   per work item, the number of kernels one iteration launches, and the lanes
   that score one candidate (any pointer may be NULL). */
int bl_get_config(bl_handle *h, int32_t *block_threads, int32_t *grid_blocks, int32_t *tile,
                  int32_t *launches_per_iter, int32_t *lanes_per_cand);

/* Release everything the handle owns. */
int bl_plan_free(bl_handle *h);

/* Message of the last failure on this handle ("" if none). */
const char *bl_last_error(const bl_handle *h);

/* Message of the last failure of a call that had no handle to report to. */
const char *bl_global_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BIOLOG_H */
