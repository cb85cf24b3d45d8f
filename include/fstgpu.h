/*
 * fstgpu.h -- C ABI of libfstgpu.so: Viterbi and forward-backward decoding
 * with large, sparse, epsilon-free weighted finite-state transducers on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Argueta & Chiang, "Decoding with Finite-State Transducers on
 * GPUs", EACL 2017.  An FST is M = (Q, Sigma, s, F, delta) with output
 * labels on the arcs (Sec. 3); the weight of a string w = w_1..w_n is
 * weight(w) = s^T (prod_t delta[w_t]) f (Eq. 1).  Viterbi evaluates Eq. 1 in
 * the (max, *) pair semiring of Sec. 3 (best path and its arcs; Alg. 1,
 * Sec. 5.1); forward-backward evaluates it in the (+, *) semiring and
 * returns expected arc counts (Alg. 2, Sec. 5.2).  The only loop that is
 * parallel is the one over the arcs of the slice delta[w_t] (Sec. 5).
 *
 * Conventions used by every entry point:
 *   - Weights are natural-log weights theta = log p (weight_kind
 *     FST_WEIGHT_LOG) or costs w = -log p (FST_WEIGHT_COST).  Scores and
 *     log Z are always returned as log-weights (theta domain).  -inf (cost
 *     +inf) means "absent"; NaN and theta = +inf are rejected.  A negative
 *     zero weight is stored as +0.
 *   - Arc ids are the caller's array order (0..num_arcs-1).
 *   - Ties in Viterbi go to the lowest arc id into each state at each step,
 *     and to the lowest state id at the final step (the paper's packed
 *     atomicMax of Sec. 5.1 would pick the highest id; this library fixes
 *     the lowest so that results are reproducible and checkable).
 *   - Viterbi runs in float32 with one rounded addition per candidate, so
 *     its score and path are bit-identical to a sequential float32 Viterbi.
 *     Forward-backward forms each arc's term from its float32 weight and
 *     the float64 value of its source (forward) or destination (backward),
 *     shifted by a float64 per-step normaliser folded into log Z; each
 *     state's log-sum takes the exact maximum and adds exp(term - maximum)
 *     in 2^-40 fixed point, so the sums do not depend on their order.
 *   - Status codes: 0 = FST_OK; every failure returns a nonzero code and
 *     sets a thread-local message readable with fst_last_error().
 *   - All entry points are host functions.  "Host" pointers are ordinary
 *     CPU memory; "device" pointers are CUDA device memory of the device
 *     that was current when the FST was created.
 *   - Environment: FSTGPU_CHAIN=0 launches the per-position kernels
 *     without programmatic dependent launch (by default a single-part plan
 *     and the single-string kernels chain each position's launch to the
 *     previous one; FSTGPU_CHAIN_PARTS=k chains the parts of plans of at
 *     most k parts, default 1: parts run unchained); FSTGPU_PART_THREADS=0
 *     builds and issues the parts of a plan from the calling thread (by
 *     default one host thread per part);
 *     FSTGPU_TUNE_CACHE names the autotuner's cache file.
 */
#ifndef FSTGPU_H_
#define FSTGPU_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FST_API __attribute__((visibility("default")))
#else
#define FST_API
#endif

#define FST_OK 0
#define FST_ERR_INVALID_ARG 1  /* a size, id, label or weight out of range */
#define FST_ERR_NO_PATH 2      /* the string has no accepting path */
#define FST_ERR_OOM 3          /* device allocation failed */
#define FST_ERR_CUDA 4         /* a CUDA runtime call failed */
#define FST_ERR_TIMEOUT 5      /* a bounded device wait expired */
#define FST_ERR_UNSUPPORTED 6  /* sizes beyond this library's limits */
#define FST_ERR_STATE 7        /* call out of order (e.g. backward before forward) */

#define FST_WEIGHT_LOG 0
#define FST_WEIGHT_COST 1

#define FST_FLAG_DEVICE_PTRS 1 /* fst_create / fst_set_weights: inputs are device pointers */

typedef struct fst_s fst_t;
typedef struct fst_plan_s fst_plan_t;

/* Build an FST on the current CUDA device (Sec. 3 tuple; Sec. 4 and Fig. 2
 * arc arrays S, T, O, P plus input labels; the start vector s and final
 * vector f of Sec. 3, generalised to per-state log-weights).
 *   num_states  Q >= 1.   num_arcs A >= 0 (A < 2^31).   num_isyms m >= 1.
 *   src, dst    [A] states in [0, Q).      ilabel [A] in [0, m).
 *   olabel      [A] any int32 (returned by Viterbi; may be NULL = all -1).
 *   weight      [A] per weight_kind.
 *   start_weight, final_weight  [Q] per weight_kind; "absent" = -inf
 *               (FST_WEIGHT_LOG) or +inf (FST_WEIGHT_COST).
 *   flags       FST_FLAG_DEVICE_PTRS if the arrays are device pointers.
 * Every input is copied; the handle owns its device memory.  The arc store
 * is re-sorted on the device into symbol-major, destination-segmented and
 * source-segmented windows (the R offsets of Fig. 2 live on the device and
 * the host).  Synchronous.  Errors: FST_ERR_INVALID_ARG (ranges, NaN,
 * theta = +inf), FST_ERR_UNSUPPORTED (padded arc count >= 2^31),
 * FST_ERR_OOM, FST_ERR_CUDA.  On error *out is NULL. */
FST_API int fst_create(int32_t num_states, int64_t num_arcs, const int32_t* src, const int32_t* dst,
               const int32_t* ilabel, const int32_t* olabel, const float* weight,
               int32_t weight_kind, const float* start_weight, const float* final_weight,
               int32_t num_isyms, int32_t flags, fst_t** out);

/* Free an FST and everything it owns.  NULL is accepted.  Plans created on
 * it must be destroyed first. (Resource management: no counterpart in the paper.) */
FST_API int fst_destroy(fst_t* fst);

/* Sizes of a built FST (host outputs, any may be NULL): states, arcs, input
 * symbols, padded arcs of the forward layout, windows of the forward
 * layout, destination segments (sum over symbols of distinct destinations)
 * and source segments. (The structures of Sec. 4 and Fig. 2, for measurement.) */
FST_API int fst_info(const fst_t* fst, int32_t* num_states, int64_t* num_arcs, int32_t* num_isyms,
             int64_t* padded_arcs, int64_t* num_windows, int64_t* dst_segments,
             int64_t* src_segments);

/* Per input symbol a (host arrays of length num_isyms, any may be NULL):
 * |delta[a]| arcs (R[a+1]-R[a] of Fig. 2), distinct destinations D_a and
 * distinct sources U_a.  Used for relaxation counts and the bytes model. */
FST_API int fst_symbol_stats(const fst_t* fst, int64_t* arcs, int64_t* dsts, int64_t* srcs);

/* Replace every arc weight (caller arc order, [num_arcs], per weight_kind;
 * host or device per flags).  Same validation as fst_create; on error the
 * FST keeps its old weights.  Used between training steps.  Synchronous
 * with respect to the host; call it only when no plan on this FST is
 * running. The weights are the theta of Sec. 3. */
FST_API int fst_set_weights(fst_t* fst, const float* weight, int32_t weight_kind, int32_t flags);

/* Replace the start and final weights of every state ([num_states] each,
 * per weight_kind; host or device per flags; a NULL array keeps its old
 * weights).  Same validation and rules as fst_set_weights.  The states with
 * a finite start weight (the live states before the first position, Sec. 3)
 * are listed again. */
FST_API int fst_set_state_weights(fst_t* fst, const float* start_weight, const float* final_weight,
                                  int32_t weight_kind, int32_t flags);

/* Plain method, one string (the paper's design, Sec. 5: one kernel launch
 * per input position over the arcs of delta[w_t], then the backtrace of
 * Sec. 5.1 on the device).  Host pointers throughout; synchronous.
 *   ids         [n] host, symbols in [0, m); n >= 0.
 *   best_score  host float: log-weight of the best path including start and
 *               final weights; -inf if there is none.
 *   arc_path    [n] host (may be NULL if n == 0): arc id taken at each
 *               position; -1 everywhere when there is no path.
 *   olabels     [n] host or NULL: output label of each arc of the path.
 * Returns FST_OK, FST_ERR_NO_PATH (outputs filled as above), or an error. */
FST_API int fst_viterbi(fst_t* fst, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path,
                int32_t* olabels);

/* Which kernels fst_viterbi uses for one string: FST_PLAIN_FRONTIER (the
 * frontier-driven steps, the default), FST_PLAIN_SLICE (the paper's
 * slice-wide relaxation, Sec. 5.1, as fst_viterbi_slice) or FST_PLAIN_AUTO
 * (the one a calibrated cost model predicts to be faster for the string;
 * the frontier kernels until fst_autotune_plain has run).  Results are
 * identical either way.  FST_PLAIN_BLOCK runs fst_viterbi and
 * fst_forward_backward as one thread block each, the position loop inside
 * the kernel (the slice-wide relaxation of Sec. 5 with the per-state values
 * in shared memory): for FSTs of at most FST_BLOCK_MAX_STATES states, where
 * launches, not arcs, take the time (FST_ERR_UNSUPPORTED above that).
 * Viterbi results are identical; forward-backward keeps unshifted float64
 * values (log Z and posteriors agree to float64 rounding). */
#define FST_PLAIN_FRONTIER 0
#define FST_PLAIN_SLICE 1
#define FST_PLAIN_AUTO 2
#define FST_PLAIN_BLOCK 3
#define FST_BLOCK_MAX_STATES 8192
FST_API int fst_set_plain_method(fst_t* fst, int32_t method);

/* Calibrate FST_PLAIN_AUTO on sample strings (host arrays: ids, offsets
 * [B+1] as in the batch calls, B >= 1).  An FST small enough for
 * FST_PLAIN_BLOCK is first timed with it (Viterbi and forward-backward of
 * the sample); when that beats the frontier kernels under every driver,
 * FST_PLAIN_AUTO takes the one-block kernels for both calls and the rest
 * is skipped (coef then reads 0, 0, 0, 0, 0).  Otherwise each string is decoded both ways
 * and timed on the host; the frontier time is fitted as d0 + d1 n and the
 * slice time as c0 + c1 n + c2 S (S = the arcs of the string's slices), by
 * least squares (with fewer than four strings of different sizes the mean
 * times decide); the method is set to FST_PLAIN_AUTO.  Before that, the
 * driver of the frontier kernels (fst_set_plain_driver: launches, or
 * persistent passes of 1, 8, 32 or one-per-SM blocks) is chosen by timing
 * Viterbi and forward-backward on the same strings.  coef [5] or NULL
 * receives d0, d1, c0, c1, c2 (microseconds).  Synchronous. (The choice between
 * two kernels for Sec. 5's plain method.) */
FST_API int fst_autotune_plain(fst_t* fst, const int32_t* ids, const int64_t* offsets, int32_t B, double* coef);

/* Driver of the single-string frontier kernels (fst_forward_backward, and
 * fst_viterbi when it uses them): FST_DRIVER_LAUNCH (one launch per
 * position and kernel kind, the default) or FST_DRIVER_PERSISTENT (one
 * cooperative launch per pass, grid_blocks blocks, 0 = one per SM,
 * positions separated by bounded grid barriers; a barrier that times out
 * makes the call return FST_ERR_TIMEOUT).  fst_autotune_plain also picks
 * the driver and grid, by timing them on its sample.  FST_ERR_UNSUPPORTED
 * without cooperative launches or for a grid that cannot be co-resident.
 * (Sec. 5 launches one kernel per position.) */
FST_API int fst_set_plain_driver(fst_t* fst, int32_t driver, int32_t grid_blocks);

/* What the single-string calls take now, for accounting (host only, no
 * device work): *method = FST_PLAIN_BLOCK when fst_viterbi and
 * fst_forward_backward run the one-block kernels (set, or chosen by
 * fst_autotune_plain); FST_PLAIN_SLICE or FST_PLAIN_FRONTIER when set;
 * FST_PLAIN_AUTO when each fst_viterbi call chooses between those two by
 * the calibrated cost model (fst_autotune_plain's coefficients); an
 * uncalibrated FST_PLAIN_AUTO reads FST_PLAIN_FRONTIER.  *driver and
 * *grid_blocks are the frontier kernels' driver (fst_set_plain_driver).
 * Any output pointer may be NULL.  FST_ERR_INVALID_ARG for a NULL handle.
 * (Accounting: no counterpart in the paper.) */
FST_API int fst_get_plain_method(const fst_t* fst, int32_t* method, int32_t* driver, int32_t* grid_blocks);

/* The paper's relaxation, kept for comparison (Sec. 5.1): Viterbi of one
 * string where, at every position, each arc of the slice delta[w_t] is
 * relaxed by its own thread whether or not its source is live, and
 * collisions on a destination are resolved by a packed 64-bit atomicMax.
 * Arguments, results and errors as fst_viterbi (bit-identical results),
 * without output labels.  The handle keeps per-arc records of the slices
 * and an (n+1) x num_states key array for the last string; fst_destroy
 * frees them. */
FST_API int fst_viterbi_slice(fst_t* fst, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path);

/* The paper's forward-backward, kept for comparison (Sec. 5.2, Eq. 3): at
 * every position each arc of the slice adds its value into its
 * destination's forward value (backward: its source's backward value) with
 * an atomic log-add-exp -- a compare-and-swap loop over
 * log(e^a + e^b) = b + log1p(e^(a-b)), a <= b, with -inf + a = a -- on
 * float32 log-probabilities kept for every position ((n+1) x num_states
 * each, held by the handle), then log Z (float64 sum) and the per-arc
 * posteriors of Alg. 2.  Arguments, results and errors as
 * fst_forward_backward.  Its float32 values are not rescaled, so its
 * posteriors drift with the string's length (see the tests). */
FST_API int fst_forward_backward_slice(fst_t* fst, const int32_t* ids, int32_t n, double* log_z,
                                       float* arc_posteriors);

/* Order of the arcs within a slice for fst_viterbi_slice and
 * fst_forward_backward_slice (the layout study of Sec. 4):
 * FST_SLICE_BY_DESTINATION (column-major / CSC, the default) or
 * FST_SLICE_BY_SOURCE (row-major / CSR, the paper's own order). */
#define FST_SLICE_BY_DESTINATION 0
#define FST_SLICE_BY_SOURCE 1
FST_API int fst_set_slice_order(fst_t* fst, int32_t order);

/* Plain method, one string: forward-backward (Alg. 2, Sec. 5.2).  Host
 * pointers; synchronous.
 *   log_z          host double: log of the total weight of the string (Eq. 1
 *                  in the (+, *) semiring); -inf if no path.
 *   arc_posteriors [num_arcs] host float or NULL: expected count of each
 *                  arc, sum_t gamma_t(k) = d log Z / d theta_k; all zero if
 *                  there is no path.
 * Returns FST_OK, FST_ERR_NO_PATH or an error. */
FST_API int fst_forward_backward(fst_t* fst, const int32_t* ids, int32_t n, double* log_z,
                         float* arc_posteriors);

/* Batched method: Alg. 1 (Sec. 5.1) for B strings decoded together, all on
 * the device.
 *   d_ids       device int32 [N], concatenated strings.
 *   d_offsets   device int64 [B+1], d_offsets[0] = 0, non-decreasing;
 *               string b is d_ids[d_offsets[b] .. d_offsets[b+1]).
 *   d_scores    device float [B] best log-weights (-inf = no path).
 *   d_paths     device int32 [N] arc ids, aligned with d_ids (-1 = no path).
 *   d_olabels   device int32 [N] or NULL.
 *   d_status    device int32 [B] or NULL: FST_OK or FST_ERR_NO_PATH per string.
 *   stream      cudaStream_t to run on (NULL = legacy default stream).
 * Builds a plan internally (see fst_plan_create), runs it and synchronises
 * the stream before returning.  The handle keeps that plan's device storage
 * (one slot for Viterbi, one for forward-backward) and the next batch call
 * of the same kind takes it over when it is large enough, instead of
 * allocating and clearing its own; fst_destroy frees it.  Calls from
 * several host threads on one handle are safe (each slot is taken under a
 * lock; a call that finds it taken allocates its own).  The return code
 * covers argument and launch errors; per-string outcomes go to d_status
 * (FST_OK, FST_ERR_NO_PATH, or FST_ERR_OOM when the live pool overflowed). */
FST_API int fst_viterbi_batch(fst_t* fst, const int32_t* d_ids, const int64_t* d_offsets, int32_t B,
                      float* d_scores, int32_t* d_paths, int32_t* d_olabels, int32_t* d_status,
                      void* stream);

/* Batched forward-backward: Alg. 2 (Sec. 5.2) for every string.  Arguments
 * as fst_viterbi_batch, plus
 *   d_weights   device float [B] or NULL (all 1): per-string factor g_b;
 *   d_logz      device double [B];
 *   d_counts    device float [num_arcs] or NULL: sum_b g_b * count_b(k),
 *               the gradient of sum_b g_b log Z_b with respect to theta. */
FST_API int fst_forward_backward_batch(fst_t* fst, const int32_t* d_ids, const int64_t* d_offsets,
                               int32_t B, const float* d_weights, double* d_logz,
                               float* d_counts, int32_t* d_status, void* stream);

/* Storage budget of the plans that fst_viterbi_batch and
 * fst_forward_backward_batch build (0 = the fst_plan_create default).  A
 * batch whose per-string storage exceeds it runs in several waves. (Memory
 * policy: no counterpart in the paper.) */
FST_API int fst_set_batch_budget(fst_t* fst, int64_t mem_budget_bytes);

/* Plans of fst_viterbi_batch and fst_forward_backward_batch: parts_viterbi
 * and parts_fb stream-parallel parts (FST_PLAN_PARTS; 0 = by batch size:
 * one Viterbi part per 32 strings, at most 2 and at most 400 / n, one
 * forward-backward part per 8 strings, at most 4 and at most 1,600 / n,
 * n the longest string) and the accumulator layout (-1 = dense when
 * the dense accumulators and the live pool fit the batch budget in one
 * wave, else compact; 0 = compact; 1 = FST_PLAN_DENSE_ACC), and whether
 * the run's launches are recorded into a CUDA graph that is then launched
 * (graph: 0 = no, 1 = yes, never on the legacy default stream or inside a
 * capture the caller began; -1 = the default, no: recording and
 * instantiating a run of thousands of launches measured slower than
 * issuing them).  The default is 0, 0, -1, -1.  A batch call keeps its
 * plan's device storage for the next call of the same kind (part by part).
 * Outside a graph capture, the parts of a plan issue their launches from
 * one host thread each. (Execution policy: no counterpart in the paper.) */
FST_API int fst_set_batch_plan(fst_t* fst, int32_t parts_viterbi, int32_t parts_fb, int32_t layout, int32_t graph);

/* A plan holds everything a batch needs on the device for the per-position
 * loops of Alg. 1 and Alg. 2 (Sec. 5): the token lists of
 * every position (strings sorted by length), the accumulators, the live
 * pool of every position (states, values, backpointers or arcs) and the
 * per-token scalars.  The accumulators are hash tables keyed by (string,
 * state), sized for 128 live states per token of the busiest position (at
 * most the symbols' destination counts) at half load; a position that
 * holds more live states than a table fits ends the run with FST_ERR_OOM,
 * like a full pool, and leaves the plan usable.  FST_PLAN_DENSE_ACC gives
 * each string a dense accumulator of 2 Q slots instead (no such limit;
 * 16 to 48 bytes a state a string, which bounds the wave size).  Once created,
 * the run calls below allocate
 * nothing, so a sequence of them can be captured into a CUDA graph and
 * replayed.  A Viterbi-only plan and a forward-backward-only plan of the
 * same batch share nothing and may run concurrently on two streams.
 *   d_ids, d_offsets  as fst_viterbi_batch; they are read during
 *               fst_plan_create only (the plan keeps its own copy).
 *   mem_budget_bytes  cap on per-step storage; strings are processed in
 *               waves that fit (0 = a quarter of the free device memory at
 *               the call, at most 32 GiB and at least 256 MiB).
 *   flags       FST_PLAN_SINGLE_WAVE: fail with FST_ERR_OOM instead of
 *               splitting into waves (needed by fst_plan_forward followed by
 *               fst_plan_backward, which keep state between calls).
 * Synchronises `stream`. */
#define FST_PLAN_SINGLE_WAVE 1
#define FST_PLAN_NO_VITERBI 2   /* do not allocate Viterbi storage (keys, state maps) */
#define FST_PLAN_NO_FB 4        /* do not allocate forward-backward storage */
#define FST_PLAN_DENSE_ACC 8    /* dense per-string accumulators (see above) */
/* FST_PLAN_PARTS(k), k in 2..255, or-ed into flags: the batch is cut into k
 * contiguous string ranges of about equal token counts, each a plan of its
 * own (with its own waves and budget share) run on its own stream; a run
 * forks from `stream` into the parts' streams and joins back (events, so a
 * run can still be captured into a CUDA graph).  The positions of the parts
 * proceed independently, which overlaps their latency-bound launches.  The
 * parts share the count accumulators.  Not with the persistent driver nor
 * the autotuner. */
#define FST_PLAN_PARTS(k) ((((int32_t)(k)) & 0xff) << 8)
FST_API int fst_plan_create(fst_t* fst, const int32_t* d_ids, const int64_t* d_offsets, int32_t B,
                    int64_t mem_budget_bytes, int32_t flags, void* stream, fst_plan_t** out);
/* Free a plan (NULL accepted).  (No counterpart in the paper.) */
FST_API int fst_plan_destroy(fst_plan_t* plan);

/* Plan statistics (host outputs, any may be NULL): strings, tokens (sum of
 * lengths), waves, longest string, arc relaxations of one pass (sum over
 * tokens of |delta[w_t]|), kernel launches of one Viterbi run and of one
 * forward-backward run, and device bytes held by the plan. The relaxations are
 * the paper's count (Sec. 5). */
FST_API int fst_plan_info(const fst_plan_t* plan, int32_t* num_strings, int64_t* num_tokens,
                  int32_t* num_waves, int32_t* max_len, int64_t* relaxations,
                  int64_t* viterbi_launches, int64_t* fb_launches, int64_t* device_bytes);

/* Run Viterbi (Alg. 1) for every string of the plan (outputs as
 * fst_viterbi_batch).  Asynchronous on `stream`; allocates nothing. */
FST_API int fst_plan_viterbi(fst_plan_t* plan, float* d_scores, int32_t* d_paths, int32_t* d_olabels,
                     int32_t* d_status, void* stream);

/* Forward pass only (Alg. 2's forward loop; log Z per string); keeps the
 * forward values in the plan for fst_plan_backward.  Requires a single-wave
 * plan. */
FST_API int fst_plan_forward(fst_plan_t* plan, double* d_logz, int32_t* d_status, void* stream);

/* Backward pass and expected counts after fst_plan_forward on the same plan:
 * d_counts[k] = sum_b d_weights[b] * count_b(k) (d_weights NULL = all 1).
 * Returns FST_ERR_STATE if no forward pass preceded it. Alg. 2's backward and count loops. */
FST_API int fst_plan_backward(fst_plan_t* plan, const float* d_weights, float* d_counts, void* stream);

/* Forward and backward for every wave of the plan (any number of waves). Alg. 2. */
FST_API int fst_plan_forward_backward(fst_plan_t* plan, const float* d_weights, double* d_logz,
                              float* d_counts, int32_t* d_status, void* stream);

/* As fst_plan_backward and fst_plan_forward_backward, with the expected
 * start and final states as well (the two ends of Alg. 2's recursion):
 *   d_start  device float [num_states] or NULL: sum_b g_b P_b(path starts in q)
 *            = sum_b g_b exp(alpha_0[q] + beta_0[q] - log Z_b), the gradient
 *            of sum_b g_b log Z_b with respect to the start log-weights;
 *   d_final  device float [num_states] or NULL: likewise with
 *            exp(alpha_n[q] + beta_n[q] - log Z_b), the final log-weights.
 * d_counts may be NULL here; at least one output is required by
 * fst_plan_backward_ex.  Strings without a path add nothing. */
FST_API int fst_plan_backward_ex(fst_plan_t* plan, const float* d_weights, float* d_counts, float* d_start,
                                 float* d_final, void* stream);
/* Alg. 2 with the expected start and final states, every wave. */
FST_API int fst_plan_forward_backward_ex(fst_plan_t* plan, const float* d_weights, double* d_logz,
                                         float* d_counts, float* d_start, float* d_final, int32_t* d_status,
                                         void* stream);

/* EM re-estimation of the arc weights from expected counts (the M-step of
 * the training by expectation-maximisation that the counts of Alg. 2 serve,
 * Sec. 4).  Each state's outgoing arcs (over all symbols) are one
 * categorical distribution:
 *     theta'_k = log((count_k + pseudo_count) / sum_{j: src_j = src_k} (count_j + pseudo_count)),
 * computed in float64 and rounded to float32; a state whose arcs' total is
 * zero keeps their current log-weights.
 *   counts       [num_arcs] float expected counts (e.g. the d_counts of
 *                fst_plan_backward), caller arc order, >= 0.
 *   pseudo_count >= 0, added to every arc.
 *   theta_out    [num_arcs] float: the new log-weights (caller-owned).
 *   flags        FST_FLAG_DEVICE_PTRS: counts and theta_out are device
 *                pointers (else host); FST_EM_APPLY: also install them as the
 *                FST's weights (as fst_set_weights with FST_WEIGHT_LOG).
 * Synchronous.  FST_ERR_INVALID_ARG for a negative, NaN or infinite count. */
#define FST_EM_APPLY 2
FST_API int fst_em_update(fst_t* fst, const float* counts, float pseudo_count, float* theta_out, int32_t flags);

/* The output-clamped FST of `fst`, for the numerator log Z(x, y) of a
 * conditional (CRF-style) likelihood: the weight of the paths that read x
 * and write y (Eq. 1 restricted to the arcs whose output label is y_t at
 * position t).  Its arc k is fst's arc k (same id, states and weight) with
 * the input label replaced by the pair (ilabel_k, olabel_k); the pairs are
 * numbered 0..*num_pairs-1 in (input, output) order and symbol *num_pairs
 * has no arcs.  So log Z(x, y) and the arc posteriors given x and y are
 * fst_forward_backward (or a plan) of the clamped FST on the pair string
 * that fst_clamp_labels makes.  The handle is an ordinary FST (free it with
 * fst_destroy); fst_set_weights takes the same weight vector as fst's. */
FST_API int fst_create_clamped(const fst_t* fst, fst_t** out, int32_t* num_pairs);

/* Pair string of (ids, olabels) for an FST made by fst_create_clamped: host
 * arrays of length n; pair_ids[t] is the symbol of (ids[t], olabels[t]), or
 * num_pairs (no arcs) when no arc carries that pair.  FST_ERR_STATE for a
 * handle that is not a clamped FST. (The CRF numerator: not in the paper.) */
FST_API int fst_clamp_labels(const fst_t* clamped, const int32_t* ids, const int32_t* olabels, int64_t n,
                             int32_t* pair_ids);

/* Acyclic input lattices composed with the FST (the generalisation of an
 * input string that Sec. 6.1 names).  A lattice has num_nodes >= 1 nodes
 * numbered in a topological order -- node 0 is the start, node
 * num_nodes-1 the end -- and num_edges >= 0 edges; edge e goes from from[e]
 * to to[e] (from[e] < to[e] < num_nodes), reads symbol label[e] in [0, m)
 * and carries the log-weight weight[e] (not NaN or +inf).  All arrays are
 * host arrays; the calls are synchronous and allocate their working tables
 * (num_nodes x num_states per table).  A string is the lattice whose edge t
 * goes from node t to t+1 with weight 0, and decodes exactly as
 * fst_viterbi / fst_forward_backward.
 *
 * Viterbi: the best pair of a lattice path and an FST path reading its
 * symbols, each step scored fl(fl(V + theta_arc) + weight_edge) in float32
 * (ties: the lowest arc id into each (node, state), then the lowest edge
 * id), plus the start and final weights.  best_score gets its log-weight
 * (-inf: none); edge_path and arc_path ([num_nodes-1] each, NULL allowed
 * when num_nodes = 1) its edges and arcs; *path_len their number.
 * Returns FST_OK, FST_ERR_NO_PATH or an error. */
FST_API int fst_lattice_viterbi(fst_t* fst, int32_t num_nodes, int32_t num_edges, const int32_t* from,
                                const int32_t* to, const int32_t* label, const float* weight, float* best_score,
                                int32_t* edge_path, int32_t* arc_path, int32_t* path_len);

/* Forward-backward over a lattice (float64 values): log Z of all (lattice
 * path, FST path) pairs, the expected count of each arc (summed over the
 * edges that read its symbol; [num_arcs] or NULL) and the posterior of each
 * edge ([num_edges] or NULL).  Returns FST_OK, FST_ERR_NO_PATH or an error.
 * Alg. 2 over the lattice (Sec. 6.1). */
FST_API int fst_lattice_forward_backward(fst_t* fst, int32_t num_nodes, int32_t num_edges, const int32_t* from,
                                         const int32_t* to, const int32_t* label, const float* weight,
                                         double* log_z, float* arc_posteriors, float* edge_posteriors);

/* The weight of one string as a parallel product over time (the parallel
 * prefix approach of Sec. 6.1): the slice of each position becomes a dense
 * num_states x num_states matrix of log-weights, adjacent matrices are
 * multiplied pairwise in parallel and the products again until one is
 * left (log2(n) dependent rounds; Q^3 work per product), then closed with
 * the start and final weights.  For small dense FSTs (num_states <= 512,
 * FST_ERR_UNSUPPORTED beyond) and long strings.
 *   log_z       host double: log Z (log-sum products in float32, the final
 *               sum in float64).
 *   best_score  host float: the best path's log-weight from max-plus
 *               products; its float32 additions are associated in tree
 *               order, so it can differ from fst_viterbi's in the last bits.
 * Host pointers; synchronous; allocates its matrices.  Returns FST_OK,
 * FST_ERR_NO_PATH or an error. */
FST_API int fst_prefix_log_z(fst_t* fst, const int32_t* ids, int32_t n, double* log_z, float* best_score);

/* log Z of one string with every value and weight in float64 (the forward
 * recursion of Alg. 2 in the log domain; plain method, one launch per
 * position).  For finite-difference checks of d log Z / d theta, which a
 * central difference of step 1e-6 can only resolve with log Z known to
 * ~1e-12.  Host pointers; synchronous.
 *   theta   [num_arcs] host float64 log-weights (caller arc order), or NULL
 *           to reuse the float64 weights of the previous call
 *           (FST_ERR_STATE if there were none).  The float32 weights used
 *           by every other entry point are not touched.
 *   ids     [n] host symbols.      log_z  host double (-inf = no path). */
FST_API int fst_log_z_f64(fst_t* fst, const double* theta, const int32_t* ids, int32_t n, double* log_z);

/* Per-launch timing of a plan's runs (the tracing subsystem).  With
 * enable != 0, every kernel that a following fst_plan_* run queues is
 * bracketed by two CUDA events on the run's stream; fst_plan_profile_read
 * waits for the last of them and returns, per kernel kind, the summed
 * device time in milliseconds and the number of launches since the last
 * read (host arrays of FST_PROF_KINDS entries, either may be NULL), then
 * starts a new accumulation.  Do not enable it while capturing a graph.
 * (Tracing: no counterpart in the paper.) */
#define FST_PROF_VIT_FIRST 0   /* Viterbi: start states push their arcs into the first position */
#define FST_PROF_VIT_STEP 1    /* Viterbi: one position's live states read out, their arcs pushed into the next */
#define FST_PROF_VIT_FINAL 2   /* Viterbi final reduction */
#define FST_PROF_BACKTRACE 3   /* Viterbi backtrace */
#define FST_PROF_FWD_FIRST 4   /* forward: start states push their arc maxima into the first position */
#define FST_PROF_FWD_SUM 5     /* forward: fixed-point sums of one position */
#define FST_PROF_FWD_STEP 6    /* forward: one position's live states read out, their arc maxima pushed into the next */
#define FST_PROF_FB_FINAL 7    /* log Z and the float64 normaliser prefix */
#define FST_PROF_BWD_STEP 8    /* backward: backward values of position t-1 and the posteriors of position t */
#define FST_PROF_COUNTS 9      /* expected counts to float */
#define FST_PROF_KINDS 10
FST_API int fst_plan_profile(fst_plan_t* plan, int32_t enable);
/* Read and restart the accumulation (no counterpart in the paper). */
FST_API int fst_plan_profile_read(fst_plan_t* plan, double* ms_by_kind, int64_t* launches_by_kind);

/* The same per-launch timing for the single-string calls of a handle
 * (fst_viterbi, fst_forward_backward): kinds and semantics as
 * fst_plan_profile / fst_plan_profile_read. (Tracing: no counterpart in the paper.) */
FST_API int fst_profile(fst_t* fst, int32_t enable);
/* Read and restart the accumulation (no counterpart in the paper). */
FST_API int fst_profile_read(fst_t* fst, double* ms_by_kind, int64_t* launches_by_kind);

/* The live work of the handle's last single-string call, for measurement:
 * *entries = live states over all positions, *arcs = arcs out of them on
 * their next symbol (-1 unless the last call was fst_forward_backward).
 * Synchronous.  Either output may be NULL. (The relaxations Sec. 5 counts,
 * restricted to live states.) */
FST_API int fst_live_work(fst_t* fst, int64_t* entries, int64_t* arcs);

/* The live work of the plan's last pass (its last wave), for measurement:
 * *entries = live states over all positions (the pool entries handed out),
 * *arcs = arcs out of those states on their next symbol (the pushes of the
 * forward pass; -1 for a plan without forward-backward storage).  Waits for
 * the plan's work on `stream`.  Either output may be NULL. (The relaxations
 * Sec. 5 counts, restricted to live states.) */
FST_API int fst_plan_live_work(fst_plan_t* plan, int64_t* entries, int64_t* arcs, void* stream);

/* How a plan advances its positions (the batched driver).
 *   FST_DRIVER_LAUNCH      one kernel launch per position and kernel kind
 *                          (the default; a run can be captured into a CUDA
 *                          graph and replayed).
 *   FST_DRIVER_PERSISTENT  one cooperative launch per pass (Viterbi, forward,
 *                          backward) of grid_blocks blocks (0 = the plan's
 *                          estimate), all co-resident, that runs every
 *                          position; positions are separated by a grid-wide
 *                          barrier in device memory instead of kernel
 *                          boundaries.  Each wait of that barrier gives up
 *                          after barrier_timeout_us (0 = keep the current
 *                          limit, 2 s by default); the run then ends early
 *                          and reports FST_ERR_TIMEOUT in the status of every
 *                          string of its wave, and the next run starts clean.
 * Results are identical under both drivers.  FST_ERR_UNSUPPORTED when the
 * device cannot launch cooperative kernels or grid_blocks cannot be
 * co-resident.  Do not run a persistent plan concurrently with another
 * persistent plan on the same device. (Sec. 5 launches one kernel per position;
 * the persistent driver has no counterpart in the paper.) */
#define FST_DRIVER_LAUNCH 0
#define FST_DRIVER_PERSISTENT 1
FST_API int fst_plan_set_driver(fst_plan_t* plan, int32_t driver, int32_t grid_blocks, int64_t barrier_timeout_us);
/* The plan's driver and, for the persistent one, the grid of its forward
 * pass (host outputs, either may be NULL). (No counterpart in the paper.) */
FST_API int fst_plan_get_driver(const fst_plan_t* plan, int32_t* driver, int32_t* grid_blocks);

/* Autotuner of the batched driver: runs the plan's own passes (Viterbi and
 * forward-backward with counts, those the plan has storage for) under each
 * candidate configuration -- the launch driver with three grid densities
 * (16, 64 or 256 live states assumed per token) and the persistent driver at
 * whole multiples of the SM count up to the co-resident limit -- keeps the
 * fastest (the best of two timed runs after a warm-up, CUDA events on
 * `stream`), and sets it on the plan.  Results are cached per device name,
 * FST shape (states, arcs, symbols) and batch shape (strings, tokens,
 * longest string, waves, passes): a later plan with the same key takes the
 * cached choice without timing (FST_TUNE_REFRESH times again).  When the
 * environment variable FSTGPU_TUNE_CACHE names a file, the cache is read
 * from and appended to it.  Allocates scratch outputs for the timing runs
 * and synchronises `stream`; do not call it during graph capture.  Host
 * outputs (any may be NULL): the chosen driver, its persistent grid (0 for
 * the launch driver) and its time in milliseconds. (No counterpart in the paper.) */
#define FST_TUNE_REFRESH 1
FST_API int fst_plan_autotune(fst_plan_t* plan, void* stream, int32_t flags, int32_t* driver, int32_t* grid_blocks,
                              double* best_ms);

/* Fault injection for testing the failure paths (made on the host; nothing
 * faults).  FST_FAULT_BARRIER_STALL: the grid barriers of the plan's
 * persistent passes wait for `value` blocks (1..1024) beyond the grid, so
 * that no wait can complete and every wait runs out (the FST_ERR_TIMEOUT
 * path).  FST_FAULT_NONE (value ignored) turns injection off. (No counterpart in the paper.) */
#define FST_FAULT_NONE 0
#define FST_FAULT_BARRIER_STALL 1
FST_API int fst_plan_fault_inject(fst_plan_t* plan, int32_t kind, int64_t value);

/* Cap the live pool of the plan's following runs at `entries` live states
 * (over all positions of a wave; 0 = the capacity the plan allocated, which
 * larger values cannot exceed).  Allocates nothing.  A run whose live states
 * do not fit stops handing out pool entries, reports FST_ERR_OOM in the
 * status of every string of its wave (scores -inf, paths -1, log Z -inf,
 * no counts) and leaves the plan usable: the next run clears what the
 * overflowing one left behind.  For memory-capped deployments and for
 * exercising that failure path. (No counterpart in the paper.) */
FST_API int fst_plan_limit_pool(fst_plan_t* plan, int64_t entries);

/* Direction switch of the forward pass (plans with FST_PLAN_DENSE_ACC and
 * the launch driver; Sec. 4 remarks that the slice can be read by
 * destination): a token with at least min_live live states, whose string
 * goes on, scatters its forward values into a dense vector, and the next
 * position pulls over the destination-ordered slice -- coalesced records,
 * a warp-segmented exact maximum and fixed-point sum per destination, one
 * atomic per destination and row of 32 arcs -- instead of pushing each arc
 * with an atomic.  Up to 16 tokens per position; the rest push.  The
 * results are the pushes' (the same exact terms).  min_live: 0 = off (the
 * default: on the 20M-arc batch every threshold measured slower than none,
 * the pull's launch per position costing more than it saves); -1 =
 * max(2048, num_states / 2); else the threshold. */
FST_API int fst_plan_set_pull(fst_plan_t* plan, int64_t min_live);

/* Bounds-checked build.  A library compiled with -DFST_DEBUG (build.py's
 * build_debug) checks, in the frontier kernels, every computed index into
 * the staging buffers, the live pool, the dense accumulators and the arc
 * records against its buffer's size; a violation is counted, the first is
 * recorded (code: 1 staging, 2 pool write, 3 pool read, 4 dense
 * accumulator, 5 arc record; its index and the bound) and the access is
 * skipped.  This call reads the record (host outputs, any may be NULL) and
 * clears it.  FST_ERR_UNSUPPORTED in a normal build. (No counterpart in the paper.) */
FST_API int fst_debug_checks(int64_t* violations, int32_t* code, int64_t* index, int64_t* bound);

/* Compact accumulators: cap the hash tables of the plan's following runs at
 * `slots` slots each (rounded down to a power of two, at least 2; 0 = the capacity
 * allocated, which larger values cannot exceed).  Allocates nothing.  A run
 * with more live states at one position than a table holds reports
 * FST_ERR_OOM for every string of its wave and leaves the plan usable, as
 * with fst_plan_limit_pool.  No effect on FST_PLAN_DENSE_ACC plans.
 * (No counterpart in the paper.) */
FST_API int fst_plan_limit_table(fst_plan_t* plan, int64_t slots);
/* Slots of each compact accumulator table (the largest over the plan's
 * parts; 0 for FST_PLAN_DENSE_ACC). (No counterpart in the paper.) */
FST_API int fst_plan_table_slots(const fst_plan_t* plan, int64_t* slots);

/* Plain-method Viterbi of one string that allocates no memory (the paper
 * has no counterpart: this is a deployment variant of fst_viterbi).  For
 * callers that cannot allocate device memory at decode time -- a host whose
 * memory manager owns every allocation, a latency-critical loop that must
 * not take the implicit synchronisation of cudaMalloc/cudaFree, a process
 * under a hard device-memory cap.  Every piece of per-call working memory
 * (accumulators, live states with backpointers, token tables) comes from one
 * fixed 32 MiB device array inside the library, resident on every device
 * that loads it until the process exits.
 *   ids        [n] host, symbols in [0, m); n >= 0.
 *   d_score    device float [1]: best log-weight, -inf when no path.
 *   d_path     device int32 [n]: arc ids of the best path (-1 when no path).
 *   d_olabels  device int32 [n] or NULL.
 *   stream     cudaStream_t of the FST's device; the call is asynchronous
 *              on it.  The FST's device must be the current device
 *              (FST_ERR_INVALID_ARG otherwise, nothing launched).
 * Score, path and output labels are bit-identical to fst_viterbi.  Being
 * asynchronous, the call cannot return FST_ERR_NO_PATH: a string without an
 * accepting path is reported only through the outputs (*d_score = -inf and
 * d_path all -1), and the return code is FST_OK.  Returns FST_ERR_UNSUPPORTED
 * (nothing is launched) when the string needs more than the fixed array:
 * about 24*Q + 16*(sum over positions of the distinct destinations of the
 * position's symbol) + 8*(the largest such count) + 60*n bytes.  The
 * first call on a device looks up the array's device address with that
 * device current: make it before any stream capture.  All calls share the array
 * and see the previous call's
 * contents, which each call clears where needed; calls that overlap on the
 * GPU race on it and must be serialised by the caller. */
FST_API int fst_viterbi_noalloc(fst_t* fst, const int32_t* ids, int32_t n, float* d_score, int32_t* d_path,
                                int32_t* d_olabels, void* stream);

/* Message of the last failing call on this host thread ("" if none).
 * (No counterpart in the paper.) */
FST_API const char* fst_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FSTGPU_H_ */
