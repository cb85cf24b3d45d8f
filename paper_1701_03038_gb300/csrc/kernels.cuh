// kernels.cuh -- launch arguments of the frontier kernels (kernels.cu).
#pragma once

#include <stdint.h>

#include "fst_internal.cuh"

namespace fstgpu {

// Device view of the source-segmented arc layout: the arcs out of state q
// on symbol a are consecutive, found through a (symbol, state) hash.
struct LayoutView {
  const int4* arcs;            // [P] {destination, theta bits, caller id, 0}
  const ulonglong2* seg_hash;  // (symbol, state) -> len << 32 | first position
  int64_t hash_mask;
  int64_t P;                   // arc records (the bounds-checked build checks against it)
};

inline LayoutView view_of(const Layout& L) { return LayoutView{L.arcs, L.seg_hash, L.hash_mask, L.P}; }

// The tokens of one input position t: slots slot0 .. slot0+n-1 of the
// step list T.step_tok (tokens of a wave in step order).  Token p is
// position t of wave-local string T.b[p]; the tokens of a string are
// consecutive, so the previous position of token p is token p - 1.  The x_*
// fields name a second position the kernel also works on: the next one for
// the forward steps (whose new live states they push there), the previous
// one for the kernels that walk the live states of t-1 (x_n = 0: none).
struct StepView {
  int32_t t;
  int32_t n;
  int32_t slot0;
  int32_t x_t, x_n, x_slot0;
  int32_t blocks;   // grid of the launch (work is a grid-stride loop)
  int32_t y_t;      // backward steps with compact accumulators: the position whose
                    // backward values this step clears (0: none)
};

struct TokenView {
  const int32_t* step_tok;  // [N] token of each step slot
  const int32_t* sym;
  const int32_t* b;
  const int64_t* stf;   // staging offset of the token inside its step
};

// State of one wave (or of one plain-method string).
//
// Accumulators, in one of two layouts, all empty between runs:
//   dense   -- per string, two parity buffers of Q slots each (the plain
//              method's single string, and plans made with
//              FST_PLAN_DENSE_ACC);
//   compact -- open-addressing hash tables keyed by (string, state), one per
//              position parity, sized for the live states of a position
//              rather than for every state of every string: a few MB that
//              stay in L2, where the dense arrays of a large batch take tens
//              of GB.  The staging lists then hold table slots.
// In both, a forward step pushes every arc out of a live state of position
// t into the accumulator of its destination at t+1 with an atomic max (the
// packed Viterbi key, or the forward maximum); the push that finds the
// accumulator empty (or inserts its key) stages the destination.  The next
// step reads each staged accumulator once, turns it into a live-pool entry
// and empties it.
//
// Live pool: for every token, the states with a finite value at its
// position: the state, its value, and the best incoming arc (Viterbi) or
// the segment of its arcs on the next symbol (forward).  The last block of a
// step hands out the pool ranges: the step's tokens get consecutive ranges
// in step order, so one position's entries are one flat range that the next
// kernels split evenly over blocks, whatever the tokens' frontier sizes.
struct FrontierState {
  int32_t Q;
  // dense: [Bw][2][Q] accumulators of acc_stride 64-bit words: Viterbi keys
  // use the first word; the forward passes need stride 2, {fixed-point sum,
  // maximum order key in the low half}, so that both sit on one cache line
  unsigned long long* acc;
  int32_t acc_stride;
  double* beta;                      // [Bw][2][Q] backward values, float64 (null for Viterbi-only state)
  int32_t* vmap;                     // [Bw][2][Q] Viterbi: pool entry of each live state (null for forward-only state)
  // compact (hmask > 0): tables of hmask + 1 slots, key (wave-local string
  // + 1) << 32 | state (0 = empty).  htab0 / htab1 hold the positions of even / odd
  // parity, 2 acc_stride words a slot: {key, Viterbi key} or {key, maximum
  // order key, fixed-point sum, 0}.  btab0..2 hold the backward values of
  // the positions t with t mod 3 = 0, 1, 2, {key, float64 bits}; bslot maps
  // each pool entry to its slot there (-1: none).  Viterbi needs no state
  // map: the backtrace finds each predecessor among its token's entries.
  unsigned long long* htab0;
  unsigned long long* htab1;
  unsigned long long* btab0;
  unsigned long long* btab1;
  unsigned long long* btab2;
  int32_t* bslot;
  uint64_t hmask;
  // Direction switch of the forward pass (dense accumulators, launch
  // driver; dense_min = 0: off).  A token with at least dense_min live
  // states, whose string goes on and whose next symbol's slice has no
  // segment longer than a window (pull_lseg), gets one of DENSE_SLOTS dense
  // value vectors for its position: the forward step scatters its values
  // there instead of pushing its arcs, and the next position pulls over
  // the destination-ordered slice.  dvec [DENSE_SLOTS][2][Q] float64 (-inf
  // between uses), dslot [N] the slot of each token (-1: none), dlist
  // [T+2][DENSE_SLOTS] the dense tokens of each position, dcnt [T+2] their
  // number.
  double* dvec;
  int32_t* dslot;
  int32_t* dlist;
  int32_t* dcnt;
  const int64_t* pull_lseg;  // [m+1] long segments of the destination-ordered slices before each symbol
  int32_t dense_min;
  const int32_t* src_by_id;          // [A] source state of each arc
  int32_t* stage;                    // staged destinations of positions of even parity
  int32_t* stage_b;                  // of odd parity
  int64_t stage_cap;                 // entries of each staging buffer
  int32_t Bw;                        // strings of the wave (dense accumulators: [Bw][2][Q])
  int32_t chain;                     // host only: launch the step kernels chained to their predecessor
  uint32_t* scnt;                    // [N] destinations staged per token
  int32_t* pool_q;                   // [cap] state
  int32_t* pool_x;                   // [cap] Viterbi: best incoming arc id; forward: first arc on the next symbol
  int32_t* pool_n;                   // [cap] Viterbi: pool entry of the best arc's source (-1 at the first
                                     // position); forward: arcs on the next symbol
  float* pool_v;                     // [cap] Viterbi score
  double* pool_d;                    // [cap] forward value r_t, float64 (may share pool_v's storage)
  int64_t* pool_base;                // [N] by token
  int32_t* pool_cnt;                 // [N] by token
  int64_t* slot_base;                // [N] by step slot: first pool entry of the slot's token
  int64_t* step_rng;                 // [2 (T+2)]: pool entries [begin, end) of each position
  int64_t* pool_top;                 // [1] entries handed out in this run
  int64_t pool_cap;
  uint32_t* flags;                   // [2]: last-block counter, error bits (1 = pool full)
  const float* theta_s;
  const float* theta_f;
  const int32_t* start_q;            // states with a finite start weight
  int32_t nstart;
  uint32_t* mkey;                    // [N] forward step maxima (order keys)
  uint32_t* ekey;                    // [N] backward step maxima
  double* csum;                      // [N] C_t = sum_{s<=t} m_s
  double* esum;                      // [N] E_t
  const double* logz;                // [Bw]
  const float* gweight;              // [Bw] or null
  const int32_t* bw_n;               // [Bw] string lengths
  const int64_t* bw_off;             // [Bw] first token of each string
};

constexpr int DENSE_SLOTS = 16;

// The destination-ordered slices the pull reads: records {source,
// destination, caller id (< 0: padding), 0}, weights, and each symbol's
// 128-arc windows [win[a], win[a+1]).
struct PullView {
  const int4* rec;
  const float* theta;
  const int64_t* win;
};

// Step offsets of a wave on the device, for the persistent passes: the
// tokens of position t are step slots step0[t] .. step0[t+1]-1.
struct WaveSteps {
  const int32_t* step0;  // [tmax + 2]
  int32_t tmax;
};

// Grid barrier of a persistent pass: bar[0] counts arrivals, bar[1] is the
// generation; a wait gives up after limit_ns.  `expected` is the number of
// blocks that meet at each barrier beyond the grid (0 in normal use; a
// fault-injection setting raises it so that the wait runs out).
struct GridSync {
  uint32_t* bar;
  uint32_t expected;
  uint64_t limit_ns;
};

// Expected counts by caller arc id.
struct CountView {
  int batched;        // 0: Kahan float pair (one string); 1: double atomics
  float* cnt;
  float* comp;
  double* cnt64;
  double* start64;    // [Q] expected start states, or null
  double* final64;    // [Q] expected final states, or null
};

// First position (Viterbi and forward): the start states push their arcs
// on w_1 into the accumulators of position 1.
int launch_vit_first(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                     cudaStream_t s);
int launch_fwd_first(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                     cudaStream_t s);
// One position of the forward passes: each staged destination of position
// t becomes a pool entry (its accumulator is read and cleared), and each
// new live state at once pushes its arcs on w_{t+1} into the accumulators
// of position t+1.  V.x_* name position t+1 (x_n = 0 at a wave's last
// position).
int launch_vit_step(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                    cudaStream_t s);
int launch_fwd_step(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                    cudaStream_t s);
// Forward sum of position t: the live states of t-1 (V.x_*) add
// exp(value - maximum) of each arc to its destination's accumulator.  With
// the direction switch, the dense tokens of t-1 pull over R (maxima, terms
// and sums of their destinations at once), and the last block hands out
// the pool ranges of t.
int launch_fwd_sum(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                   const PullView& R, cudaStream_t s);

// Backward step of position t: for each live state q of position t-1
// (V.x_*), beta_{t-1}[q] over its arcs on w_t, and the posterior of each of
// those arcs.
int launch_bwd_step(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                    const CountView& C, cudaStream_t s);
// Persistent passes (one cooperative launch of `grid` blocks runs every
// position of the wave, separated by bounded grid barriers).  `grid` must be
// co-resident: at most persist_grid_limit(0: Viterbi, 1: forward,
// 2: backward); FST_ERR_UNSUPPORTED otherwise.  G.bar must be zero.
int persist_grid_limit(int which);
int launch_vit_persist(const LayoutView& L, const TokenView& T, const WaveSteps& D, const FrontierState& S,
                       int32_t grid, const GridSync& G, cudaStream_t s);
int launch_fwd_persist(const LayoutView& L, const TokenView& T, const WaveSteps& D, const FrontierState& S,
                       int32_t grid, const GridSync& G, cudaStream_t s);
int launch_bwd_persist(const LayoutView& L, const TokenView& T, const WaveSteps& D, const FrontierState& S,
                       const CountView& C, int32_t grid, const GridSync& G, cudaStream_t s);
// Best final state of each string; jfinal gets its pool entry (-1: no path).
int launch_vit_final(const FrontierState& S, int32_t Bw, float* scores, int32_t* jfinal, int32_t* status,
                     cudaStream_t s);
// The best path of each string, following the pool entries' predecessors.
int launch_backtrace(const FrontierState& S, const int32_t* olabel_by_id, int32_t Bw, const int32_t* jfinal,
                     int32_t* paths, int32_t* olabels, cudaStream_t s);
int launch_fb_final(const FrontierState& S, int32_t Bw, double* logz, int32_t* status, cudaStream_t s);
int launch_counts_out(int64_t A, const CountView& C, float* out, cudaStream_t s);
// Expected final states of every string (and expected start states of the
// empty strings, whose paths start where they end), added to C.final64 and
// C.start64 with the strings' weights.  Needs the forward pass and log Z.
int launch_final_posteriors(const FrontierState& S, int32_t Bw, const CountView& C, cudaStream_t s);
// p[i] = -inf, i < n.
int launch_fill_neg_inf(double* p, int64_t n, cudaStream_t s);
// out[i] = (float)in[i], i < n.
int launch_to_float(const double* in, int64_t n, float* out, cudaStream_t s);
// Bounds-checked build (compiled with FST_DEBUG): the kernels check every
// computed index into the staging buffers, the live pool, the dense
// accumulators and the arc records against its buffer's size, count the
// violations, record the first (check code, index, bound) and skip the
// access.  Reads and clears that record; FST_ERR_UNSUPPORTED in a normal
// build.
int debug_read(int64_t* violations, int32_t* code, int64_t* index, int64_t* bound);

// Zero n 64-bit words of accumulators if an error bit is set in *flag: a
// run whose pool overflowed (or that gave up at a barrier) leaves staged
// accumulators behind.
int launch_clear_if_overflow(const uint32_t* flag, unsigned long long* acc, int64_t n, int num_sms, cudaStream_t s);
// Compact accumulators: clear the backward values of position y_t (after
// the pass's last step, which reads those of position 1).
int launch_bwd_clear(const FrontierState& S, int32_t pos, int num_sms, cudaStream_t s);

}  // namespace fstgpu
