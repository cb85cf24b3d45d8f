// kernels.cuh -- launch arguments of the frontier kernels (kernels.cu).
#pragma once

#include <stdint.h>

#include "fst_internal.cuh"

namespace fstgpu {

// Device view of one arc layout.
struct LayoutView {
  const int32_t* other;      // [P] gathered state: source (forward layout) or destination (backward)
  const float* theta;        // [P]
  const int32_t* arc_id;     // [P] caller arc id, -1 on padding
  const int32_t* seg_state;  // [nseg] destination (forward) or source (backward)
  const int32_t* seg_pos;    // [nseg] first padded position
  const int32_t* seg_len;    // [nseg] arcs
  const int64_t* sym_seg;    // [m+1] segments of each input symbol
  const int32_t* xseg;       // [P] segment of the other layout holding the same arc
  const ulonglong2* seg_hash;  // (symbol, state) -> segment (source-segmented layout only)
  int64_t hash_mask;
};

inline LayoutView view_of(const Layout& L) {
  return LayoutView{L.other, L.theta, L.arc_id, L.seg_state, L.seg_pos, L.seg_len, L.sym_seg, L.xseg,
                    L.seg_hash, L.hash_mask};
}

// The tokens of one input position t: slots slot0 .. slot0+n-1 of the
// step list T.step_tok (tokens of a wave in step order).  Token p is
// position t of wave-local string T.b[p]; the tokens of a string are
// consecutive, so the previous position of token p is token p - 1.  The x_*
// fields name another step whose pool entries the kernel also reads: the
// previous position for the expand kernels, position t-2 for the backward
// reduce (x_n = 0: none).
struct StepView {
  int32_t t;
  int32_t n;
  int32_t slot0;
  int32_t x_t, x_n, x_slot0;
  int32_t blocks;   // grid of the launch (work is a grid-stride loop)
};

struct TokenView {
  const int32_t* step_tok;  // [N] token of each step slot
  const int32_t* sym;
  const int32_t* b;
  const int64_t* stf;   // forward staging offset of the token inside its step
  const int64_t* stb;   // backward staging offset of the token inside its step
};

// State of one wave (or of one plain-method string).
//
// Frontiers: dense per string, two parity buffers, entries tagged with the
// token that wrote them (a mismatching tag reads as -inf), so nothing is
// cleared between positions and a fresh run epoch invalidates everything.
//
// Live pool: for every token, the states with a finite forward (Viterbi)
// value at its position, with the backpointer (Viterbi) or the forward
// segment and stored value (forward).  The last block of a step's expand
// kernel hands out the pool ranges: the step's tokens get consecutive ranges
// in step order, so one position's entries are one flat range that the next
// kernels split evenly over warps, whatever the tokens' frontier sizes.
//
// Staging: the segments a step has to reduce, per token, deduplicated with
// a touch bitmap per string that the reduce kernel clears again.
struct FrontierState {
  int32_t Q;
  int32_t W;                         // 32-bit words of a touch bitmap
  const uint32_t* epoch;             // device: tags of this run start at *epoch
  uint32_t tok0;                     // token p writes tag *epoch + tok0 + p
  unsigned long long* alpha;         // [Bw][2][Q]
  unsigned long long* beta;          // [Bw][2][Q] (null for Viterbi-only state)
  uint32_t* touch;                   // [Bw][W], all zero between kernels
  uint32_t* touch_b;                 // second touch bitmap: positions of odd parity in the forward passes
  int32_t* stage;                    // staging of the current step
  int32_t* stage_b;                  // second staging buffer: positions of odd parity in the forward passes
  uint32_t* scnt_f;                  // [N] segments staged per token, forward direction
  uint32_t* scnt_b;                  // [N] backward direction
  int32_t* pool_q;                   // [cap] state (-1: the value turned out -inf)
  int32_t* pool_x;                   // [cap] Viterbi: backpointer (forward position); forward: forward segment
  float* pool_v;                     // [cap] forward value r_t (null for Viterbi)
  int64_t* pool_base;                // [N] by token
  int32_t* pool_cnt;                 // [N] by token
  int64_t* slot_base;                // [N] by step slot: first pool entry of the slot's token
  int64_t* bslot_base;               // [N] by step slot: first flat backward staging index
  int64_t* step_rng;                 // [2 (T+2)]: pool entries [begin, end) of each position
  int64_t* bstep_rng;                // [2 (T+2)]: flat backward staging indices [0, end) of each position
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

// Expected counts per forward padded arc position.
struct CountView {
  int batched;        // 0: Kahan float pair (one string); 1: double atomics
  float* cnt;
  float* comp;
  double* cnt64;
};

// Expand of the first position (Viterbi and forward): the start states
// stage the forward segments their arcs on w_1 lead to.
int launch_expand(const LayoutView& Lb, const TokenView& T, const StepView& V, const FrontierState& S, cudaStream_t s);
// One position of the forward passes: each staged forward segment of
// position t becomes a frontier entry (reduce), and each new live state
// immediately stages the segments of position t+1 its arcs lead to
// (expand).  V.x_* name position t+1 (x_n = 0 at a wave's last position).
int launch_vit_step(const LayoutView& Lf, const LayoutView& Lb, const TokenView& T, const StepView& V,
                    const FrontierState& S, cudaStream_t s);
int launch_fwd_step(const LayoutView& Lf, const LayoutView& Lb, const TokenView& T, const StepView& V,
                    const FrontierState& S, cudaStream_t s);
// Backward expand: posteriors of the arcs into the live states of position
// t and staging of the sources whose backward value at t-1 is needed.
int launch_bwd_expand(const LayoutView& Lf, const TokenView& T, const StepView& V, const FrontierState& S,
                      const CountView& C, cudaStream_t s);
// Backward reduce: backward values of the staged sources; also restores the
// forward values of position t-2 for the next backward expand.
int launch_bwd_reduce(const LayoutView& Lb, const TokenView& T, const StepView& V, const FrontierState& S,
                      cudaStream_t s);
int launch_vit_final(const FrontierState& S, int32_t Bw, float* scores, int32_t* qfinal, int32_t* status,
                     cudaStream_t s);
int launch_backtrace(const LayoutView& Lf, const FrontierState& S, const int32_t* olabel_by_id, int32_t Bw,
                     const int32_t* qfinal, int32_t* paths, int32_t* olabels, cudaStream_t s);
int launch_fb_final(const FrontierState& S, int32_t Bw, double* logz, int32_t* status, cudaStream_t s);
int launch_counts_out(const int32_t* arc_id_fwd, int64_t P, const CountView& C, float* out, cudaStream_t s);

}  // namespace fstgpu
