// kernels.cuh -- launch arguments of the relaxation kernels (kernels.cu).
#pragma once

#include <stdint.h>

#include "fst_internal.cuh"

namespace fstgpu {

// Device view of one arc layout.
struct LayoutView {
  const int32_t* other;
  const float* theta;
  const double* theta64;
  const WinMeta* win;
  const int32_t* seg_state;
  const int32_t* seg_pos;
  const int64_t* sym_win;
  const int64_t* sym_seg;
};

inline LayoutView view_of(const Layout& L) {
  return LayoutView{L.other, L.theta, L.theta64, L.win, L.seg_state, L.seg_pos, L.sym_win, L.sym_seg};
}

// Tokens of one wave: token p is position t (1-based) of wave-local string b.
struct TokenView {
  const int32_t* sym;
  const int32_t* b;
  const int32_t* t;
  const int64_t* cbase;   // base of the token's per-segment storage (forward segments)
  const int64_t* lbase;     // long-segment scratch slots (forward layout)
  const int64_t* lbase_b;   // long-segment scratch slots (backward layout)
  const int64_t* lwbase;    // long-window scratch slots (forward layout)
  const int64_t* lwbase_b;  // long-window scratch slots (backward layout)
  const int64_t* wbase;     // first window-liveness byte of the token (forward windows)
  const int64_t* bwbase;    // first mark byte of the token in the backward windows
};

// Work list of one step: items are (group, window-of-slice) pairs; a group
// is up to GMAX tokens of the same step with the same symbol.
struct WorkView {
  int single;        // 1: one token (p0, sym0); the group arrays are unused
  int32_t p0, sym0;
  int32_t g0, g1;    // group range of this step
  int64_t nitems;
  const int32_t* grp_first;
  const int32_t* grp_cnt;
  const int32_t* grp_sym;
  const int64_t* grp_item;  // item offset of each group inside its step (this layout)
  const int32_t* sorted_tok;
};

// Per-wave state shared by the passes.
struct WaveState {
  int32_t Q;
  const uint32_t* epoch;             // device: tags of this run start at *epoch
  uint32_t tok0;                     // first global token of the wave: token p writes *epoch + tok0 + p
  unsigned long long* alpha;         // [Bw][2][Q] tagged frontier
  unsigned long long* beta;          // [Bw][2][Q]
  int32_t* bp;                       // compact backpointers (forward segments)
  float* rc;                         // compact forward values r_t (forward segments)
  uint32_t* mkey;                    // [N] forward step maxima (order keys)
  uint32_t* ekey;                    // [N] backward step maxima
  double* csum;                      // [N] C_t = sum_{s<=t} m_s
  double* esum;                      // [N] E_t
  unsigned long long* skey;          // long-segment max keys
  uint32_t* scnt;                    // long-segment arrival counters
  float2* spart;                     // long-window (max, sum) partials
  const float* theta_s;
  const float* theta_f;
  const double* logz;                // [Bw] (wave-local view)
  const float* gweight;              // [Bw] or null
  int32_t* bw_n;                     // [Bw] string lengths
  int64_t* bw_off;                   // [Bw] first token of each wave string
  // Live-state bitmaps (bit q set = state q has a finite value): forward
  // values at position t live in rotation t % 3 of abm, backward values at
  // position t in rotation t % 3 of bbm; string b's bitmap of rotation r
  // starts at r * bm_rot + b * W.  The driver clears a rotation before the
  // launch that fills it.
  uint32_t* abm;
  uint32_t* bbm;
  const uint32_t* bm_start;          // states with a finite start weight
  const uint32_t* bm_final;          // states with a finite final weight
  int32_t W;                         // 32-bit words per bitmap
  int64_t bm_rot;
  // Summaries of the bitmaps: bit i of a summary is set when word i of the
  // bitmap is nonzero (one bit per 32 states).  Forward summaries are kept
  // per token for the whole pass (tsum + p * Ws): the backward pass prunes
  // its relaxation to sources whose forward value is finite.  Backward
  // summaries rotate like the bitmaps.
  uint32_t* tsum;
  uint32_t* bsum;
  const uint32_t* sum_start;
  const uint32_t* sum_final;
  int32_t Ws;                        // 32-bit words per summary
  int64_t sum_rot;
  // one byte per (token, forward window): 1 when the window wrote a finite
  // forward value for that token (cleared before each forward pass)
  uint8_t* wlive;
  // Window marks, one byte per (token, forward window) in fin and per
  // (token, backward window) in bin: set when the window holds an arc out of
  // a state whose forward value at the previous position is finite.  A pass
  // visits only marked windows of tokens past the first position; every
  // unmarked window holds arcs from dead sources only.  bin may be null.
  uint8_t* fin;
  uint8_t* bin;
  const int32_t* b_seg_state;
  const int32_t* b_seg_pos;
  const int32_t* b_seg_len;
  const int64_t* b_sym_seg;
  const int64_t* b_sym_win;
  const int32_t* b_fwin;
  const int64_t* f_sym_win;
  // Backward marks, one byte per (token, backward window): set when the
  // window holds an arc into a state whose backward value at that token's
  // position is finite.  The backward pass visits a window of a token when
  // its forward mark (bin) and backward mark (bmk) are set; at the first
  // position only the backward mark, at the last only the forward mark.
  uint8_t* bmk;
  const int32_t* f_seg_state;
  const int32_t* f_seg_pos;
  const int32_t* f_seg_len;
  const int64_t* f_sym_seg;
  const int32_t* f_bwin;
};

struct CountView {
  int batched;        // 0: Kahan float pair per arc; 1: double atomics
  float* cnt;         // [P_bwd]
  float* comp;        // [P_bwd]
  double* cnt64;      // [P_bwd]
};

// `grid` of the step launchers is the device's SM count.
int launch_vit_step(const LayoutView& L, const TokenView& T, const WorkView& W, const WaveState& S,
                    int grid, cudaStream_t s);
int launch_fwd_step(const LayoutView& L, const TokenView& T, const WorkView& W, const WaveState& S,
                    int grid, cudaStream_t s);
// Restoring the stored forward values of one position into the dense
// frontier (the forward layout's work list of that position; only strings
// longer than t_bwd).  It rides along with a backward step whose frontier
// reads touch the other parity buffer; W.nitems == 0 means none.
struct ScatterJob {
  LayoutView L;
  WorkView W;
  int32_t t_bwd;
};

int launch_bwd_step(const LayoutView& L, const TokenView& T, const WorkView& W, const WaveState& S,
                    const CountView& C, const ScatterJob& J, int grid, cudaStream_t s);
int launch_vit_final(const WaveState& S, int32_t Bw, float* scores, int32_t* qfinal, int32_t* status, cudaStream_t s);
int launch_backtrace(const LayoutView& Lf, const int32_t* tok_sym, const int64_t* cbase, const WaveState& S,
                     const int32_t* olabel_by_id, const int32_t* arc_id_fwd, int32_t Bw,
                     const int32_t* qfinal, int32_t* paths, int32_t* olabels, cudaStream_t s);
int launch_fb_final(const WaveState& S, int32_t Bw, double* logz, int32_t* status, cudaStream_t s);
int launch_counts_out(const int32_t* arc_id_bwd, int64_t P, const CountView& C, float* out, cudaStream_t s);

}  // namespace fstgpu
