// kernels.cu -- the per-position kernels and their epilogues.
//
// For input position t the paper relaxes every arc of the slice delta[w_t],
// one thread per arc, and resolves collisions on a destination with atomics:
// a packed 64-bit (probability | arc) atomicMax for Viterbi (Sec. 5.1) and an
// atomic log-add-exp for forward and backward (Sec. 5.2, Eq. 3).
//
// The frontiers of real decoding are sparse: a handful of states out of
// hundreds of thousands hold a finite value at a position.  An arc whose
// source is -inf contributes -inf to a max or a log-sum-exp and zero to a
// posterior, so skipping it changes no result.  Each position therefore
// runs two kernels, both driven by the live states only:
//
//   expand  -- every live state q of position t-1 finds its segment (w_t, q)
//              in the source-segmented layout and marks, through a touch
//              bitmap per string, the destination segments (w_t, q') of the
//              destination-segmented layout that its arcs lead to;
//   reduce  -- every marked destination segment is reduced over all its arcs
//              in arc order (a dead source reads as -inf), giving one
//              frontier entry; the touch bits are cleared on the way.
//
// The reduce visits each destination once, in a fixed order, with no
// atomics on values: results do not depend on scheduling.  Viterbi keys
// (order-preserving float bits << 32 | ~arc position) give the best score
// and, on ties, the lowest position, i.e. the lowest arc id since the arcs of
// a segment are sorted by id.  Forward and backward carry (max, scaled sum)
// pairs; each step's values are shifted by that step's maximum, the running
// shift kept in float64.  The backward pass mirrors the forward one: expand
// over the live states of position t (posteriors of their incoming arcs,
// staging of the sources), reduce over the staged source segments.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "kernels.cuh"

namespace fstgpu {
namespace {

constexpr int KT = 256;  // threads per block of the step kernels
constexpr int FT = 256;  // threads per block of the final reductions

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

__device__ __forceinline__ int32_t warp_id_global() { return (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }

__device__ __forceinline__ float decode_max(uint32_t k) { return k ? fkey_inv(k) : neg_inf(); }


// Owner of flat entry j among the n slots whose first entries base[0..n)
// are nondecreasing with base[0] <= j: the last slot with base <= j.  A warp
// first finds the owner of its chunk start j0 (warp-uniform, 32-way search),
// then each lane walks forward to its own entry (usually zero or one step).
__device__ __forceinline__ int32_t warp_owner(const int64_t* __restrict__ base, int32_t n, int64_t j0) {
  const int lane = threadIdx.x & 31;
  int32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const int32_t step = (hi - lo + 31) / 32;
    const int32_t k = lo + lane * step;
    const uint32_t bal = __ballot_sync(FULL, k < hi && __ldcg(base + k) <= j0);
    lo = lo + (31 - __clz(bal)) * step;  // bal != 0: base[lo] <= j0
    hi = min(hi, lo + step);
  }
  return lo;
}
__device__ __forceinline__ int32_t lane_owner(const int64_t* __restrict__ base, int32_t n, int32_t k, int64_t j) {
  while (k + 1 < n && __ldcg(base + k + 1) <= j) ++k;
  return k;
}

// Segment (a, q) of the source-segmented layout: a lookup in its
// open-addressing table (load factor <= 1/2, one 16-byte probe on average);
// -1 when q has no arc on a.
__device__ __forceinline__ int64_t find_seg(const LayoutView& L, int32_t a, int32_t q) {
  const uint64_t k = seg_hash_key(a, q);
  uint64_t h = seg_hash_slot(k, L.hash_mask);
  for (int64_t probe = 0; probe <= L.hash_mask; ++probe) {
    const ulonglong2 e = __ldg(L.seg_hash + h);
    if (e.x == k) return (int64_t)e.y;
    if (e.x == ~0ull) return -1;
    h = (h + 1) & (uint64_t)L.hash_mask;
  }
  return -1;
}

// Staging buffer and touch bitmap of forward position t (two of each, by
// parity: a step reads position t's while it fills position t+1's).
__device__ __forceinline__ int32_t* fwd_stage(const FrontierState& S, int32_t t) { return (t & 1) ? S.stage_b : S.stage; }
__device__ __forceinline__ uint32_t* fwd_touch(const FrontierState& S, int32_t t) { return (t & 1) ? S.touch_b : S.touch; }

// Touch q in string bitmap tb: true for the first toucher only.
__device__ __forceinline__ bool touch_first(uint32_t* tb, int32_t q) {
  const uint32_t bit = 1u << (q & 31);
  return (atomicOr(tb + (q >> 5), bit) & bit) == 0u;
}
__device__ __forceinline__ void untouch(uint32_t* tb, int32_t q) { atomicAnd(tb + (q >> 5), ~(1u << (q & 31))); }

// The last block of a kernel to finish hands out consecutive ranges, in step
// order, to the step's tokens: prefix sums of their counts cnt[p] from
// *top (or 0), written per slot (slot_out) and, for the pool, per token
// (base_out, cnt_out); rng_out[0..1] gets the step's [begin, end) and *top
// the end.  The tokens from the first whose range would pass `cap` on get
// empty ranges (slot base INT64_MAX, so no flat index maps to them) and
// raise error bit 1: every status of the run then reports FST_ERR_OOM.
// Each thread takes RPT consecutive slots (their loads issued together),
// then the block scans the thread totals (two warp levels); RPT * KT slots
// per round.
constexpr int RPT = 4;

__device__ void ranges_last_block(const TokenView& T, const StepView& V, const FrontierState& S,
                                  const uint32_t* cnt, int64_t* top, int64_t cap, int64_t* slot_out,
                                  int64_t* base_out, int32_t* cnt_out, int64_t* rng_out) {
  __shared__ int last;
  __shared__ long long wsum[KT / 32];
  __shared__ long long first_bad, carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(S.flags, 1u) == gridDim.x - 1u);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const long long begin = top ? (long long)__ldcg(top) : 0ll;
  if (threadIdx.x == 0) {
    first_bad = (long long)INT64_MAX;
    carry = begin;
  }
  __syncthreads();
  for (int32_t c = 0; c < V.n; c += KT * RPT) {
    const int32_t k0 = c + (int32_t)threadIdx.x * RPT;
    int32_t pv[RPT];
    long long mv[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) pv[i] = k0 + i < V.n ? __ldg(T.step_tok + V.slot0 + k0 + i) : -1;
    long long run = 0;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      mv[i] = pv[i] >= 0 ? (long long)__ldcg(cnt + pv[i]) : 0ll;
      run += mv[i];
    }
    long long incl = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long o = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += o;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    long long base = carry, round = 0;
#pragma unroll
    for (int w = 0; w < KT / 32; ++w) {
      base += w < warp ? wsum[w] : 0ll;
      round += wsum[w];
    }
    base += incl - run;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      if (pv[i] < 0) continue;
      const long long m = mv[i];
      const bool fit = base + m <= (long long)cap;
      if (!fit) atomicMin(&first_bad, base);
      slot_out[V.slot0 + k0 + i] = fit ? base : INT64_MAX;
      if (base_out) base_out[pv[i]] = fit ? base : 0;
      if (cnt_out) cnt_out[pv[i]] = fit ? (int32_t)m : 0;
      base += m;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += round;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long end = carry < first_bad ? carry : first_bad;
    if (first_bad != (long long)INT64_MAX) atomicOr(S.flags + 1, 1u);
    rng_out[0] = begin;
    rng_out[1] = end;
    if (top) *top = end;
    S.flags[0] = 0u;
  }
}

// ======================================================================
// Block-flattened arc walks.  Thread i of a block owns the arcs
// [e0_i, e0_i + len_i) of one segment; the block visits the arcs of all its
// threads 256 at a time, so a hub's segment (hundreds of arcs out of one
// state on one symbol) spreads over the block instead of holding up one
// thread.  Reductions go through shared-memory atomics on order-independent
// operations (max, integer add), so their results do not depend on which
// thread met which arc.
// ======================================================================
template <class Ctx>
struct BlockScratch {
  int32_t excl[KT];   // first flat arc of each thread's segment
  int32_t e0[KT];
  int32_t wsum[KT / 32];
  unsigned long long acc[KT];
  Ctx ctx[KT];
};

// Exclusive prefix of len over the block; *total gets the sum.
__device__ __forceinline__ int32_t block_excl(int32_t len, int32_t* wsum, int32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = len;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t o = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int32_t base = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < KT / 32; ++w) {
    const int32_t x = wsum[w];
    base += w < warp ? x : 0;
    tot += x;
  }
  *total = tot;
  return base + incl - len;
}

// Thread owning flat arc a: the last thread whose first flat arc is <= a.
__device__ __forceinline__ int block_owner(const int32_t* excl, int32_t a) {
  int o = 0;
#pragma unroll
  for (int step = KT / 2; step >= 1; step >>= 1)
    if (excl[o + step] <= a) o += step;
  return o;
}

// visit(e, ctx) for every arc of every thread's segment.
template <class Ctx, class F>
__device__ __forceinline__ void block_visit(BlockScratch<Ctx>& sh, int32_t e0, int32_t len, const Ctx& mine,
                                            F visit) {
  int32_t total;
  const int32_t ex = block_excl(len, sh.wsum, &total);
  sh.excl[threadIdx.x] = ex;
  sh.e0[threadIdx.x] = e0;
  sh.ctx[threadIdx.x] = mine;
  __syncthreads();
  for (int32_t a = threadIdx.x; a < total; a += KT) {
    const int o = block_owner(sh.excl, a);
    visit(sh.e0[o] + (a - sh.excl[o]), sh.ctx[o]);
  }
  __syncthreads();
}

// Reductions over each thread's segment: Op maps a value to a 64-bit key,
// combines keys atomically and maps the result back.
struct RedKey {  // Viterbi: max of packed (score, ~position) keys
  typedef unsigned long long T;
  static __device__ __forceinline__ unsigned long long key(T v) { return v; }
  static __device__ __forceinline__ T value(unsigned long long k) { return k; }
  static __device__ __forceinline__ void atomic(unsigned long long* a, unsigned long long k) { if (k) atomicMax(a, k); }
};
struct RedMax {  // max of floats through their order-preserving keys (0 = nothing)
  typedef float T;
  static __device__ __forceinline__ unsigned long long key(T v) {
    return v == __int_as_float(0xff800000) ? 0ull : (unsigned long long)fkey(v);
  }
  static __device__ __forceinline__ T value(unsigned long long k) {
    return k ? fkey_inv((uint32_t)k) : __int_as_float(0xff800000);
  }
  static __device__ __forceinline__ void atomic(unsigned long long* a, unsigned long long k) { if (k) atomicMax(a, k); }
};
struct RedSum {  // exact integer sum
  typedef unsigned long long T;
  static __device__ __forceinline__ unsigned long long key(T v) { return v; }
  static __device__ __forceinline__ T value(unsigned long long k) { return k; }
  static __device__ __forceinline__ void atomic(unsigned long long* a, unsigned long long k) { if (k) atomicAdd(a, k); }
};

template <class Op, class Ctx, class F>
__device__ __forceinline__ typename Op::T block_reduce(BlockScratch<Ctx>& sh, int32_t e0, int32_t len,
                                                       const Ctx& mine, F value) {
  int32_t total;
  const int32_t ex = block_excl(len, sh.wsum, &total);
  sh.excl[threadIdx.x] = ex;
  sh.e0[threadIdx.x] = e0;
  sh.ctx[threadIdx.x] = mine;
  sh.acc[threadIdx.x] = 0ull;
  __syncthreads();
  for (int32_t a = threadIdx.x; a < total; a += KT) {
    const int o = block_owner(sh.excl, a);
    Op::atomic(&sh.acc[o], Op::key(value(sh.e0[o] + (a - sh.excl[o]), sh.ctx[o])));
  }
  __syncthreads();
  const typename Op::T r = Op::value(sh.acc[threadIdx.x]);
  __syncthreads();
  return r;
}

// exp(v - m), v <= m, as a 2^-40 fixed-point integer: sums of these are exact
// and so independent of the order in which the block happens to add them
constexpr double FIX_ONE = 1099511627776.0;  // 2^40
__device__ __forceinline__ unsigned long long fix_exp(float v, float m) {
  return v == __int_as_float(0xff800000) ? 0ull : __double2ull_rn((double)__expf(v - m) * FIX_ONE);
}
__device__ __forceinline__ float fix_log_sum(float m, unsigned long long s) {
  return (m == __int_as_float(0xff800000) || s == 0ull) ? __int_as_float(0xff800000)
                                                        : m + (float)log((double)s / FIX_ONE);
}

// Per-thread context the arc walks need from the owner thread.
struct TokCtx {
  int32_t p, b;
  float sh;  // a step shift (forward m_{t-1} or backward e_t), or unused
  float m;   // the segment's maximum (second pass of a log-sum-exp)
};

// ======================================================================
// Expand (Alg. 1 / Alg. 2 forward loops, restricted to live sources).
// Sources: the pool entries of position t-1 (their token's successor is the
// token that reads w_t), or every start state for every token at t = 1.
// ======================================================================
__global__ void __launch_bounds__(KT) k_expand(LayoutView Lb, TokenView T, StepView V, FrontierState S) {
  __shared__ BlockScratch<TokCtx> sh;
  const int lane = threadIdx.x & 31;
  const int64_t R0 = V.t == 1 ? 0 : S.step_rng[2 * V.x_t];
  const int64_t R1 = V.t == 1 ? (int64_t)V.n * S.nstart : S.step_rng[2 * V.x_t + 1];
  for (int64_t cb = R0 + (int64_t)blockIdx.x * KT; cb < R1; cb += (int64_t)gridDim.x * KT) {
    const int64_t c0 = cb + (int64_t)(threadIdx.x & ~31);  // this warp's 32 entries (block-uniform loop)
    const int64_t j = c0 + lane;
    int32_t p = -1, q = -1;
    if (V.t == 1) {
      if (j < R1) {
        p = __ldg(T.step_tok + V.slot0 + (int32_t)(j / S.nstart));
        q = __ldg(S.start_q + (int32_t)(j % S.nstart));
      }
    } else {
      const int64_t* base = S.slot_base + V.x_slot0;
      const int32_t k0 = warp_owner(base, V.x_n, c0);
      if (j < R1) {
        const int32_t pp = __ldg(T.step_tok + V.x_slot0 + lane_owner(base, V.x_n, k0, j));
        if (S.bw_n[__ldg(T.b + pp)] >= V.t) {  // the string goes on to position t
          p = pp + 1;
          q = S.pool_q[j];
        }
      }
    }
    // the source's arcs on w_t: its segment of the source-segmented layout
    int32_t e0 = 0, len = 0;
    TokCtx me{p, 0, 0.f, 0.f};
    if (p >= 0 && q >= 0) {
      const int64_t sg = find_seg(Lb, __ldg(T.sym + p), q);
      if (sg >= 0) {
        e0 = __ldg(Lb.seg_pos + sg);
        len = __ldg(Lb.seg_len + sg);
        me.b = __ldg(T.b + p);
      }
    }
    block_visit(sh, e0, len, me, [&](int32_t e, const TokCtx& c) {
      const int32_t d = __ldg(Lb.other + e);
      if (touch_first(fwd_touch(S, V.t) + (int64_t)c.b * S.W, d))
        fwd_stage(S, V.t)[__ldg(T.stf + c.p) + atomicAdd(S.scnt_f + c.p, 1u)] = __ldg(Lb.xseg + e);
    });
  }
  ranges_last_block(T, V, S, S.scnt_f, S.pool_top, S.pool_cap, S.slot_base, S.pool_base, S.pool_cnt,
                    S.step_rng + 2 * V.t);
}

// Flat entry j of the reduce at position t: token p and its staging index i.
struct Entry {
  int32_t p, i;
};
__device__ __forceinline__ Entry step_entry(const TokenView& T, const StepView& V, const int64_t* slot_base,
                                            int32_t k0, int64_t j) {
  const int32_t k = lane_owner(slot_base + V.slot0, V.n, k0, j);
  Entry x;
  x.p = __ldg(T.step_tok + V.slot0 + k);
  x.i = (int32_t)(j - __ldcg(slot_base + V.slot0 + k));
  return x;
}

// ======================================================================
// One forward position, fused (Alg. 1 inner max, Sec. 5.1; Alg. 2 forward
// loop, Sec. 5.2): reduce the staged destination segments of position t
// into frontier entries, then expand every new live state into the
// segments of position t+1 (the next token of its string) right away.
// ======================================================================
// Expand live state q (just computed for token p at position t) into the
// segments of position t+1: returns its arcs on w_{t+1}.
__device__ __forceinline__ void next_arcs(const LayoutView& Lb, const TokenView& T, const FrontierState& S,
                                          int32_t t, int32_t p, int32_t b, int32_t q, int32_t* e0, int32_t* len) {
  *e0 = 0;
  *len = 0;
  if (q < 0 || S.bw_n[b] <= t) return;  // dead, or the string ends at t
  const int64_t sg = find_seg(Lb, __ldg(T.sym + p + 1), q);
  if (sg < 0) return;
  *e0 = __ldg(Lb.seg_pos + sg);
  *len = __ldg(Lb.seg_len + sg);
}

template <bool FWD>
__device__ __forceinline__ void fwd_position(const LayoutView& Lf, const LayoutView& Lb, const TokenView& T,
                                             const StepView& V, const FrontierState& S, BlockScratch<TokCtx>& sh) {
  const int lane = threadIdx.x & 31;
  const uint32_t tag_base = *S.epoch + S.tok0;
  const int32_t t = V.t;
  const int64_t R0 = S.step_rng[2 * t], R1 = S.step_rng[2 * t + 1];
  const int32_t* stg = fwd_stage(S, t);
  uint32_t* tch = fwd_touch(S, t);
  for (int64_t cb = R0 + (int64_t)blockIdx.x * KT; cb < R1; cb += (int64_t)gridDim.x * KT) {
    const int64_t c0 = cb + (int64_t)(threadIdx.x & ~31);  // this warp's 32 entries (block-uniform loop)
    const int32_t k0 = warp_owner(S.slot_base + V.slot0, V.n, c0);
    const int64_t j = c0 + lane;
    const bool act = j < R1;
    int32_t d = 0, e0 = 0, len = 0, sg = 0;
    TokCtx me{0, 0, 0.f, 0.f};
    if (act) {
      const Entry x = step_entry(T, V, S.slot_base, k0, j);
      me.p = x.p;
      me.b = __ldg(T.b + x.p);
      me.sh = (FWD && t > 1) ? decode_max(S.mkey[x.p - 1]) : 0.f;
      sg = stg[__ldg(T.stf + x.p) + x.i];
      d = __ldg(Lf.seg_state + sg);
      untouch(tch + (int64_t)me.b * S.W, d);
      if (me.sh != neg_inf()) {
        e0 = __ldg(Lf.seg_pos + sg);
        len = __ldg(Lf.seg_len + sg);
      }
    }
    // the value of source q on arc e, as the previous position left it
    auto src_value = [&](int32_t e, const TokCtx& c) {
      const int32_t q = __ldg(Lf.other + e);
      return (t == 1) ? __ldg(S.theta_s + q)
                      : tagged_value(__ldg(S.alpha + ((int64_t)c.b * 2 + ((t - 1) & 1)) * S.Q + q),
                                     tag_base + (uint32_t)(c.p - 1));
    };
    int32_t live = -1;  // the entry's state if its value is finite
    if (!FWD) {
      const unsigned long long best = block_reduce<RedKey>(sh, e0, len, me, [&](int32_t e, const TokCtx& c) {
        const float cand = __fadd_rn(src_value(e, c), __ldg(Lf.theta + e));
        return cand == neg_inf() ? 0ull
                                 : (((unsigned long long)fkey(cand) << 32) | (unsigned long long)(~(uint32_t)e));
      });
      if (act) {
        if (best)
          S.alpha[((int64_t)me.b * 2 + (t & 1)) * S.Q + d] =
              tagged_make(fkey_inv((uint32_t)(best >> 32)), tag_base + (uint32_t)me.p);
        S.pool_q[j] = best ? d : -1;
        S.pool_x[j] = best ? (int32_t)(~(uint32_t)best) : -1;
        live = best ? d : -1;
      }
    } else {
      auto value = [&](int32_t e, const TokCtx& c) {
        const float a = src_value(e, c);
        return a == neg_inf() ? neg_inf() : (a - c.sh) + __ldg(Lf.theta + e);
      };
      // log-sum-exp in two order-independent passes: max, then the
      // fixed-point sum of exp(v - max)
      me.m = block_reduce<RedMax>(sh, e0, len, me, value);
      const unsigned long long su = block_reduce<RedSum>(
          sh, e0, me.m == neg_inf() ? 0 : len, me, [&](int32_t e, const TokCtx& c) { return fix_exp(value(e, c), c.m); });
      if (act) {
        const float r = fix_log_sum(me.m, su);
        if (r != neg_inf()) {
          S.alpha[((int64_t)me.b * 2 + (t & 1)) * S.Q + d] = tagged_make(r, tag_base + (uint32_t)me.p);
          atomicMax(S.mkey + me.p, fkey(r));
        }
        S.pool_q[j] = r != neg_inf() ? d : -1;
        S.pool_x[j] = sg;
        S.pool_v[j] = r;
        live = r != neg_inf() ? d : -1;
      }
    }
    // expand the new live state into position t+1
    int32_t xe0 = 0, xlen = 0;
    if (act && V.x_n > 0) next_arcs(Lb, T, S, t, me.p, me.b, live, &xe0, &xlen);
    const TokCtx nx{me.p + 1, me.b, 0.f, 0.f};
    int32_t* nstg = fwd_stage(S, t + 1);
    uint32_t* ntch = fwd_touch(S, t + 1);
    block_visit(sh, xe0, xlen, nx, [&](int32_t e, const TokCtx& c) {
      const int32_t dn = __ldg(Lb.other + e);
      if (touch_first(ntch + (int64_t)c.b * S.W, dn))
        nstg[__ldg(T.stf + c.p) + atomicAdd(S.scnt_f + c.p, 1u)] = __ldg(Lb.xseg + e);
    });
  }
  // pool ranges of position t+1's tokens
  if (V.x_n > 0) {
    StepView Vn = V;
    Vn.t = V.x_t;
    Vn.n = V.x_n;
    Vn.slot0 = V.x_slot0;
    ranges_last_block(T, Vn, S, S.scnt_f, S.pool_top, S.pool_cap, S.slot_base, S.pool_base, S.pool_cnt,
                      S.step_rng + 2 * Vn.t);
  }
}

__global__ void __launch_bounds__(KT) k_vit_step(LayoutView Lf, LayoutView Lb, TokenView T, StepView V,
                                                 FrontierState S) {
  __shared__ BlockScratch<TokCtx> sh;
  fwd_position<false>(Lf, Lb, T, V, S, sh);
}

__global__ void __launch_bounds__(KT) k_fwd_step(LayoutView Lf, LayoutView Lb, TokenView T, StepView V,
                                                 FrontierState S) {
  __shared__ BlockScratch<TokCtx> sh;
  fwd_position<true>(Lf, Lb, T, V, S, sh);
}

// ======================================================================
// Backward expand fused with the posteriors (Alg. 2 backward and count
// loops; Sec. 5.2).  For each live state q of position t (finite forward
// value, a pool entry) whose backward value beta_t[q] is finite, every arc
// e into q on w_t with a finite forward value at its source gets
//   gamma_t(e) = exp(alpha_{t-1}[src] + theta_e + beta_t[q] - log Z),
// and its source is staged for the backward value at t-1.  Sources whose
// forward value is -inf are never staged: every posterior through them is
// zero, and no later backward step reads their backward value.
// ======================================================================
__device__ __forceinline__ void add_count(const CountView& C, int32_t e, float g) {
  if (C.batched) {
    atomicAdd(C.cnt64 + e, (double)g);
  } else {
    // compensated float32 summation (one string: one writer per arc and step)
    const float s0 = C.cnt[e], cmp = C.comp[e];
    const float y = __fsub_rn(g, cmp);
    const float s1 = __fadd_rn(s0, y);
    C.comp[e] = __fsub_rn(__fsub_rn(s1, s0), y);
    C.cnt[e] = s1;
  }
}

// owner context of the backward expand: token, string, mprev, and the
// float64 exponent offset (ub - e_t) + K of its destination
struct BwdCtx {
  int32_t p, b;
  float mprev, gw;
  double off;
};

__global__ void __launch_bounds__(KT) k_bwd_expand(LayoutView Lf, TokenView T, StepView V, FrontierState S,
                                                   CountView C) {
  __shared__ BlockScratch<BwdCtx> sh;
  const int lane = threadIdx.x & 31;
  const uint32_t tag_base = *S.epoch + S.tok0;
  const int32_t t = V.t;
  const int64_t R0 = S.step_rng[2 * t], R1 = S.step_rng[2 * t + 1];
  for (int64_t cb = R0 + (int64_t)blockIdx.x * KT; cb < R1; cb += (int64_t)gridDim.x * KT) {
    const int64_t c0 = cb + (int64_t)(threadIdx.x & ~31);  // this warp's 32 entries (block-uniform loop)
    const int32_t k0 = warp_owner(S.slot_base + V.slot0, V.n, c0);
    const int64_t j = c0 + lane;
    int32_t e0 = 0, len = 0;
    BwdCtx me{0, 0, 0.f, 0.f, 0.0};
    if (j < R1) {
      const Entry x = step_entry(T, V, S.slot_base, k0, j);
      const int32_t p = x.p, b = __ldg(T.b + p), n = S.bw_n[b];
      const double lz = S.logz[b];
      // shifts: e_t = this step's backward maximum, m_{t-1} the forward one;
      // K = C_{t-1} + E_t - log Z collects the float64 running sums
      const float et = (t == n) ? 0.f : decode_max(S.ekey[p]);
      const double tE = (t == n) ? 0.0 : S.esum[p + 1] + (double)et;
      if (x.i == 0 && lz != -INFINITY) S.esum[p] = tE;  // E_t, read by the step at t-1
      const double K = ((t == 1) ? 0.0 : S.csum[p - 1]) + tE - lz;
      const float mprev = (t == 1) ? 0.f : decode_max(S.mkey[p - 1]);
      const int32_t q = S.pool_q[j];
      if (lz != -INFINITY && q >= 0 && et != neg_inf() && mprev != neg_inf()) {
        const float ub = (t == n) ? __ldg(S.theta_f + q)
                                  : tagged_value(__ldg(S.beta + ((int64_t)b * 2 + (t & 1)) * S.Q + q),
                                                 tag_base + (uint32_t)p);
        if (ub != neg_inf()) {
          const int32_t sg = S.pool_x[j];
          e0 = __ldg(Lf.seg_pos + sg);
          len = __ldg(Lf.seg_len + sg);
          me = BwdCtx{p, b, mprev, S.gweight ? S.gweight[b] : 1.f, ((double)ub - (double)et) + K};
        }
      }
    }
    block_visit(sh, e0, len, me, [&](int32_t e, const BwdCtx& c) {
      const int32_t src = __ldg(Lf.other + e);
      const float ra = (t == 1) ? __ldg(S.theta_s + src)
                                : tagged_value(__ldg(S.alpha + ((int64_t)c.b * 2 + ((t - 1) & 1)) * S.Q + src),
                                               tag_base + (uint32_t)(c.p - 1));
      const float th = __ldg(Lf.theta + e);
      if (ra == neg_inf() || th == neg_inf()) return;
      // the exponent adds terms of either sign and tens in size that cancel
      // to a small number: formed in float64
      const double ex = ((double)ra - (double)c.mprev) + (double)th + c.off;
      add_count(C, e, __expf((float)ex) * c.gw);
      if (t >= 2 && touch_first(S.touch + (int64_t)c.b * S.W, src))
        S.stage[__ldg(T.stb + c.p) + atomicAdd(S.scnt_b + c.p, 1u)] = __ldg(Lf.xseg + e);
    });
  }
  if (t >= 2)
    ranges_last_block(T, V, S, S.scnt_b, nullptr, INT64_MAX, S.bslot_base, nullptr, nullptr, S.bstep_rng + 2 * t);
}

// ======================================================================
// Backward reduce: beta_{t-1}[q] = LSE over the arcs q -> q' on w_t of
// theta + beta_t[q'] - e_t, for every staged source segment (q, w_t).  The
// same launch restores the forward values of position t-2 into the dense
// frontier (their parity buffer held alpha_t, which nothing reads any more);
// the next backward expand needs them.
// ======================================================================
__global__ void __launch_bounds__(KT) k_bwd_reduce(LayoutView Lb, TokenView T, StepView V, FrontierState S) {
  __shared__ BlockScratch<TokCtx> sh;
  const int lane = threadIdx.x & 31;
  const uint32_t tag_base = *S.epoch + S.tok0;
  const int32_t t = V.t;
  if (V.x_n > 0) {
    const int64_t R0 = S.step_rng[2 * V.x_t], R1 = S.step_rng[2 * V.x_t + 1];
    for (int64_t cb = R0 + (int64_t)blockIdx.x * KT; cb < R1; cb += (int64_t)gridDim.x * KT) {
      const int64_t c0 = cb + (int64_t)(threadIdx.x & ~31);
      const int64_t* base = S.slot_base + V.x_slot0;
      const int32_t k0 = warp_owner(base, V.x_n, c0);
      const int64_t j = c0 + lane;
      if (j >= R1) continue;
      const int32_t p2 = __ldg(T.step_tok + V.x_slot0 + lane_owner(base, V.x_n, k0, j));
      const int32_t q = S.pool_q[j];
      if (q >= 0)
        S.alpha[((int64_t)__ldg(T.b + p2) * 2 + (V.x_t & 1)) * S.Q + q] =
            tagged_make(S.pool_v[j], tag_base + (uint32_t)p2);
    }
  }
  const int64_t R1 = S.bstep_rng[2 * t + 1];
  for (int64_t cb = (int64_t)blockIdx.x * KT; cb < R1; cb += (int64_t)gridDim.x * KT) {
    const int64_t c0 = cb + (int64_t)(threadIdx.x & ~31);
    const int32_t k0 = warp_owner(S.bslot_base + V.slot0, V.n, c0);
    const int64_t j = c0 + lane;
    const bool act = j < R1;
    int32_t q = 0, e0 = 0, len = 0;
    TokCtx me{0, 0, 0.f, 0.f};
    int32_t n = 0;
    if (act) {
      const Entry x = step_entry(T, V, S.bslot_base, k0, j);
      me.p = x.p;
      me.b = __ldg(T.b + x.p);
      n = S.bw_n[me.b];
      me.sh = (t == n) ? 0.f : decode_max(S.ekey[x.p]);
      const int32_t sg = S.stage[__ldg(T.stb + x.p) + x.i];
      q = __ldg(Lb.seg_state + sg);
      untouch(S.touch + (int64_t)me.b * S.W, q);
      if (me.sh != neg_inf()) {
        e0 = __ldg(Lb.seg_pos + sg);
        len = __ldg(Lb.seg_len + sg);
      }
    }
    auto value = [&](int32_t e, const TokCtx& c) {
      const int32_t d = __ldg(Lb.other + e);
      const float ub = (t == S.bw_n[c.b]) ? __ldg(S.theta_f + d)
                                          : tagged_value(__ldg(S.beta + ((int64_t)c.b * 2 + (t & 1)) * S.Q + d),
                                                         tag_base + (uint32_t)c.p);
      return ub == neg_inf() ? neg_inf() : __ldg(Lb.theta + e) + (ub - c.sh);
    };
    me.m = block_reduce<RedMax>(sh, e0, len, me, value);
    const unsigned long long su = block_reduce<RedSum>(
        sh, e0, me.m == neg_inf() ? 0 : len, me, [&](int32_t e, const TokCtx& c) { return fix_exp(value(e, c), c.m); });
    if (!act) continue;
    const float u = fix_log_sum(me.m, su);
    if (u != neg_inf()) {
      S.beta[((int64_t)me.b * 2 + ((t - 1) & 1)) * S.Q + q] = tagged_make(u, tag_base + (uint32_t)(me.p - 1));
      atomicMax(S.ekey + me.p - 1, fkey(u));
    }
  }
}

// ======================================================================
// Epilogues: final reductions (Alg. 1 return line; Alg. 2 Z), backtrace
// (Sec. 5.1), and counts back to caller arc order.  A string's candidates
// are the live states of its last position (its pool entries), or the
// start states when it is empty.
// ======================================================================
__global__ void __launch_bounds__(FT) k_vit_final(FrontierState S, float* __restrict__ scores,
                                                  int32_t* __restrict__ qfinal, int32_t* __restrict__ status) {
  __shared__ unsigned long long red[FT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = blockIdx.x;
  const int32_t n = S.bw_n[b];
  const int64_t p = S.bw_off[b] + n - 1;
  const unsigned long long* ab = S.alpha + (b * 2 + (n & 1)) * S.Q;
  const uint32_t tg = *S.epoch + S.tok0 + (uint32_t)p;
  const int32_t* cand = n == 0 ? S.start_q : S.pool_q + S.pool_base[p];
  const int32_t ncand = n == 0 ? S.nstart : S.pool_cnt[p];
  unsigned long long best = 0ull;
  for (int32_t i = threadIdx.x; i < ncand; i += FT) {
    const int32_t q = cand[i];
    if (q < 0) continue;
    const float a = n == 0 ? __ldg(S.theta_s + q) : tagged_value(ab[q], tg);
    const float c = __fadd_rn(a, __ldg(S.theta_f + q));
    if (c != neg_inf()) {
      const unsigned long long key = ((unsigned long long)fkey(c) << 32) | (unsigned long long)(~(uint32_t)q);
      best = key > best ? key : best;
    }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(FULL, best, d);
    best = o > best ? o : best;
  }
  if (lane == 0) red[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < FT / 32; ++w) best = red[w] > best ? red[w] : best;
    const bool oom = (S.flags[1] & 1u) != 0u;
    scores[b] = (best && !oom) ? fkey_inv((uint32_t)(best >> 32)) : neg_inf();
    qfinal[b] = (best && !oom) ? (int32_t)(~(uint32_t)best) : -1;
    if (status) status[b] = oom ? FST_ERR_OOM : (best ? FST_OK : FST_ERR_NO_PATH);
  }
}

// One warp per string: at each position the warp finds the state among the
// token's pool entries and follows its backpointer.
__global__ void k_backtrace(LayoutView Lf, FrontierState S, const int32_t* __restrict__ olabel_by_id, int32_t Bw,
                            const int32_t* __restrict__ qfinal, int32_t* __restrict__ paths,
                            int32_t* __restrict__ olabels) {
  const int lane = threadIdx.x & 31;
  const int64_t b = warp_id_global();
  if (b >= Bw) return;
  const int32_t n = S.bw_n[b];
  const int64_t off = S.bw_off[b];
  int32_t q = qfinal[b];
  if (q < 0) {
    for (int32_t t = lane; t < n; t += 32) {
      paths[off + t] = -1;
      if (olabels) olabels[off + t] = -1;
    }
    return;
  }
  for (int32_t t = n; t >= 1; --t) {
    const int64_t p = off + t - 1;
    const int64_t pb = S.pool_base[p];
    const int32_t pc = S.pool_cnt[p];
    int32_t pos = -1;
    for (int32_t c = 0; c < pc; c += 32) {
      const int32_t i = c + lane;
      const uint32_t hit = __ballot_sync(FULL, i < pc && S.pool_q[pb + i] == q);
      if (hit) {
        pos = S.pool_x[pb + c + __ffs(hit) - 1];
        break;
      }
    }
    if (pos < 0) {  // cannot happen for a state on the best path; leave a marker
      for (int32_t u = lane; u < t; u += 32) {
        paths[off + u] = -1;
        if (olabels) olabels[off + u] = -1;
      }
      break;
    }
    const int32_t id = __ldg(Lf.arc_id + pos);
    if (lane == 0) {
      paths[p] = id;
      if (olabels) olabels[p] = olabel_by_id[id];
    }
    q = __ldg(Lf.other + pos);
  }
}

// log Z of one string (Alg. 2, Z): C_{n-1} + log sum_q exp(r_n[q] + final[q]).
// Warp 0 first writes the running normalisers C_t (a warp scan, float64).
__global__ void __launch_bounds__(FT) k_fb_final(FrontierState S, double* __restrict__ logz,
                                                 int32_t* __restrict__ status) {
  __shared__ float red_m[FT / 32];
  __shared__ unsigned long long red_lo[FT], red_hi[FT];
  __shared__ double c_prev;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = blockIdx.x;
  const int32_t n = S.bw_n[b];
  const int64_t off = S.bw_off[b];
  if (warp == 0) {
    // C_t = sum_{s<=t} m_s (-inf once some position has no live state)
    if (lane == 0) c_prev = 0.0;
    __syncwarp();
    double carry = 0.0;
    for (int32_t t0 = 0; t0 < n; t0 += 32) {
      const int32_t t = t0 + lane;
      double v = 0.0;
      if (t < n) {
        const float m = decode_max(S.mkey[off + t]);
        v = (m == neg_inf()) ? -INFINITY : (double)m;
      }
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const double o = __shfl_up_sync(FULL, v, d);
        if (lane >= d) v += o;
      }
      v += carry;
      if (t < n) S.csum[off + t] = v;
      if (t == n - 2) c_prev = v;
      carry = __shfl_sync(FULL, v, 31);
    }
  }
  const int64_t p = off + n - 1;
  const int32_t* cand = n == 0 ? S.start_q : S.pool_q + S.pool_base[p];
  const int32_t ncand = n == 0 ? S.nstart : S.pool_cnt[p];
  auto value = [&](int32_t i) -> float {
    const int32_t q = cand[i];
    if (q < 0) return neg_inf();
    const float a = n == 0 ? __ldg(S.theta_s + q) : S.pool_v[S.pool_base[p] + i];
    return __fadd_rn(a, __ldg(S.theta_f + q));
  };
  // the candidates sit in the pool in scheduling order: the sum is made
  // order-independent (bitwise repeatable) by adding exp(v - max) as
  // integers, in units of 2^-62
  float mx = neg_inf();
  for (int32_t i = threadIdx.x; i < ncand; i += FT) mx = fmaxf(mx, value(i));
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, d));
  if (lane == 0) red_m[warp] = mx;
  __syncthreads();
  for (int w = 0; w < FT / 32; ++w) mx = fmaxf(mx, red_m[w]);
  unsigned long long lo = 0ull, hi = 0ull;  // 128-bit accumulator
  if (mx != neg_inf()) {
    for (int32_t i = threadIdx.x; i < ncand; i += FT) {
      const float v = value(i);
      if (v == neg_inf()) continue;
      const unsigned long long u = __double2ull_rn((double)__expf(v - mx) * 4611686018427387904.0);  // 2^62
      lo += u;
      hi += (lo < u) ? 1ull : 0ull;
    }
  }
  red_lo[threadIdx.x] = lo;
  red_hi[threadIdx.x] = hi;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < FT; ++i) {
      lo += red_lo[i];
      hi += red_hi[i] + ((lo < red_lo[i]) ? 1ull : 0ull);
    }
    const double sum = ((double)hi * 18446744073709551616.0 + (double)lo) * 2.168404344971009e-19;  // 2^64, 2^-62
    const bool oom = (S.flags[1] & 1u) != 0u;
    const double cp = c_prev;
    double lz = -INFINITY;
    if (!oom && mx != neg_inf() && cp != -INFINITY) lz = cp + (double)mx + log(sum);
    logz[b] = lz;
    if (status) status[b] = oom ? FST_ERR_OOM : ((lz == -INFINITY) ? FST_ERR_NO_PATH : FST_OK);
  }
}

__global__ void k_counts_out(const int32_t* __restrict__ arc_id, int64_t P, CountView C, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const int32_t k = arc_id[i];
  if (k < 0) return;
  out[k] = C.batched ? (float)C.cnt64[i] : __fsub_rn(C.cnt[i], C.comp[i]);
}

inline int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return FST_OK;
}

// Step kernels are grid-stride loops over flat entries; the grid is the
// driver's estimate, at most what can be resident at once.
template <class K>
inline unsigned step_grid(K kernel, int* cache, const StepView& V) {
  if (*cache <= 0) {
    int dev = 0, sms = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, KT, 0) != cudaSuccess || nb <= 0 || sms <= 0) {
      (void)cudaGetLastError();
      sms = 1;
      nb = 1;
    }
    *cache = sms * nb;
  }
  return (unsigned)std::max(1, std::min(V.blocks, *cache));
}

int g_grid[5] = {0, 0, 0, 0, 0};

}  // namespace

int launch_expand(const LayoutView& Lb, const TokenView& T, const StepView& V, const FrontierState& S, cudaStream_t s) {
  k_expand<<<step_grid(k_expand, &g_grid[0], V), KT, 0, s>>>(Lb, T, V, S);
  return check_launch("k_expand");
}

int launch_vit_step(const LayoutView& Lf, const LayoutView& Lb, const TokenView& T, const StepView& V,
                    const FrontierState& S, cudaStream_t s) {
  k_vit_step<<<step_grid(k_vit_step, &g_grid[1], V), KT, 0, s>>>(Lf, Lb, T, V, S);
  return check_launch("k_vit_step");
}

int launch_fwd_step(const LayoutView& Lf, const LayoutView& Lb, const TokenView& T, const StepView& V,
                    const FrontierState& S, cudaStream_t s) {
  k_fwd_step<<<step_grid(k_fwd_step, &g_grid[2], V), KT, 0, s>>>(Lf, Lb, T, V, S);
  return check_launch("k_fwd_step");
}

int launch_bwd_expand(const LayoutView& Lf, const TokenView& T, const StepView& V, const FrontierState& S,
                      const CountView& C, cudaStream_t s) {
  k_bwd_expand<<<step_grid(k_bwd_expand, &g_grid[3], V), KT, 0, s>>>(Lf, T, V, S, C);
  return check_launch("k_bwd_expand");
}

int launch_bwd_reduce(const LayoutView& Lb, const TokenView& T, const StepView& V, const FrontierState& S,
                      cudaStream_t s) {
  k_bwd_reduce<<<step_grid(k_bwd_reduce, &g_grid[4], V), KT, 0, s>>>(Lb, T, V, S);
  return check_launch("k_bwd_reduce");
}

int launch_vit_final(const FrontierState& S, int32_t Bw, float* scores, int32_t* qfinal, int32_t* status,
                     cudaStream_t s) {
  if (Bw <= 0) return FST_OK;
  k_vit_final<<<(unsigned)Bw, FT, 0, s>>>(S, scores, qfinal, status);
  return check_launch("k_vit_final");
}

int launch_backtrace(const LayoutView& Lf, const FrontierState& S, const int32_t* olabel_by_id, int32_t Bw,
                     const int32_t* qfinal, int32_t* paths, int32_t* olabels, cudaStream_t s) {
  if (Bw <= 0) return FST_OK;
  k_backtrace<<<(unsigned)((Bw + 7) / 8), 256, 0, s>>>(Lf, S, olabel_by_id, Bw, qfinal, paths, olabels);
  return check_launch("k_backtrace");
}

int launch_fb_final(const FrontierState& S, int32_t Bw, double* logz, int32_t* status, cudaStream_t s) {
  if (Bw <= 0) return FST_OK;
  k_fb_final<<<(unsigned)Bw, FT, 0, s>>>(S, logz, status);
  return check_launch("k_fb_final");
}

int launch_counts_out(const int32_t* arc_id_fwd, int64_t P, const CountView& C, float* out, cudaStream_t s) {
  if (P <= 0) return FST_OK;
  k_counts_out<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(arc_id_fwd, P, C, out);
  return check_launch("k_counts_out");
}

}  // namespace fstgpu
