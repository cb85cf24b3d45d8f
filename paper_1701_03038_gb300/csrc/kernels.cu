// kernels.cu -- the per-position relaxation kernels and their epilogues.
//
// For input position t the paper relaxes every arc of the slice
// delta[w_t] with one thread per arc and resolves collisions on a state
// with atomics: a packed 64-bit (probability | arc) atomicMax for Viterbi
// (Sec. 5.1) and an atomic log-add-exp for forward and backward (Sec. 5.2,
// Eq. 3).  Here one warp owns one 128-arc window of a segmented slice
// (see store.cu): each lane loads 4 arcs with two 16-byte loads, gathers the
// frontier, and the warp reduces every segment with a segmented shuffle
// scan.  Only a segment longer than a window is combined across warps: with
// the packed 64-bit atomicMax for Viterbi and with ordered per-window
// partials for log-sum-exp; the last warp to arrive finalises it.
//
// Values: Viterbi keys are (order-preserving float32 bits << 32) | ~arc
// position, so a 64-bit max picks the best score and, on ties, the lowest
// position -- the lowest arc id, because arcs of a segment are sorted by id.
// Forward and backward carry (max, scaled sum) pairs; each step's values are
// shifted by that step's maximum, with the running shift kept in float64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kernels.cuh"

namespace fstgpu {
namespace {

constexpr int KT = 256;  // threads per block of the step kernels
#ifndef KT_MIN_BLOCKS
#define KT_MIN_BLOCKS 3
#endif
#ifndef KT_MIN_BLOCKS_BWD
#define KT_MIN_BLOCKS_BWD 2
#endif


__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

struct MaxKey {
  typedef unsigned long long T;
  static __device__ __forceinline__ T identity() { return 0ull; }
  static __device__ __forceinline__ T combine(T a, T b) { return a > b ? a : b; }
  static __device__ __forceinline__ T shfl_up(T v, int d) { return __shfl_up_sync(FULL, v, d); }
};

// log-sum-exp pairs (M, S): the value M + log(S).
struct LogAdd {
  typedef float2 T;
  static __device__ __forceinline__ T identity() { return make_float2(__int_as_float(0xff800000), 0.f); }
  static __device__ __forceinline__ T combine(T a, T b) {
    if (a.x < b.x) { T c = a; a = b; b = c; }
    if (b.x == __int_as_float(0xff800000)) return a;
    return make_float2(a.x, a.y + b.y * __expf(b.x - a.x));
  }
  static __device__ __forceinline__ T shfl_up(T v, int d) {
    return make_float2(__shfl_up_sync(FULL, v.x, d), __shfl_up_sync(FULL, v.y, d));
  }
};

// Segmented inclusive scan over lanes: each lane contributes the aggregate
// of its last partial segment; `lane_head` = the lane contains a segment
// start.  Returns the aggregate from the lane's last segment start (or the
// window start) through this lane.
template <class Op>
__device__ __forceinline__ typename Op::T seg_scan_lanes(typename Op::T agg, bool lane_head, int lane) {
  const uint32_t hm = __ballot_sync(FULL, lane_head);
  const uint32_t le = hm & (0xffffffffu >> (31 - lane));
  const int start = le ? 31 - __clz(le) : 0;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    typename Op::T o = Op::shfl_up(agg, d);
    if (lane - d >= start) agg = Op::combine(o, agg);
  }
  return agg;
}

// Full segmented prefix at each of the lane's 4 arcs (bit j of h = arc j
// starts a segment).  At a segment's last arc this is the segment total.
template <class Op>
__device__ __forceinline__ void window_scan(const typename Op::T (&e)[APL], uint32_t h, int lane,
                                            typename Op::T (&full)[APL]) {
  typename Op::T p[APL];
  p[0] = e[0];
#pragma unroll
  for (int j = 1; j < APL; ++j) p[j] = ((h >> j) & 1u) ? e[j] : Op::combine(p[j - 1], e[j]);
  const typename Op::T incl = seg_scan_lanes<Op>(p[APL - 1], h != 0u, lane);
  typename Op::T carry = Op::shfl_up(incl, 1);
  if (lane == 0) carry = Op::identity();
  const int first = h ? __ffs(h) - 1 : APL;
#pragma unroll
  for (int j = 0; j < APL; ++j) full[j] = (j < first) ? Op::combine(carry, p[j]) : p[j];
}

// Work-list resolution.  A warp walks items item0, item0 + nwarps, ...; the
// group of the last item and, in lane j, the data of the group's j-th token
// stay in registers until an item falls outside the group.  Item, window and
// arc indices fit in 32 bits (padded arcs < 2^31 is enforced at build).
struct Group {
  int32_t g, sym, cnt, segbase;
  int32_t lo, hi, wbase;
};

__device__ __forceinline__ void find_group(const LayoutView& L, const WorkView& W, int32_t item, Group& G) {
  if (W.single) {
    G.g = 0; G.lo = 0; G.hi = (int32_t)W.nitems; G.sym = W.sym0; G.cnt = 1;
  } else {
    int lo = G.g >= 0 ? G.g + 1 : W.g0;  // items only grow inside a warp's walk
    int hi = W.g1 - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(W.grp_item + mid) <= item) lo = mid; else hi = mid - 1;
    }
    G.g = lo;
    G.lo = (int32_t)__ldg(W.grp_item + lo);
    G.hi = (lo + 1 < W.g1) ? (int32_t)__ldg(W.grp_item + lo + 1) : (int32_t)W.nitems;
    G.sym = __ldg(W.grp_sym + lo);
    G.cnt = __ldg(W.grp_cnt + lo);
  }
  G.wbase = (int32_t)__ldg(L.sym_win + G.sym);
  G.segbase = (int32_t)__ldg(L.sym_seg + G.sym);
}

__device__ __forceinline__ int32_t group_token(const WorkView& W, const Group& G, int lane) {
  return W.single ? W.p0 : __ldg(W.sorted_tok + __ldg(W.grp_first + G.g) + lane);
}

struct Win {
  int32_t w;
  int32_t seg, lseg, lwin0, lcnt;
  uint32_t h;   // this lane's head bits
  int32_t hb;   // heads of the window before this lane
};

__device__ __forceinline__ Win load_win(const LayoutView& L, int32_t w, int lane) {
  Win x;
  x.w = w;
  const int4 m0 = __ldg(reinterpret_cast<const int4*>(L.win + w));
  const uint4 m1 = __ldg(reinterpret_cast<const uint4*>(L.win + w) + 1);
  x.seg = m0.x; x.lseg = m0.y; x.lwin0 = m0.z; x.lcnt = m0.w;
  const int q = lane >> 3;
  const uint32_t word = q == 0 ? m1.x : (q == 1 ? m1.y : (q == 2 ? m1.z : m1.w));
  const int sh = (lane & 7) * 4;
  x.h = (word >> sh) & 0xFu;
  x.hb = __popc(word & ((1u << sh) - 1u)) + (q > 0 ? __popc(m1.x) : 0) + (q > 1 ? __popc(m1.y) : 0) +
         (q > 2 ? __popc(m1.z) : 0);
  return x;
}

__device__ __forceinline__ int32_t warp_id_global() { return (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }
__device__ __forceinline__ int32_t warps_total() { return (int32_t)((gridDim.x * blockDim.x) >> 5); }

__device__ __forceinline__ int64_t shfl64(int64_t v, int src) {
  return (int64_t)__shfl_sync(FULL, (long long)v, src);
}

__device__ __forceinline__ float decode_max(uint32_t k) { return k ? fkey_inv(k) : neg_inf(); }

__device__ __forceinline__ float lse_value(float2 v) {
  return v.x == neg_inf() ? neg_inf() : v.x + logf(v.y);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, d));
  return v;
}

// Two-level liveness of the arcs' gather states.  The summary word (one bit
// per 32-state block) is read first -- it is small enough to stay in L1 --
// and the state's own bitmap word only when its block holds a live state.
// Summary words of the next token are issued early so their loads overlap
// the current token's work.
struct Live {
  const uint32_t* fine;
  const uint32_t* sum;
};

__device__ __forceinline__ void summary_words(const uint32_t* __restrict__ sum, const int32_t (&st)[APL],
                                              uint32_t (&wd)[APL]) {
#pragma unroll
  for (int k = 0; k < APL; ++k) wd[k] = __ldg(sum + (st[k] >> 10));
}

__device__ __forceinline__ uint32_t live_of(const uint32_t* __restrict__ fine, const uint32_t (&sw)[APL],
                                            const int32_t (&st)[APL]) {
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < APL; ++k)
    if ((sw[k] >> ((st[k] >> 5) & 31)) & 1u) m |= ((__ldg(fine + (st[k] >> 5)) >> (st[k] & 31)) & 1u) << k;
  return m;
}

__device__ __forceinline__ void set_live(uint32_t* fine, uint32_t* sum, int32_t q) {
  atomicOr(fine + (q >> 5), 1u << (q & 31));
  atomicOr(sum + (q >> 10), 1u << ((q >> 5) & 31));
}

// State q has a finite forward value for token p, which is not the last of
// its string: mark, for token p + 1 (input symbol a), the backward window(s)
// of the segment (a, q) and the forward windows of that segment's arcs.
// Marks are plain byte stores (several writers store the same 1).
__device__ __forceinline__ void mark_next(const WaveState& S, const TokenView& T, int32_t p, int32_t q) {
  const int32_t pn = p + 1;
  const int32_t a = __ldg(T.sym + pn);
  int64_t lo = __ldg(S.b_sym_seg + a), hi = __ldg(S.b_sym_seg + a + 1);
  const int64_t end = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(S.b_seg_state + mid) < q) lo = mid + 1; else hi = mid;
  }
  if (lo >= end || __ldg(S.b_seg_state + lo) != q) return;  // q has no arc on symbol a
  const int32_t pos0 = __ldg(S.b_seg_pos + lo), len = __ldg(S.b_seg_len + lo);
  if (S.bin) {
    const int64_t bb = __ldg(T.bwbase + pn) - __ldg(S.b_sym_win + a);
    for (int32_t w = pos0 / WIN; w <= (pos0 + len - 1) / WIN; ++w) S.bin[bb + w] = 1;
  }
  const int64_t fb = __ldg(T.wbase + pn) - __ldg(S.f_sym_win + a);
  for (int32_t i = 0; i < len; ++i) S.fin[fb + __ldg(S.b_fwin + pos0 + i)] = 1;
}

// State q has a finite backward value at the position of token p (which is
// not the first of its string): mark, for token p (input symbol a), the
// backward windows that hold the arcs of the forward segment (a, q), i.e.
// the arcs into q.
__device__ __forceinline__ void mark_prev(const WaveState& S, const TokenView& T, int32_t p, int32_t q) {
  const int32_t a = __ldg(T.sym + p);
  int64_t lo = __ldg(S.f_sym_seg + a), hi = __ldg(S.f_sym_seg + a + 1);
  const int64_t end = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(S.f_seg_state + mid) < q) lo = mid + 1; else hi = mid;
  }
  if (lo >= end || __ldg(S.f_seg_state + lo) != q) return;  // no arc on symbol a enters q
  const int32_t pos0 = __ldg(S.f_seg_pos + lo), len = __ldg(S.f_seg_len + lo);
  const int64_t bb = __ldg(T.bwbase + p) - __ldg(S.b_sym_win + a);
  for (int32_t i = 0; i < len; ++i) S.bmk[bb + __ldg(S.f_bwin + pos0 + i)] = 1;
}

// Tokens of the group (bit j = token j) that visit this window: every token
// at the first position; later, the tokens that marked it, and every token
// on a long segment's window (its segment counts the arrivals of all of them).
__device__ __forceinline__ uint32_t tokens_to_visit(const uint8_t* __restrict__ marks, int32_t cnt, int32_t t0,
                                                    bool is_long, int64_t my_base, int32_t wslice, int lane) {
  if (t0 == 1 || is_long) return cnt >= 32 ? FULL : ((1u << cnt) - 1u);
  return __ballot_sync(FULL, lane < cnt && marks[my_base + wslice] != 0);
}

// ======================================================================
// Viterbi step (Alg. 1 inner loop; Sec. 5.1)
// ======================================================================
__device__ __forceinline__ void vit_write(const LayoutView& L, const WaveState& S, const TokenView& T, int32_t p,
                                          bool has_next, int64_t cb, int32_t s, int32_t sl, unsigned long long key,
                                          unsigned long long* aout, uint32_t tag, uint32_t* bmout, uint32_t* smout) {
  S.bp[cb + sl] = key ? (int32_t)(~(uint32_t)key) : -1;
  if (key) {
    const int32_t q = __ldg(L.seg_state + s);
    aout[q] = tagged_make(fkey_inv((uint32_t)(key >> 32)), tag);
    set_live(bmout, smout, q);
    if (has_next) mark_next(S, T, p, q);
  }
}

__device__ __forceinline__ Live fwd_live(const WaveState& S, int32_t p, int32_t b, int32_t t) {
  // liveness of the forward values the position-t relaxation of token p reads
  if (t == 1) return Live{S.bm_start, S.sum_start};
  return Live{S.abm + (int64_t)((t - 1) % 3) * S.bm_rot + (int64_t)b * S.W, S.tsum + (int64_t)(p - 1) * S.Ws};
}

__global__ void __launch_bounds__(KT, KT_MIN_BLOCKS) k_vit_step(LayoutView L, TokenView T, WorkView W, WaveState S) {
  const int lane = threadIdx.x & 31;
  const uint32_t tag_base = *S.epoch + S.tok0;
  const int32_t nw = warps_total();
  Group G;
  G.g = -1; G.hi = -1; G.lo = 0;
  int32_t tp = 0, tb = 0, tt = 0, tn = 0;
  int64_t tcb = 0, twb = 0;
  int32_t tlb = 0;
  for (int32_t item = warp_id_global(); item < (int32_t)W.nitems; item += nw) {
    if (item >= G.hi) {
      find_group(L, W, item, G);
      if (lane < G.cnt) {
        tp = group_token(W, G, lane);
        tb = __ldg(T.b + tp); tt = __ldg(T.t + tp); tcb = __ldg(T.cbase + tp); tlb = (int32_t)__ldg(T.lbase + tp);
        tn = S.bw_n[tb];
        twb = __ldg(T.wbase + tp);
      }
    }
    const int32_t wslice = item - G.lo;
    const Win x = load_win(L, G.wbase + wslice, lane);
    const bool is_long = x.lseg >= 0;
    uint32_t todo = tokens_to_visit(S.fin, G.cnt, __shfl_sync(FULL, tt, 0), is_long, twb, wslice, lane);
    if (!todo) continue;  // no token has a live source in this window
    const int32_t base = x.w * WIN + lane * APL;
    const int4 s4 = __ldg(reinterpret_cast<const int4*>(L.other + base));
    const float4 t4 = __ldg(reinterpret_cast<const float4*>(L.theta + base));
    const int32_t src[APL] = {s4.x, s4.y, s4.z, s4.w};
    const float th[APL] = {t4.x, t4.y, t4.z, t4.w};
    const uint32_t hn = __shfl_down_sync(FULL, x.h, 1);
    uint32_t wn[APL];
    int jn = __ffs(todo) - 1;
    summary_words(fwd_live(S, __shfl_sync(FULL, tp, jn), __shfl_sync(FULL, tb, jn), __shfl_sync(FULL, tt, jn)).sum,
                  src, wn);
    for (int j = jn; j >= 0; j = jn) {
      todo &= todo - 1u;
      jn = todo ? __ffs(todo) - 1 : -1;
      const int32_t p = __shfl_sync(FULL, tp, j), b = __shfl_sync(FULL, tb, j), t = __shfl_sync(FULL, tt, j);
      const bool has_next = t < __shfl_sync(FULL, tn, j);
      // every arc is relaxed; a source whose bit is clear contributes -inf
      // without reading its 8-byte frontier entry
      const uint32_t lv = live_of(fwd_live(S, p, b, t).fine, wn, src);
      if (jn >= 0)
        summary_words(fwd_live(S, __shfl_sync(FULL, tp, jn), __shfl_sync(FULL, tb, jn), __shfl_sync(FULL, tt, jn)).sum,
                      src, wn);
      if (!is_long && !__any_sync(FULL, lv != 0u)) continue;  // no live source: every segment stays -inf
      float a[APL];
      if (t == 1) {
#pragma unroll
        for (int k = 0; k < APL; ++k) a[k] = ((lv >> k) & 1u) ? __ldg(S.theta_s + src[k]) : neg_inf();
      } else {
        const unsigned long long* ab = S.alpha + ((int64_t)b * 2 + ((t - 1) & 1)) * S.Q;
        const uint32_t tg = tag_base + (uint32_t)(p - 1);
#pragma unroll
        for (int k = 0; k < APL; ++k) a[k] = ((lv >> k) & 1u) ? tagged_value(__ldg(ab + src[k]), tg) : neg_inf();
      }
      unsigned long long key[APL];
#pragma unroll
      for (int k = 0; k < APL; ++k) {
        const float cand = __fadd_rn(a[k], th[k]);
        key[k] = (cand == neg_inf()) ? 0ull
                                     : (((unsigned long long)fkey(cand) << 32) |
                                        (unsigned long long)(~(uint32_t)(base + k)));
      }
      unsigned long long full[APL];
      window_scan<MaxKey>(key, x.h, lane, full);
      const int64_t cb = shfl64(tcb, j);
      unsigned long long* aout = S.alpha + ((int64_t)b * 2 + (t & 1)) * S.Q;
      uint32_t* bmout = S.abm + (int64_t)(t % 3) * S.bm_rot + (int64_t)b * S.W;
      uint32_t* smout = S.tsum + (int64_t)p * S.Ws;
      const uint32_t tag = tag_base + (uint32_t)p;
      if (!is_long) {
        int cum = x.hb;
#pragma unroll
        for (int k = 0; k < APL; ++k) {
          cum += (x.h >> k) & 1u;
          const bool tail = (k < APL - 1) ? ((x.h >> (k + 1)) & 1u) : (lane == 31 || (hn & 1u));
          if (tail) {
            const int32_t s = x.seg + cum - 1;
            vit_write(L, S, T, p, has_next, cb, s, s - G.segbase, full[k], aout, tag, bmout, smout);
          }
        }
      } else {
        const int32_t lb = __shfl_sync(FULL, tlb, j);
        if (lane == 31) {
          // a destination segment that spans warps: packed 64-bit atomicMax
          const int64_t slot = (int64_t)lb + x.lseg;
          atomicMax(S.skey + slot, full[APL - 1]);
          __threadfence();
          const uint32_t prev = atomicAdd(S.scnt + slot, 1u);
          if (prev == (uint32_t)x.lcnt - 1u) {
            __threadfence();
            const unsigned long long kf = atomicMax(S.skey + slot, 0ull);
            vit_write(L, S, T, p, has_next, cb, x.seg, x.seg - G.segbase, kf, aout, tag, bmout, smout);
            S.skey[slot] = 0ull;
            S.scnt[slot] = 0u;
          }
        }
      }
    }
  }
}

// ======================================================================
// Long-segment log-sum-exp: per-window partials, combined in window order
// by the last warp to arrive.  Returns the segment total in every lane of
// the finalising warp; `fin` tells whether this warp finalised.
// ======================================================================
__device__ __forceinline__ bool long_lse_arrive(const LayoutView& L, const WaveState& S, const Win& x,
                                                int64_t lslot, int64_t lwslot, float2 part, int lane,
                                                float2& total) {
  uint32_t prev = 0;
  if (lane == 31) {
    const int32_t w0 = __ldg(L.seg_pos + x.seg) / WIN;
    S.spart[lwslot + x.lwin0 + (x.w - w0)] = part;
    __threadfence();
    prev = atomicAdd(S.scnt + lslot + x.lseg, 1u);
  }
  prev = __shfl_sync(FULL, prev, 31);
  if (prev != (uint32_t)x.lcnt - 1u) return false;
  __threadfence();
  float2 acc = LogAdd::identity();
  const volatile float2* pp = S.spart + lwslot + x.lwin0;
  for (int j = lane; j < x.lcnt; j += 32) {
    float2 v;
    v.x = pp[j].x;
    v.y = pp[j].y;
    acc = LogAdd::combine(acc, v);
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    float2 o = make_float2(__shfl_xor_sync(FULL, acc.x, d), __shfl_xor_sync(FULL, acc.y, d));
    acc = (lane & d) ? LogAdd::combine(o, acc) : LogAdd::combine(acc, o);
  }
  if (lane == 0) S.scnt[lslot + x.lseg] = 0u;
  total = acc;
  return true;
}

// ======================================================================
// Forward step (Alg. 2 forward loop; Sec. 5.2)
// ======================================================================
__global__ void __launch_bounds__(KT, KT_MIN_BLOCKS) k_fwd_step(LayoutView L, TokenView T, WorkView W, WaveState S) {
  const int lane = threadIdx.x & 31;
  const uint32_t tag_base = *S.epoch + S.tok0;
  const int32_t nw = warps_total();
  Group G;
  G.g = -1; G.hi = -1; G.lo = 0;
  int32_t tp = 0, tb = 0, tt = 0, tn = 0, tlb = 0, tlw = 0;
  int64_t tcb = 0, twb = 0;
  float tm = 0.f;
  for (int32_t item = warp_id_global(); item < (int32_t)W.nitems; item += nw) {
    if (item >= G.hi) {
      find_group(L, W, item, G);
      if (lane < G.cnt) {
        tp = group_token(W, G, lane);
        tb = __ldg(T.b + tp); tt = __ldg(T.t + tp); tcb = __ldg(T.cbase + tp);
        tlb = (int32_t)__ldg(T.lbase + tp); tlw = (int32_t)__ldg(T.lwbase + tp); twb = __ldg(T.wbase + tp);
        tm = tt > 1 ? decode_max(S.mkey[tp - 1]) : 0.f;
        tn = S.bw_n[tb];
      }
    }
    const int32_t wslice = item - G.lo;
    const Win x = load_win(L, G.wbase + wslice, lane);
    const bool is_long = x.lseg >= 0;
    // unvisited (token, window) pairs write nothing: readers of the stored
    // forward values consult the window-liveness bytes
    uint32_t todo = tokens_to_visit(S.fin, G.cnt, __shfl_sync(FULL, tt, 0), is_long, twb, wslice, lane);
    if (!todo) continue;
    const int32_t base = x.w * WIN + lane * APL;
    const int4 s4 = __ldg(reinterpret_cast<const int4*>(L.other + base));
    const float4 t4 = __ldg(reinterpret_cast<const float4*>(L.theta + base));
    const int32_t src[APL] = {s4.x, s4.y, s4.z, s4.w};
    const float th[APL] = {t4.x, t4.y, t4.z, t4.w};
    const uint32_t hn = __shfl_down_sync(FULL, x.h, 1);
    uint32_t wn[APL];
    int jn = __ffs(todo) - 1;
    summary_words(fwd_live(S, __shfl_sync(FULL, tp, jn), __shfl_sync(FULL, tb, jn), __shfl_sync(FULL, tt, jn)).sum,
                  src, wn);
    for (int j = jn; j >= 0; j = jn) {
      todo &= todo - 1u;
      jn = todo ? __ffs(todo) - 1 : -1;
      const int32_t p = __shfl_sync(FULL, tp, j), b = __shfl_sync(FULL, tb, j), t = __shfl_sync(FULL, tt, j);
      const float mprev = __shfl_sync(FULL, tm, j);
      const bool has_next = t < __shfl_sync(FULL, tn, j);
      const uint32_t lv = live_of(fwd_live(S, p, b, t).fine, wn, src);
      if (jn >= 0)
        summary_words(fwd_live(S, __shfl_sync(FULL, tp, jn), __shfl_sync(FULL, tb, jn), __shfl_sync(FULL, tt, jn)).sum,
                      src, wn);
      const int64_t cb = shfl64(tcb, j);
      if (!is_long && !__any_sync(FULL, lv != 0u)) {
        // no live source: every segment of the window is -inf at this position
        int cum = x.hb;
#pragma unroll
        for (int k = 0; k < APL; ++k) {
          cum += (x.h >> k) & 1u;
          const bool tail = (k < APL - 1) ? ((x.h >> (k + 1)) & 1u) : (lane == 31 || (hn & 1u));
          if (tail) S.rc[cb + (x.seg + cum - 1 - G.segbase)] = neg_inf();
        }
        continue;
      }
      float a[APL];
      if (t == 1) {
#pragma unroll
        for (int k = 0; k < APL; ++k) a[k] = ((lv >> k) & 1u) ? __ldg(S.theta_s + src[k]) : neg_inf();
      } else {
        const unsigned long long* ab = S.alpha + ((int64_t)b * 2 + ((t - 1) & 1)) * S.Q;
        const uint32_t tg = tag_base + (uint32_t)(p - 1);
#pragma unroll
        for (int k = 0; k < APL; ++k) {
          const float r = ((lv >> k) & 1u) ? tagged_value(__ldg(ab + src[k]), tg) : neg_inf();
          a[k] = (r == neg_inf() || mprev == neg_inf()) ? neg_inf() : r - mprev;
        }
      }
      float2 e[APL];
#pragma unroll
      for (int k = 0; k < APL; ++k) {
        const float v = a[k] + th[k];
        e[k] = (v == neg_inf()) ? LogAdd::identity() : make_float2(v, 1.f);
      }
      float2 full[APL];
      window_scan<LogAdd>(e, x.h, lane, full);
      unsigned long long* aout = S.alpha + ((int64_t)b * 2 + (t & 1)) * S.Q;
      uint32_t* bmout = S.abm + (int64_t)(t % 3) * S.bm_rot + (int64_t)b * S.W;
      uint32_t* smout = S.tsum + (int64_t)p * S.Ws;
      const uint32_t tag = tag_base + (uint32_t)p;
      float rmax = neg_inf();
      if (!is_long) {
        int cum = x.hb;
#pragma unroll
        for (int k = 0; k < APL; ++k) {
          cum += (x.h >> k) & 1u;
          const bool tail = (k < APL - 1) ? ((x.h >> (k + 1)) & 1u) : (lane == 31 || (hn & 1u));
          if (tail) {
            const int32_t s = x.seg + cum - 1;
            const float r = lse_value(full[k]);
            S.rc[cb + (s - G.segbase)] = r;
            if (r != neg_inf()) {
              const int32_t q = __ldg(L.seg_state + s);
              aout[q] = tagged_make(r, tag);
              set_live(bmout, smout, q);
              if (has_next) mark_next(S, T, p, q);
            }
            rmax = fmaxf(rmax, r);
          }
        }
        rmax = warp_max(rmax);
        // the backward pass restores forward values only in windows marked live
        const int64_t wbt = shfl64(twb, j);
        if (lane == 0 && rmax != neg_inf()) S.wlive[wbt + wslice] = 1;
      } else {
        float2 tot;
        const int64_t wbt = shfl64(twb, j);
        if (long_lse_arrive(L, S, x, __shfl_sync(FULL, tlb, j), __shfl_sync(FULL, tlw, j), full[APL - 1], lane, tot)) {
          const float r = lse_value(tot);
          if (lane == 0) {
            S.rc[cb + (x.seg - G.segbase)] = r;
            if (r != neg_inf()) {
              const int32_t q = __ldg(L.seg_state + x.seg);
              aout[q] = tagged_make(r, tag);
              set_live(bmout, smout, q);
              if (has_next) mark_next(S, T, p, q);
              // the segment's first window carries its head
              S.wlive[wbt + (__ldg(L.seg_pos + x.seg) / WIN - G.wbase)] = 1;
            }
          }
          rmax = r;
        }
      }
      if (lane == 0 && rmax != neg_inf()) atomicMax(S.mkey + p, fkey(rmax));
    }
  }
}

// ======================================================================
// Scatter the stored forward values of one position t_s back into the
// dense frontier (needed by the backward step t_s + 1 when step t_s + 2 has
// overwritten that parity buffer).  Only windows that the forward pass
// marked live are read.  Runs inside the backward step t_s + 2, whose
// frontier reads use the other parity buffer.
// ======================================================================
__device__ __forceinline__ void scatter_alpha_items(const LayoutView& L, const TokenView& T, const WorkView& W,
                                                    const WaveState& S, int32_t t_bwd) {
  const int lane = threadIdx.x & 31;
  const uint32_t tag_base = *S.epoch + S.tok0;
  const int32_t nw = warps_total();
  Group G;
  G.g = -1; G.hi = -1; G.lo = 0;
  int32_t tp = 0, tb = 0, tt = 0, tn = 0;
  int64_t tcb = 0, twb = 0;
  for (int32_t item = warp_id_global(); item < (int32_t)W.nitems; item += nw) {
    if (item >= G.hi) {
      find_group(L, W, item, G);
      if (lane < G.cnt) {
        tp = group_token(W, G, lane);
        tb = __ldg(T.b + tp); tt = __ldg(T.t + tp); tcb = __ldg(T.cbase + tp); tn = S.bw_n[tb];
        twb = __ldg(T.wbase + tp);
      }
    }
    const int32_t wslice = item - G.lo;
    // lane j: is window `wslice` live for token j (and is its frontier needed)?
    const bool need = lane < G.cnt && tn > t_bwd && S.wlive[twb + wslice] != 0;
    uint32_t todo = __ballot_sync(FULL, need);
    if (!todo) continue;
    const Win x = load_win(L, G.wbase + wslice, lane);
    while (todo) {
      const int j = __ffs(todo) - 1;
      todo &= todo - 1;
      const int32_t p = __shfl_sync(FULL, tp, j), b = __shfl_sync(FULL, tb, j), t = __shfl_sync(FULL, tt, j);
      const int64_t cb = shfl64(tcb, j);
      unsigned long long* aout = S.alpha + ((int64_t)b * 2 + (t & 1)) * S.Q;
      const uint32_t tag = tag_base + (uint32_t)p;
      int cum = x.hb;
#pragma unroll
      for (int k = 0; k < APL; ++k) {
        if ((x.h >> k) & 1u) {
          const int32_t s = x.seg + cum;
          const float r = S.rc[cb + (s - G.segbase)];
          if (r != neg_inf()) aout[__ldg(L.seg_state + s)] = tagged_make(r, tag);
          ++cum;
        }
      }
    }
  }
}

// ======================================================================
// Backward step fused with the expected counts (Alg. 2 backward loop and
// count loop; Sec. 5.2).  Segments are by source state.
// ======================================================================
__device__ __forceinline__ Live bwd_live(const WaveState& S, int32_t b, int32_t t, int32_t n) {
  // liveness of the backward values the position-t relaxation reads
  if (t == n) return Live{S.bm_final, S.sum_final};
  const int64_t r = t % 3;
  return Live{S.bbm + r * S.bm_rot + (int64_t)b * S.W, S.bsum + r * S.sum_rot + (int64_t)b * S.Ws};
}

__global__ void __launch_bounds__(KT, KT_MIN_BLOCKS_BWD) k_bwd_step(LayoutView L, TokenView T, WorkView W,
                                                                    WaveState S, CountView C, ScatterJob J) {
  const int lane = threadIdx.x & 31;
  const uint32_t tag_base = *S.epoch + S.tok0;
  const int32_t nw = warps_total();
  Group G;
  G.g = -1; G.hi = -1; G.lo = 0;
  // lane j: token j of the group
  int32_t tp = 0, tb = 0, tt = 0, tn = 0, tlb = 0, tlw = 0;
  int64_t tbb = 0;
  float tm = 0.f, te = 0.f, tw = 0.f;
  double tK = 0.0;
  bool tlive = false;
  for (int32_t item = warp_id_global(); item < (int32_t)W.nitems; item += nw) {
    if (item >= G.hi) {
      find_group(L, W, item, G);
      if (lane < G.cnt) {
        tp = group_token(W, G, lane);
        tb = __ldg(T.b + tp); tt = __ldg(T.t + tp);
        tlb = (int32_t)__ldg(T.lbase_b + tp); tlw = (int32_t)__ldg(T.lwbase_b + tp);
        tbb = __ldg(T.bwbase + tp);
        tn = S.bw_n[tb];
        const double lz = S.logz[tb];
        tlive = lz != -INFINITY;
        te = (tt == tn) ? 0.f : decode_max(S.ekey[tp]);
        const double tE = (tt == tn) ? 0.0 : S.esum[tp + 1] + (double)te;
        const double Ctm1 = (tt == 1) ? 0.0 : S.csum[tp - 1];
        tK = Ctm1 + tE - lz;
        tm = (tt == 1) ? 0.f : decode_max(S.mkey[tp - 1]);
        tw = S.gweight ? S.gweight[tb] : 1.f;
        // E_t for the next position's launch: written once per token
        if (item == G.lo && tlive) S.esum[tp] = tE;
      } else {
        tlive = false;
      }
    }
    const int32_t wslice = item - G.lo;
    const Win x = load_win(L, G.wbase + wslice, lane);
    const bool is_long = x.lseg >= 0;
    bool visit = false;
    if (lane < G.cnt && tlive) {
      if (is_long) {
        // every window of a long segment has the same source: all of them are
        // visited, or none (their arrivals are counted); the forward marks
        // cover every window of the segment of a live source
        visit = (tt == 1) ? __ldg(S.theta_s + __ldg(L.seg_state + x.seg)) != neg_inf() : S.bin[tbb + wslice] != 0;
      } else if (tt == 1 && tt == tn) {
        visit = true;
      } else if (tt == 1) {
        visit = S.bmk[tbb + wslice] != 0;
      } else if (tt == tn) {
        visit = S.bin[tbb + wslice] != 0;
      } else {
        visit = S.bin[tbb + wslice] != 0 && S.bmk[tbb + wslice] != 0;
      }
    }
    uint32_t todo = __ballot_sync(FULL, visit);
    if (!todo) continue;  // no live token has a source with a finite forward value here
    const int32_t base = x.w * WIN + lane * APL;
    const int4 d4 = __ldg(reinterpret_cast<const int4*>(L.other + base));
    const float4 t4 = __ldg(reinterpret_cast<const float4*>(L.theta + base));
    const int32_t dst[APL] = {d4.x, d4.y, d4.z, d4.w};
    const float th[APL] = {t4.x, t4.y, t4.z, t4.w};
    const uint32_t hn = __shfl_down_sync(FULL, x.h, 1);
    // segment (source state) of each arc; padding arcs belong to the window's last segment
    int32_t qs[APL];
    {
      int cum = x.hb;
#pragma unroll
      for (int k = 0; k < APL; ++k) {
        cum += (x.h >> k) & 1u;
        qs[k] = __ldg(L.seg_state + (is_long ? x.seg : x.seg + cum - 1));
      }
    }
    float gacc[APL] = {0.f, 0.f, 0.f, 0.f};
    uint32_t wn[APL];
    int jn = __ffs(todo) - 1;
    summary_words(bwd_live(S, __shfl_sync(FULL, tb, jn), __shfl_sync(FULL, tt, jn), __shfl_sync(FULL, tn, jn)).sum,
                  dst, wn);
    for (int j = jn; j >= 0; j = jn) {
      todo &= todo - 1u;
      jn = todo ? __ffs(todo) - 1 : -1;
      const int32_t p = __shfl_sync(FULL, tp, j), b = __shfl_sync(FULL, tb, j), t = __shfl_sync(FULL, tt, j);
      const int32_t n = __shfl_sync(FULL, tn, j);
      // beta_t at the destinations; a destination whose bit is clear is -inf
      uint32_t lv = live_of(bwd_live(S, b, t, n).fine, wn, dst);
      if (jn >= 0)
        summary_words(bwd_live(S, __shfl_sync(FULL, tb, jn), __shfl_sync(FULL, tt, jn), __shfl_sync(FULL, tn, jn)).sum,
                      dst, wn);
      // Only sources whose forward value alpha_{t-1} is finite matter: every
      // posterior through a dead source is zero, and a finite-alpha state
      // reaches only finite-alpha states, so its backward value is exact
      // without the pruned terms.  Coarse test here; the source's own value
      // is read below.
      {
        const uint32_t* asm_ = (t == 1) ? S.sum_start : S.tsum + (int64_t)(p - 1) * S.Ws;
        uint32_t al = 0;
#pragma unroll
        for (int k = 0; k < APL; ++k) al |= ((__ldg(asm_ + (qs[k] >> 10)) >> ((qs[k] >> 5) & 31)) & 1u) << k;
        lv &= al;
      }
      if (!is_long && !__any_sync(FULL, lv != 0u)) continue;  // no arc joins a live source to a live state
      // raw values: ub = beta_t[dst] before its step shift (theta_f at the
      // last position), ra = alpha_{t-1}[src] before its shift (theta_s at
      // the first); -inf where the state is dead
      const float et = (t == n) ? 0.f : __shfl_sync(FULL, te, j);
      const float mprev = (t == 1) ? 0.f : __shfl_sync(FULL, tm, j);
      float ub[APL];
      if (t == n) {
#pragma unroll
        for (int k = 0; k < APL; ++k) ub[k] = ((lv >> k) & 1u) ? __ldg(S.theta_f + dst[k]) : neg_inf();
      } else {
        const unsigned long long* bb = S.beta + ((int64_t)b * 2 + (t & 1)) * S.Q;
        const uint32_t tg = tag_base + (uint32_t)p;
#pragma unroll
        for (int k = 0; k < APL; ++k) ub[k] = ((lv >> k) & 1u) ? tagged_value(__ldg(bb + dst[k]), tg) : neg_inf();
      }
      // alpha_{t-1} at the sources (one state per segment: cached loads)
      float ra[APL];
      {
        const unsigned long long* ab = S.alpha + ((int64_t)b * 2 + ((t - 1) & 1)) * S.Q;
        const uint32_t tga = tag_base + (uint32_t)(p - 1);
#pragma unroll
        for (int k = 0; k < APL; ++k)
          ra[k] = !((lv >> k) & 1u) ? neg_inf()
                                    : (t == 1 ? __ldg(S.theta_s + qs[k]) : tagged_value(__ldg(ab + qs[k]), tga));
      }
      const bool dead_shift = (et == neg_inf()) || (mprev == neg_inf());
      float v[APL];
#pragma unroll
      for (int k = 0; k < APL; ++k)
        v[k] = (ub[k] == neg_inf() || ra[k] == neg_inf() || dead_shift) ? neg_inf() : th[k] + (ub[k] - et);
      // beta_{t-1} by source segment (not needed for t == 1)
      if (t >= 2) {
        float2 e[APL];
#pragma unroll
        for (int k = 0; k < APL; ++k) e[k] = (v[k] == neg_inf()) ? LogAdd::identity() : make_float2(v[k], 1.f);
        float2 full[APL];
        window_scan<LogAdd>(e, x.h, lane, full);
        unsigned long long* bout = S.beta + ((int64_t)b * 2 + ((t - 1) & 1)) * S.Q;
        uint32_t* bmout = S.bbm + (int64_t)((t - 1) % 3) * S.bm_rot + (int64_t)b * S.W;
        uint32_t* smout = S.bsum + (int64_t)((t - 1) % 3) * S.sum_rot + (int64_t)b * S.Ws;
        const uint32_t tag = tag_base + (uint32_t)(p - 1);
        float umax = neg_inf();
        if (!is_long) {
          int cum = x.hb;
#pragma unroll
          for (int k = 0; k < APL; ++k) {
            cum += (x.h >> k) & 1u;
            const bool tail = (k < APL - 1) ? ((x.h >> (k + 1)) & 1u) : (lane == 31 || (hn & 1u));
            if (tail) {
              const float u = lse_value(full[k]);
              if (u != neg_inf()) {
                bout[qs[k]] = tagged_make(u, tag);
                set_live(bmout, smout, qs[k]);
                mark_prev(S, T, p - 1, qs[k]);
              }
              umax = fmaxf(umax, u);
            }
          }
        } else {
          float2 tot;
          if (long_lse_arrive(L, S, x, __shfl_sync(FULL, tlb, j), __shfl_sync(FULL, tlw, j), full[APL - 1], lane,
                              tot)) {
            const float u = lse_value(tot);
            if (lane == 0 && u != neg_inf()) {
              const int32_t q = __ldg(L.seg_state + x.seg);
              bout[q] = tagged_make(u, tag);
              set_live(bmout, smout, q);
              mark_prev(S, T, p - 1, q);
            }
            umax = u;
          }
        }
        umax = warp_max(umax);
        if (lane == 0 && umax != neg_inf()) atomicMax(S.ekey + p - 1, fkey(umax));
      }
      // posteriors gamma_t(k) = exp(alpha_{t-1}[src] + theta_k + beta_t[dst] - log Z);
      // the exponent adds terms of either sign and tens in size that cancel to
      // a small number, so it is formed in float64 (live arcs only)
      const double K = __shfl_sync(FULL, tK, j);
      const float gw = __shfl_sync(FULL, tw, j);
#pragma unroll
      for (int k = 0; k < APL; ++k) {
        if (v[k] == neg_inf()) continue;
        const double ex = ((double)ra[k] - (double)mprev) + (double)th[k] + ((double)ub[k] - (double)et) + K;
        gacc[k] += __expf((float)ex) * gw;
      }
    }
    // accumulate this item's counts
#pragma unroll
    for (int k = 0; k < APL; ++k) {
      if (gacc[k] == 0.f) continue;
      const int32_t pos = base + k;
      if (C.batched) {
        atomicAdd(C.cnt64 + pos, (double)gacc[k]);
      } else {
        // compensated float32 summation (one string: no concurrent writer)
        const float gv = gacc[k];
        const float s0 = C.cnt[pos], cmp = C.comp[pos];
        const float y = __fsub_rn(gv, cmp);
        const float s1 = __fadd_rn(s0, y);
        C.comp[pos] = __fsub_rn(__fsub_rn(s1, s0), y);
        C.cnt[pos] = s1;
      }
    }
  }
  // alpha_{t-2} for the next launch (backward step t - 1), into the parity
  // buffer this step does not read
  if (J.W.nitems > 0) scatter_alpha_items(J.L, T, J.W, S, J.t_bwd);
}

// ======================================================================
// Epilogues: final reduction (Alg. 1 return line; Alg. 2 Z), backtrace
// (Sec. 5.1), and counts back to caller arc order.
// ======================================================================
// The states that can end a path at the last position lie in the 32-state
// groups whose bit is set both in the position's forward summary (groups
// holding a state written with a finite value) and in the summary of final
// states.  A block per string: its warps stride over 32-word chunks of the
// summaries, and for each marked group a warp reads its 32 states
// (consecutive, one per lane) from the dense frontier, FV groups at a time.
constexpr int FV = 4;
constexpr int FT = 256;  // threads of the final-reduction blocks

template <class F>
__device__ __forceinline__ void for_final_groups(const uint32_t* __restrict__ live, const uint32_t* __restrict__ fin,
                                                 int32_t Ws, F f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int32_t c = warp * 32; c < Ws; c += (FT / 32) * 32) {
    const int32_t wi = c + lane;
    const uint32_t word = wi < Ws ? live[wi] & __ldg(fin + wi) : 0u;
    uint32_t lanes = __ballot_sync(FULL, word != 0u);
    while (lanes) {
      const int l = __ffs(lanes) - 1;
      lanes &= lanes - 1u;
      uint32_t wd = __shfl_sync(FULL, word, l);  // warp-uniform
      const int32_t g0 = (c + l) * 32;
      while (wd) {
        int32_t q[FV];
#pragma unroll
        for (int u = 0; u < FV; ++u) {
          q[u] = wd ? (g0 + __ffs(wd) - 1) * 32 + lane : -1;
          wd &= wd - 1u;
        }
        f(q);
      }
    }
  }
}

__global__ void __launch_bounds__(FT) k_vit_final(WaveState S, float* __restrict__ scores,
                                                  int32_t* __restrict__ qfinal, int32_t* __restrict__ status) {
  __shared__ unsigned long long red[FT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = blockIdx.x;
  const int32_t n = S.bw_n[b];
  const int64_t p = S.bw_off[b] + n - 1;
  const unsigned long long* ab = S.alpha + (b * 2 + (n & 1)) * S.Q;
  const uint32_t tg = *S.epoch + S.tok0 + (uint32_t)p;
  const int32_t Q = S.Q;
  unsigned long long best = 0ull;
  for_final_groups(n == 0 ? S.sum_start : S.tsum + p * S.Ws, S.sum_final, S.Ws, [&](const int32_t (&q)[FV]) {
    float a[FV], fv[FV];
#pragma unroll
    for (int u = 0; u < FV; ++u) {
      const bool ok = q[u] >= 0 && q[u] < Q;
      a[u] = !ok ? neg_inf() : (n == 0 ? __ldg(S.theta_s + q[u]) : tagged_value(ab[q[u]], tg));
      fv[u] = ok ? __ldg(S.theta_f + q[u]) : neg_inf();
    }
#pragma unroll
    for (int u = 0; u < FV; ++u) {
      const float cnd = __fadd_rn(a[u], fv[u]);
      if (cnd != neg_inf()) {
        const unsigned long long k = ((unsigned long long)fkey(cnd) << 32) | (unsigned long long)(~(uint32_t)q[u]);
        best = k > best ? k : best;
      }
    }
  });
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(FULL, best, d);
    best = o > best ? o : best;
  }
  if (lane == 0) red[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < FT / 32; ++w) best = red[w] > best ? red[w] : best;
    scores[b] = best ? fkey_inv((uint32_t)(best >> 32)) : neg_inf();
    qfinal[b] = best ? (int32_t)(~(uint32_t)best) : -1;
    if (status) status[b] = best ? FST_OK : FST_ERR_NO_PATH;
  }
}

// One warp per string; a 32-way search finds the state's segment at each step.
__global__ void k_backtrace(LayoutView L, const int32_t* __restrict__ tok_sym, const int64_t* __restrict__ cbase,
                            WaveState S, const int32_t* __restrict__ olabel_by_id,
                            const int32_t* __restrict__ arc_id, int32_t Bw, const int32_t* __restrict__ qfinal,
                            int32_t* __restrict__ paths, int32_t* __restrict__ olabels) {
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
    const int32_t sym = tok_sym[p];
    int64_t lo = L.sym_seg[sym], hi = L.sym_seg[sym + 1];
    while (hi - lo > 32) {
      const int64_t step = (hi - lo + 31) / 32;
      const int64_t i = lo + (int64_t)lane * step;
      const bool le = (i < hi) && (L.seg_state[i] <= q);
      const uint32_t bal = __ballot_sync(FULL, le);
      const int last = bal ? 31 - __clz(bal) : 0;
      lo = lo + (int64_t)last * step;
      hi = min(hi, lo + step);
    }
    const int64_t i = lo + lane;
    const uint32_t bal = __ballot_sync(FULL, (i < hi) && (L.seg_state[i] == q));
    int32_t pos = -1;
    if (bal) {
      const int64_t s = lo + (__ffs(bal) - 1);
      pos = S.bp[cbase[p] + (s - L.sym_seg[sym])];
    }
    if (pos < 0) {  // cannot happen for a live state; leave a marker instead of faulting
      if (lane == 0) paths[p] = -1;
      break;
    }
    const int32_t k = arc_id[pos];
    if (lane == 0) {
      paths[p] = k;
      if (olabels) olabels[p] = olabel_by_id[k];
    }
    q = L.other[pos];
  }
}

// log Z of one string (Alg. 2, Z): C_{n-1} + log sum_q exp(alpha_n[q] +
// final[q]), alpha_n the shifted forward values of the last position.  Warp
// 0 also writes the running normalisers C_t (a warp scan); the other
// partial sums are online (max, sum) pairs per lane, exp in float32 as in
// the step kernels, sums in float64, combined in a fixed order.
__global__ void __launch_bounds__(FT) k_fb_final(WaveState S, double* __restrict__ logz,
                                                 int32_t* __restrict__ status) {
  __shared__ float red_m[FT / 32];
  __shared__ double red_s[FT / 32];
  __shared__ double c_prev;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = blockIdx.x;
  const int32_t n = S.bw_n[b];
  const int64_t off = S.bw_off[b];
  if (warp == 0) {
    // C_t = sum_{s<=t} m_s in float64 (-inf once some position has no path)
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
  const unsigned long long* ab = S.alpha + (b * 2 + (n & 1)) * S.Q;
  const uint32_t tg = *S.epoch + S.tok0 + (uint32_t)p;
  const int32_t Q = S.Q;
  float mx = neg_inf();
  double sum = 0.0;
  for_final_groups(n == 0 ? S.sum_start : S.tsum + p * S.Ws, S.sum_final, S.Ws, [&](const int32_t (&q)[FV]) {
    float a[FV], fv[FV];
#pragma unroll
    for (int u = 0; u < FV; ++u) {
      const bool ok = q[u] >= 0 && q[u] < Q;
      a[u] = !ok ? neg_inf() : (n == 0 ? __ldg(S.theta_s + q[u]) : tagged_value(ab[q[u]], tg));
      fv[u] = ok ? __ldg(S.theta_f + q[u]) : neg_inf();
    }
#pragma unroll
    for (int u = 0; u < FV; ++u) {
      const float v = __fadd_rn(a[u], fv[u]);
      if (v == neg_inf()) continue;
      if (v > mx) {
        sum = (mx == neg_inf()) ? 1.0 : sum * (double)__expf(mx - v) + 1.0;
        mx = v;
      } else {
        sum += (double)__expf(v - mx);
      }
    }
  });
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const float om = __shfl_xor_sync(FULL, mx, d);
    const double os = __shfl_xor_sync(FULL, sum, d);
    if (om != neg_inf()) {
      if (om > mx) {
        sum = (mx == neg_inf()) ? os : os + sum * (double)__expf(mx - om);
        mx = om;
      } else {
        sum += os * (double)__expf(om - mx);
      }
    }
  }
  if (lane == 0) {
    red_m[warp] = mx;
    red_s[warp] = sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < FT / 32; ++w) {
      const float om = red_m[w];
      const double os = red_s[w];
      if (om == neg_inf()) continue;
      if (om > mx) {
        sum = (mx == neg_inf()) ? os : os + sum * (double)__expf(mx - om);
        mx = om;
      } else {
        sum += os * (double)__expf(om - mx);
      }
    }
    const double cp = c_prev;
    double lz = -INFINITY;
    if (mx != neg_inf() && cp != -INFINITY) lz = cp + (double)mx + log(sum);
    logz[b] = lz;
    if (status) status[b] = (lz == -INFINITY) ? FST_ERR_NO_PATH : FST_OK;
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

// Step kernels are grid-stride loops: the grid is the number of blocks that
// can be resident at once (all warps advance through the work list
// together, which keeps the frontiers being gathered in L2).
template <class K>
inline int resident_blocks(K kernel, int* cache) {
  if (*cache <= 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, KT, 0) != cudaSuccess || nb <= 0) {
      (void)cudaGetLastError();
      nb = 1;
    }
    *cache = nb;
  }
  return *cache;
}

inline unsigned grid_clamp(int64_t nitems, int num_sms, int per_sm) {
  int64_t need = (nitems + (KT / 32) - 1) / (KT / 32);
  if (need < 1) need = 1;
  const int64_t cap = (int64_t)num_sms * per_sm;
  return (unsigned)(need < cap ? need : cap);
}

int g_occ[4] = {0, 0, 0, 0};

}  // namespace

int launch_vit_step(const LayoutView& L, const TokenView& T, const WorkView& W, const WaveState& S, int grid,
                    cudaStream_t s) {
  if (W.nitems <= 0) return FST_OK;
  k_vit_step<<<grid_clamp(W.nitems, grid, resident_blocks(k_vit_step, &g_occ[0])), KT, 0, s>>>(L, T, W, S);
  return check_launch("k_vit_step");
}

int launch_fwd_step(const LayoutView& L, const TokenView& T, const WorkView& W, const WaveState& S, int grid,
                    cudaStream_t s) {
  if (W.nitems <= 0) return FST_OK;
  k_fwd_step<<<grid_clamp(W.nitems, grid, resident_blocks(k_fwd_step, &g_occ[1])), KT, 0, s>>>(L, T, W, S);
  return check_launch("k_fwd_step");
}

int launch_bwd_step(const LayoutView& L, const TokenView& T, const WorkView& W, const WaveState& S,
                    const CountView& C, const ScatterJob& J, int grid, cudaStream_t s) {
  const int64_t items = W.nitems > J.W.nitems ? W.nitems : J.W.nitems;
  if (items <= 0) return FST_OK;
  k_bwd_step<<<grid_clamp(items, grid, resident_blocks(k_bwd_step, &g_occ[2])), KT, 0, s>>>(L, T, W, S, C, J);
  return check_launch("k_bwd_step");
}

int launch_vit_final(const WaveState& S, int32_t Bw, float* scores, int32_t* qfinal, int32_t* status, cudaStream_t s) {
  if (Bw <= 0) return FST_OK;
  k_vit_final<<<(unsigned)Bw, FT, 0, s>>>(S, scores, qfinal, status);
  return check_launch("k_vit_final");
}

int launch_backtrace(const LayoutView& Lf, const int32_t* tok_sym, const int64_t* cbase, const WaveState& S,
                     const int32_t* olabel_by_id, const int32_t* arc_id_fwd, int32_t Bw, const int32_t* qfinal,
                     int32_t* paths, int32_t* olabels, cudaStream_t s) {
  if (Bw <= 0) return FST_OK;
  k_backtrace<<<(unsigned)((Bw + 3) / 4), 128, 0, s>>>(Lf, tok_sym, cbase, S, olabel_by_id, arc_id_fwd, Bw,
                                                       qfinal, paths, olabels);
  return check_launch("k_backtrace");
}

int launch_fb_final(const WaveState& S, int32_t Bw, double* logz, int32_t* status, cudaStream_t s) {
  if (Bw <= 0) return FST_OK;
  k_fb_final<<<(unsigned)Bw, FT, 0, s>>>(S, logz, status);
  return check_launch("k_fb_final");
}

int launch_counts_out(const int32_t* arc_id_bwd, int64_t P, const CountView& C, float* out, cudaStream_t s) {
  if (P <= 0) return FST_OK;
  k_counts_out<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(arc_id_bwd, P, C, out);
  return check_launch("k_counts_out");
}

}  // namespace fstgpu
