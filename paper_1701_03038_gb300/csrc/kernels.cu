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
// posterior, so skipping it changes no result.  The kernels therefore walk
// only the arcs out of live states, found through a (symbol, state) hash of
// the source-segmented layout, and keep the paper's push direction:
//
//   Viterbi  -- one launch per position: read and clear the accumulators of
//               the destinations staged at t (the packed key of the best
//               arc), write them to the live pool, and push every arc of
//               each new live state into position t+1 with a 64-bit
//               atomicMax of (order-preserving score bits << 32 | ~arc id):
//               the best score wins, and on ties the lowest arc id;
//   forward  -- two launches per position: the atomicMax of the arc values
//               (order keys), then, once every maximum is final, an integer
//               atomicAdd of exp(value - maximum) in 2^-40 fixed point.  Both
//               are exact, so the log-sum-exp does not depend on the order
//               in which the atomics land;
//   backward -- one launch per position: each live state q of t-1 reduces
//               beta over its own arcs on w_t (pull, in shared memory) and
//               adds the posterior of each arc.
//
// The push that finds an accumulator empty stages its destination, so each
// position's live states are listed exactly once, with no bitmap.  Forward
// values are shifted by the previous position's maximum and backward values
// by the next position's; the running shifts are kept in float64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>

#include "kernels.cuh"

namespace fstgpu {
namespace {

constexpr int KT = 256;  // threads per block of the step kernels
constexpr int FT = 256;  // threads per block of the final reductions

// Error bits of a run (FrontierState::flags[1]): the live pool overflowed,
// or a grid barrier of a persistent pass gave up waiting.
constexpr uint32_t ERR_POOL = 1u;
constexpr uint32_t ERR_TIMEOUT = 2u;
__device__ __forceinline__ int32_t run_error(uint32_t err) {
  return (err & ERR_TIMEOUT) ? FST_ERR_TIMEOUT : FST_ERR_OOM;
}

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

// Bounds-checked build (FST_DEBUG): in_bounds(code, i, n) checks 0 <= i < n,
// and on a violation counts it, records the first (code, index, bound) and
// returns false so that the caller skips the access.  A normal build
// compiles every check away.
enum : int { CHK_STAGE = 1, CHK_POOL_WRITE = 2, CHK_POOL_READ = 3, CHK_ACC = 4, CHK_ARC = 5, CHK_TOKEN = 6 };
#ifdef FST_DEBUG
__device__ unsigned long long g_dbg[4];  // violations, code, index, bound
__device__ __noinline__ bool in_bounds_slow(int code, long long i, long long n) {
  if (atomicAdd(&g_dbg[0], 1ull) == 0ull) {
    g_dbg[1] = (unsigned long long)code;
    g_dbg[2] = (unsigned long long)i;
    g_dbg[3] = (unsigned long long)n;
  }
  return false;
}
__device__ __forceinline__ bool in_bounds(int code, long long i, long long n) {
  return (i >= 0 && i < n) ? true : in_bounds_slow(code, i, n);
}
#else
__device__ __forceinline__ bool in_bounds(int, long long, long long) { return true; }
#endif

__device__ __forceinline__ float decode_max(uint32_t k) { return k ? fkey_inv(k) : neg_inf(); }

// Owner of flat entry j among the n slots whose first entries base[0..n)
// are nondecreasing with base[0] <= j: the last slot with base <= j.  The
// warp first finds the owner of its chunk start j0 (warp-uniform, 32-way
// search); flat_owner then places each lane among the 32 slots that follow.
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
// An entry for lanes past the range end: the last entry, or c0 when the
// warp lies wholly past it (the result is unused there).
__device__ __forceinline__ int64_t clamp_entry(int64_t j, int64_t c0, int64_t R1) {
  const int64_t last = R1 - 1 > c0 ? R1 - 1 : c0;
  return j < last ? j : last;
}

struct Owner {
  int32_t k;      // the owning slot
  int64_t first;  // its first entry, base[k]
};
// Owner of this lane's entry j >= c0, c0 the warp's first entry (uniform).
// All 32 lanes take part: the warp loads the 32 slot bases from the owner
// of c0 on and each lane binary-searches them in registers (five shuffles);
// an entry past them (a run of slots with no entries) is walked to.
__device__ __forceinline__ Owner flat_owner(const int64_t* __restrict__ base, int32_t n, int64_t c0, int64_t j) {
  const int lane = threadIdx.x & 31;
  const int32_t k0 = warp_owner(base, n, c0);
  const long long bv = k0 + lane < n ? (long long)__ldcg(base + k0 + lane) : (long long)INT64_MAX;
  int idx = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const long long v = __shfl_sync(FULL, bv, idx + step);
    if (v <= j) idx += step;
  }
  Owner o{k0 + idx, (int64_t)__shfl_sync(FULL, bv, idx)};
  if (idx == 31) {
    while (o.k + 1 < n) {
      const int64_t nb = __ldcg(base + o.k + 1);
      if (nb > j) break;
      ++o.k;
      o.first = nb;
    }
  }
  return o;
}

// The arcs out of state q on symbol a: a lookup in the open-addressing
// table of the source-segmented layout (load factor <= 1/2, one 16-byte
// probe on average) giving their first position and count (0 when none).
struct Arcs {
  int32_t pos, len;
};
__device__ __forceinline__ Arcs find_arcs(const LayoutView& L, int32_t a, int32_t q) {
  const uint64_t k = seg_hash_key(a, q);
  uint64_t h = seg_hash_slot(k, L.hash_mask);
  for (int64_t probe = 0; probe <= L.hash_mask; ++probe) {
    const ulonglong2 e = __ldg(L.seg_hash + h);
    if (e.x == k) {
      const Arcs r{(int32_t)(uint32_t)e.y, (int32_t)(e.y >> 32)};
      if (r.len > 0 && !in_bounds(CHK_ARC, (long long)r.pos + r.len - 1, L.P)) return Arcs{0, 0};
      return r;
    }
    if (e.x == ~0ull) break;
    h = (h + 1) & (uint64_t)L.hash_mask;
  }
  return Arcs{0, 0};
}

// Staging buffer of forward position t (two, by parity: a step reads
// position t's while it fills position t+1's).
__device__ __forceinline__ int32_t* fwd_stage(const FrontierState& S, int32_t t) { return (t & 1) ? S.stage_b : S.stage; }

// Slot of state q of wave-local string b at position t in the dense
// [Bw][2][Q] arrays.
__device__ __forceinline__ int64_t acc_slot(const FrontierState& S, int32_t b, int32_t t, int32_t q) {
  return ((int64_t)b * 2 + (t & 1)) * S.Q + q;
}
// Its Viterbi key, forward sum and forward maximum.
__device__ __forceinline__ unsigned long long* vit_key(const FrontierState& S, int64_t slot) {
  return S.acc + slot * S.acc_stride;
}
__device__ __forceinline__ unsigned long long* fwd_sum(const FrontierState& S, int64_t slot) { return S.acc + 2 * slot; }
__device__ __forceinline__ unsigned long long* fwd_max(const FrontierState& S, int64_t slot) {
  return S.acc + 2 * slot + 1;
}

// Compact accumulators: open-addressing hash tables with linear probing.
// A slot's first word is its key, (string + 1) << 32 | state (0 = empty):
// a table holds one position of each string, and keying by the string
// rather than the token puts a state that stays live two positions later
// in the same slot, whose line is then still in L2;
// the next word the Viterbi key or the forward maximum, and in forward
// tables the third the fixed-point sum.
__device__ __forceinline__ bool compact(const FrontierState& S) { return S.hmask != 0ull; }
__device__ __forceinline__ int hwords(const FrontierState& S) { return 2 * S.acc_stride; }
__device__ __forceinline__ unsigned long long* htab(const FrontierState& S, int32_t t) {
  return (t & 1) ? S.htab1 : S.htab0;
}
__device__ __forceinline__ unsigned long long* btab(const FrontierState& S, int32_t t) {
  const int32_t r = t % 3;
  return r == 0 ? S.btab0 : (r == 1 ? S.btab1 : S.btab2);
}
__device__ __forceinline__ unsigned long long tab_key(int32_t b, int32_t q) {
  return ((unsigned long long)(uint32_t)(b + 1) << 32) | (unsigned long long)(uint32_t)q;
}
// Home slot: multiplicative (Fibonacci) hashing; bits 32 and up of the
// product depend on both the string and the state.
__device__ __forceinline__ uint64_t tab_home(unsigned long long k, uint64_t mask) {
  return ((k * 0x9E3779B97F4A7C15ull) >> 32) & mask;
}
// The slot of key k in a table of w words a slot: where it already is, or
// the first empty slot of its probe sequence, taken with a compare-and-swap
// (*fresh = true: this call inserted it).  -1: the table is full.
__device__ __forceinline__ int64_t tab_claim(unsigned long long* tab, int w, uint64_t mask, unsigned long long k,
                                             bool* fresh) {
  uint64_t h = tab_home(k, mask);
  for (uint64_t n = 0; n <= mask; ++n) {
    const unsigned long long old = atomicCAS(tab + h * (uint64_t)w, 0ull, k);
    if (old == 0ull || old == k) {
      *fresh = old == 0ull;
      return (int64_t)h;
    }
    h = (h + 1) & mask;
  }
  *fresh = false;
  return -1;
}
// The slot holding key k, its first two words in *e; -1 when absent.
__device__ __forceinline__ int64_t tab_find(const unsigned long long* tab, int w, uint64_t mask,
                                            unsigned long long k, ulonglong2* e) {
  uint64_t h = tab_home(k, mask);
  for (uint64_t n = 0; n <= mask; ++n) {
    const ulonglong2 x = __ldcg((const ulonglong2*)(tab + h * (uint64_t)w));
    if (x.x == k) {
      *e = x;
      return (int64_t)h;
    }
    if (x.x == 0ull) break;
    h = (h + 1) & mask;
  }
  return -1;
}

// The last block of a kernel to finish hands out consecutive ranges, in step
// order, to the step's tokens: prefix sums of their counts cnt[p] from
// *top (or 0), written per slot (slot_out) and, for the pool, per token
// (base_out, cnt_out); rng_out[0..1] gets the step's [begin, end) and *top
// the end.  The tokens from the first whose range would pass `cap` on get
// empty ranges (slot base INT64_MAX, so no flat index maps to them) and
// raise error bit 1: every status of the run then reports FST_ERR_OOM.
// Each thread takes RPT consecutive slots: it sums their counts (loads
// issued together), the block scans the thread totals (two warp levels),
// and the thread reloads its slots to write their ranges.  RPT * KT slots
// per round.
constexpr int RPT = 8;

__device__ void ranges_last_block(const TokenView& T, const StepView& V, const FrontierState& S,
                                  const uint32_t* cnt, int64_t* top, int64_t cap, int64_t* slot_out,
                                  int64_t* base_out, int32_t* cnt_out, int64_t* rng_out) {
  __shared__ int last;
  __shared__ long long wsum[KT / 32];
  __shared__ long long first_bad, carry;
  __shared__ int dsel;
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
    dsel = 0;
  }
  __syncthreads();
  for (int32_t c = 0; c < V.n; c += KT * RPT) {
    const int32_t k0 = c + (int32_t)threadIdx.x * RPT;
    // the thread's total first (its loads in flight together), then the
    // ranges, re-reading the counts from cache
    long long run = 0;
#pragma unroll
    for (int i = 0; i < RPT; ++i)
      if (k0 + i < V.n) run += (long long)__ldcg(cnt + __ldg(T.step_tok + V.slot0 + k0 + i));
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
    int32_t pv[RPT];
    uint32_t mv[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) pv[i] = k0 + i < V.n ? __ldg(T.step_tok + V.slot0 + k0 + i) : -1;
#pragma unroll
    for (int i = 0; i < RPT; ++i) mv[i] = pv[i] >= 0 ? __ldcg(cnt + pv[i]) : 0u;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      if (pv[i] < 0) break;
      const int32_t p = pv[i];
      const long long m = (long long)mv[i];
      const bool fit = base + m <= (long long)cap;
      if (!fit) atomicMin(&first_bad, base);
      slot_out[V.slot0 + k0 + i] = fit ? base : INT64_MAX;
      if (base_out) base_out[p] = fit ? base : 0;
      if (cnt_out) cnt_out[p] = fit ? (int32_t)m : 0;
      if (S.dense_min > 0) {
        // direction switch: a token with many live states whose string goes
        // on takes a dense value vector (while slots last)
        int32_t slot = -1;
        int32_t a = 0;
        if (fit && m >= S.dense_min && S.bw_n[__ldg(T.b + p)] > V.t &&
            (a = __ldg(T.sym + p + 1), __ldg(S.pull_lseg + a + 1) == __ldg(S.pull_lseg + a))) {
          const int k = atomicAdd(&dsel, 1);
          if (k < DENSE_SLOTS) {
            slot = k;
            S.dlist[(int64_t)V.t * DENSE_SLOTS + k] = p;
          }
        }
        S.dslot[p] = slot;
      }
      base += m;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += round;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long end = carry < first_bad ? carry : first_bad;
    if (first_bad != (long long)INT64_MAX) atomicOr(S.flags + 1, ERR_POOL);
    rng_out[0] = begin;
    rng_out[1] = end;
    if (top) *top = end;
    if (S.dense_min > 0) S.dcnt[V.t] = dsel < DENSE_SLOTS ? dsel : DENSE_SLOTS;
    S.flags[0] = 0u;
  }
}

// ======================================================================
// Block-flattened arc walks.  Thread i of a block owns the arcs
// [e0_i, e0_i + len_i) of one segment; the block visits the arcs of all its
// threads KT * VU at a time (VU arcs per thread, their loads in flight
// together), so a hub's segment (hundreds of arcs out of one state on one
// symbol) spreads over the block instead of holding up one thread.
// Reductions go through shared-memory atomics on order-independent
// operations (max, integer add), so their results do not depend on which
// thread met which arc.
// ======================================================================
constexpr int VU = 4;

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

template <class Ctx>
__device__ __forceinline__ int32_t block_stage(BlockScratch<Ctx>& sh, int32_t e0, int32_t len, const Ctx& mine) {
  int32_t total;
  const int32_t ex = block_excl(len, sh.wsum, &total);
  sh.excl[threadIdx.x] = ex;
  sh.e0[threadIdx.x] = e0;
  sh.ctx[threadIdx.x] = mine;
  sh.acc[threadIdx.x] = 0ull;
  __syncthreads();
  return total;
}

// Order key of a float64 value rounded to float32 (0 = -inf, nothing).
__device__ __forceinline__ uint32_t fkey64(double v) { return v == -INFINITY ? 0u : fkey((float)v); }

// Reductions over each thread's segment: Op maps a value to a 64-bit key,
// combines keys atomically and maps the result back.
struct RedMaxD {  // exact max of float64 values through their order keys (0 = nothing)
  typedef double T;
  static __device__ __forceinline__ unsigned long long key(T v) { return v == -INFINITY ? 0ull : dkey(v); }
  static __device__ __forceinline__ T value(unsigned long long k) { return k ? dkey_inv(k) : -INFINITY; }
  static __device__ __forceinline__ void atomic(unsigned long long* a, unsigned long long k) { if (k) atomicMax(a, k); }
};
struct RedSum {  // exact integer sum
  typedef unsigned long long T;
  static __device__ __forceinline__ unsigned long long key(T v) { return v; }
  static __device__ __forceinline__ T value(unsigned long long k) { return k; }
  static __device__ __forceinline__ void atomic(unsigned long long* a, unsigned long long k) { if (k) atomicAdd(a, k); }
};

// Atomic max of key into a[p] for the lanes that hold one (p >= 0), with one
// atomic per run of equal p: the lanes of a warp hold consecutive flat
// entries, so equal tokens are adjacent and a segmented max over the warp
// (five shuffle rounds) leaves each run's maximum on its last lane.  All 32
// lanes call it.
__device__ __forceinline__ void warp_max_by_token(uint32_t* a, int32_t p, uint32_t key) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t k2 = __shfl_up_sync(FULL, key, d);
    const int32_t p2 = __shfl_up_sync(FULL, p, d);
    if (lane >= d && p2 == p) key = k2 > key ? k2 : key;
  }
  const int32_t pn = __shfl_down_sync(FULL, p, 1);
  if (p >= 0 && key != 0u && (lane == 31 || pn != p)) atomicMax(a + p, key);
}

// A slot in token p's staging list for every lane with want set: one
// atomicAdd per group of lanes with the same token.  All 32 lanes call it;
// returns the lane's index in the list (undefined when !want).
__device__ __forceinline__ uint32_t warp_stage_index(uint32_t* cnt, int32_t p, bool want) {
  const int lane = threadIdx.x & 31;
  const uint32_t wants = __ballot_sync(FULL, want);
  const uint32_t peers = __match_any_sync(FULL, want ? p : -1) & wants;
  const int head = peers ? __ffs(peers) - 1 : lane;
  uint32_t base = 0u;
  if (want && lane == head) base = atomicAdd(cnt + p, (uint32_t)__popc(peers));
  base = __shfl_sync(FULL, base, head);
  return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// ======================================================================
// Push (Alg. 1 / Alg. 2 forward loops over the arcs of live sources).
// ======================================================================
struct PushCtx {
  int32_t p;  // token of the destination position
  int32_t b;  // wave-local string
  double r;   // value of the source (Viterbi: a float32 score, held exactly)
};

// The arcs of every thread's segment out of a live source, pushed into
// position t: the atomic max on each destination's accumulator, and the
// staging of a destination met first.  VU arcs per thread a round, their
// loads and atomics issued together.  Compact accumulators take one
// compare-and-swap on the key (the home slot, almost always) and a max that
// returns nothing; the insert that took the slot stages it.  All threads of
// the block call it.
template <bool VIT>
__device__ __forceinline__ void block_push(const LayoutView& L, const TokenView& T, const FrontierState& S,
                                           int32_t t, BlockScratch<PushCtx>& sh, int32_t e0, int32_t len,
                                           const PushCtx& mine) {
  const int32_t total = block_stage(sh, e0, len, mine);
  const bool cpt = compact(S);
  unsigned long long* tab = htab(S, t);
  const int w = hwords(S);
  int32_t* stg = fwd_stage(S, t);
  for (int32_t a0 = 0; a0 < total; a0 += KT * VU) {
    int oo[VU];
    int4 arc[VU];
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      const int32_t a = a0 + u * KT + (int32_t)threadIdx.x;
      oo[u] = a < total ? block_owner(sh.excl, a) : -1;
      if (oo[u] >= 0 && !in_bounds(CHK_ARC, (long long)sh.e0[oo[u]] + (a - sh.excl[oo[u]]), L.P)) oo[u] = -1;
      arc[u] = oo[u] >= 0 ? __ldg(L.arcs + sh.e0[oo[u]] + (a - sh.excl[oo[u]])) : make_int4(0, 0, 0, 0);
    }
    unsigned long long cand[VU];
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      cand[u] = 0ull;
      if (oo[u] < 0) continue;
      const double r = sh.ctx[oo[u]].r;
      if (VIT) {
        // one rounded float32 addition per candidate
        const float x = __fadd_rn((float)r, __int_as_float(arc[u].y));
        if (x != neg_inf()) cand[u] = ((unsigned long long)fkey(x) << 32) | (unsigned long long)(~(uint32_t)arc[u].z);
      } else {
        // the exact float64 maximum (its term in the sum is then exactly 1)
        const double v = r + (double)__int_as_float(arc[u].y);
        if (v != -INFINITY) cand[u] = dkey(v);
      }
    }
    bool first[VU];
    int32_t sv[VU];  // the staged value: the state, or its slot
    if (cpt) {
      unsigned long long key[VU], old[VU];
      uint64_t h[VU];
#pragma unroll
      for (int u = 0; u < VU; ++u) {
        key[u] = cand[u] ? tab_key(sh.ctx[oo[u]].b, arc[u].x) : 0ull;
        h[u] = tab_home(key[u], S.hmask);
        old[u] = cand[u] ? atomicCAS(tab + h[u] * (uint64_t)w, 0ull, key[u]) : 0ull;
      }
#pragma unroll
      for (int u = 0; u < VU; ++u) {
        first[u] = cand[u] != 0ull && old[u] == 0ull;
        int64_t slot = (int64_t)h[u];
        if (cand[u] != 0ull && old[u] != 0ull && old[u] != key[u])  // the home slot holds another key
          slot = tab_claim(tab, w, S.hmask, key[u], &first[u]);
        if (cand[u] != 0ull) {
          if (slot < 0) {
            atomicOr(S.flags + 1, ERR_POOL);
          } else {
            atomicMax(tab + slot * w + 1, cand[u]);
          }
        }
        sv[u] = (int32_t)slot;
      }
    } else {
#pragma unroll
      for (int u = 0; u < VU; ++u) {
        first[u] = false;
        sv[u] = arc[u].x;
        if (cand[u] != 0ull) {
          const int64_t slot = acc_slot(S, sh.ctx[oo[u]].b, t, arc[u].x);
          if (in_bounds(CHK_ACC, slot, (long long)S.Bw * 2 * S.Q))
            first[u] = atomicMax(VIT ? vit_key(S, slot) : fwd_max(S, slot), cand[u]) == 0ull;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      const int32_t p = oo[u] >= 0 ? sh.ctx[oo[u]].p : 0;
      const uint32_t i = warp_stage_index(S.scnt, p, first[u]);
      if (first[u] && in_bounds(CHK_STAGE, __ldg(T.stf + p) + i, S.stage_cap)) stg[__ldg(T.stf + p) + i] = sv[u];
    }
  }
  __syncthreads();
}

// Live source j of position t-1 for the tokens of position t: at t = 1 the
// start states of every token (j = token slot * nstart + start index), else
// the pool entries of position t-1 (V.x_*) whose string goes on to t.
struct Source {
  int32_t p;   // token at position t, -1 when the entry's string ends at t-1
  int32_t q;   // state
  double r;    // value at t-1 (the start weight at t = 1)
  bool head;   // first entry of its token (writes the token's scalars)
};
__device__ __forceinline__ Source source_at(const TokenView& T, const StepView& V, const FrontierState& S,
                                            const Owner& o, int64_t j) {
  Source x{-1, 0, 0.0, false};
  if (V.t == 1) {
    x.p = __ldg(T.step_tok + V.slot0 + (int32_t)(j / S.nstart));
    x.q = __ldg(S.start_q + (int32_t)(j % S.nstart));
    x.r = (double)__ldg(S.theta_s + x.q);
    x.head = j % S.nstart == 0;
  } else if (in_bounds(CHK_POOL_READ, j, S.pool_cap)) {
    const int32_t pp = __ldg(T.step_tok + V.x_slot0 + o.k);
    if (S.bw_n[__ldg(T.b + pp)] >= V.t) {
      x.p = pp + 1;
      x.q = __ldcg(S.pool_q + j);
      x.r = __ldcg(S.pool_d + j);
      x.head = o.first == j;
    }
  }
  return x;
}
// Range of the live sources of position t-1.
__device__ __forceinline__ void source_range(const StepView& V, const FrontierState& S, int64_t* R0, int64_t* R1) {
  if (V.t == 1) {
    *R0 = 0;
    *R1 = (int64_t)V.n * S.nstart;
  } else {
    *R0 = __ldcg(S.step_rng + 2 * V.x_t);
    *R1 = __ldcg(S.step_rng + 2 * V.x_t + 1);
  }
}
// The source's arcs on w_t: looked up at t = 1, stored in the pool by the
// forward step afterwards.
__device__ __forceinline__ Arcs source_arcs(const LayoutView& L, const TokenView& T, const StepView& V,
                                            const FrontierState& S, const Source& x, int64_t j) {
  return V.t == 1 ? find_arcs(L, __ldg(T.sym + x.p), x.q) : Arcs{__ldcg(S.pool_x + j), __ldcg(S.pool_n + j)};
}

// First position: the start states of every token push their arcs on w_1.
template <bool VIT>
__device__ __forceinline__ void first_position(const LayoutView& L, const TokenView& T, const StepView& V,
                                               const FrontierState& S, BlockScratch<PushCtx>& sh) {
  const int64_t R1 = (int64_t)V.n * S.nstart;
  for (int64_t cb = (int64_t)blockIdx.x * KT; cb < R1; cb += (int64_t)gridDim.x * KT) {
    const int64_t j = cb + threadIdx.x;
    int32_t e0 = 0, len = 0;
    PushCtx me{0, 0, 0.0};
    if (j < R1) {
      const Source x = source_at(T, V, S, Owner{0, 0}, j);
      const Arcs r = find_arcs(L, __ldg(T.sym + x.p), x.q);
      e0 = r.pos;
      len = r.len;
      me = PushCtx{x.p, __ldg(T.b + x.p), x.r};
    }
    block_push<VIT>(L, T, S, 1, sh, e0, len, me);
  }
  ranges_last_block(T, V, S, S.scnt, S.pool_top, S.pool_cap, S.slot_base, S.pool_base, S.pool_cnt, S.step_rng + 2);
}

// Chained launches of the per-position kernels (programmatic dependent
// launch).  A step kernel launched with programmatic stream serialization
// may be scheduled while the previous kernel of its stream still runs.  Its
// first instruction waits until that kernel has completed and its writes
// are visible (griddepcontrol.wait), so no access of the step precedes it;
// then it lets the next position's kernel be scheduled in turn.  What
// overlaps is the launch and block scheduling of position t+1 with the work
// of position t.  Launched without the attribute, both do nothing.
__device__ __forceinline__ void chain_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__global__ void __launch_bounds__(KT) k_vit_first(LayoutView L, TokenView T, StepView V, FrontierState S) {
  __shared__ BlockScratch<PushCtx> sh;
  chain_enter();
  first_position<true>(L, T, V, S, sh);
}
__global__ void __launch_bounds__(KT) k_fwd_first(LayoutView L, TokenView T, StepView V, FrontierState S) {
  __shared__ BlockScratch<PushCtx> sh;
  chain_enter();
  first_position<false>(L, T, V, S, sh);
}

// Flat entry j of position t: token p and its staging index i.
struct Entry {
  int32_t p, i;
};
__device__ __forceinline__ Entry step_entry(const TokenView& T, const StepView& V, const Owner& o, int64_t j) {
  Entry x;
  x.p = __ldg(T.step_tok + V.slot0 + o.k);
  x.i = (int32_t)(j - o.first);
  return x;
}

// ======================================================================
// One forward position, fused (Alg. 1 inner max, Sec. 5.1; Alg. 2 forward
// loop, Sec. 5.2): every destination staged at t becomes a pool entry, and
// every new live state pushes its arcs on w_{t+1} right away.
//   Viterbi: the accumulator holds the packed key of the best arc.
//   forward: r_t[d] = (M_d - m_{t-1}) + log(sum_d), M_d the largest
//   r_{t-1}[src] + theta over the live arcs into d, sum_d the fixed-point
//   sum of exp(r_{t-1}[src] + theta - M_d) and m_{t-1} the largest value of
//   the token's previous position.
// ======================================================================
template <bool VIT>
__device__ __forceinline__ void step_position(const LayoutView& L, const TokenView& T, const StepView& V,
                                              const FrontierState& S, BlockScratch<PushCtx>& sh) {
  const int lane = threadIdx.x & 31;
  const int32_t t = V.t;
  const bool pull = !VIT && S.dense_min > 0;
  if (pull && t >= 2) {
    // the dense vectors of position t-1 were last read by the pull and the
    // sum of position t: back to -inf
    const int32_t nd = __ldcg(S.dcnt + t - 1);
    for (int32_t k = 0; k < nd; ++k) {
      const int32_t p = __ldcg(S.dlist + (int64_t)(t - 1) * DENSE_SLOTS + k);
      const int64_t base = __ldcg(S.pool_base + p);
      const int32_t cnt = __ldcg(S.pool_cnt + p);
      double* D = S.dvec + ((int64_t)k * 2 + ((t - 1) & 1)) * S.Q;
      for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += (int64_t)gridDim.x * blockDim.x)
        D[__ldcg(S.pool_q + base + j)] = -INFINITY;
    }
  }
  const int64_t R0 = __ldcg(S.step_rng + 2 * t), R1 = __ldcg(S.step_rng + 2 * t + 1);
  const int32_t* stg = fwd_stage(S, t);
  for (int64_t cb = R0 + (int64_t)blockIdx.x * KT; cb < R1; cb += (int64_t)gridDim.x * KT) {
    const int64_t c0 = cb + (int64_t)(threadIdx.x & ~31);  // this warp's 32 entries (block-uniform loop)
    const int64_t j = c0 + lane;
    const Owner o = flat_owner(S.slot_base + V.slot0, V.n, c0, clamp_entry(j, c0, R1));
    int32_t e0 = 0, len = 0;
    PushCtx nx{0, 0, 0.0};
    int32_t mk_p = -1;  // forward: the token and order key of this lane's value
    uint32_t mk_key = 0u;
    if (j < R1 && in_bounds(CHK_POOL_WRITE, j, S.pool_cap) &&
        in_bounds(CHK_STAGE, __ldg(T.stf + step_entry(T, V, o, j).p) + step_entry(T, V, o, j).i, S.stage_cap)) {
      const Entry x = step_entry(T, V, o, j);
      const int32_t b = __ldg(T.b + x.p);
      const int32_t sv = __ldcg(stg + __ldg(T.stf + x.p) + x.i);  // the state, or its table slot
      const bool cpt = compact(S);
      unsigned long long* ce = cpt ? htab(S, t) + (int64_t)sv * hwords(S) : nullptr;
      ulonglong2 kv = make_ulonglong2(0ull, 0ull);  // compact: {key, Viterbi key or maximum}
      if (cpt) kv = __ldcg((const ulonglong2*)ce);
      const int32_t d = cpt ? (int32_t)(uint32_t)kv.x : sv;
      const int64_t slot = acc_slot(S, b, t, d);
      double r;
      if (VIT) {
        const unsigned long long key = cpt ? kv.y : __ldcg(vit_key(S, slot));
        const float rv = fkey_inv((uint32_t)(key >> 32));
        r = rv;
        S.pool_v[j] = rv;
        const int32_t id = (int32_t)(~(uint32_t)key);  // the best incoming arc
        S.pool_x[j] = id;
        if (!cpt) {
          // the predecessor entry: the source's entry at t-1, which the step
          // before this one recorded in the state map of that position
          S.pool_n[j] = t > 1 ? __ldcg(S.vmap + acc_slot(S, b, t - 1, __ldg(S.src_by_id + id))) : -1;
          S.vmap[slot] = (int32_t)j;
        }
      } else {
        const ulonglong2 a = cpt ? make_ulonglong2(__ldcg(ce + 2), kv.y) : __ldcg((const ulonglong2*)fwd_sum(S, slot));
        const float sh_prev = t > 1 ? decode_max(__ldcg(S.mkey + x.p - 1)) : 0.f;
        r = fix_log_sum64(dkey_inv(a.y) - (double)sh_prev, a.x);
        S.pool_d[j] = r;
        mk_p = x.p;
        mk_key = fkey64(r);
      }
      S.pool_q[j] = d;
      // the accumulator is emptied only once its value has been used: a store
      // issued right behind the load of the same word measured 25% slower
      asm volatile("" ::: "memory");
      if (cpt) {
        *(ulonglong2*)ce = make_ulonglong2(0ull, 0ull);
        if (!VIT) ce[2] = 0ull;
      } else if (VIT) {
        *vit_key(S, slot) = 0ull;
      } else {
        *(ulonglong2*)fwd_sum(S, slot) = make_ulonglong2(0ull, 0ull);
      }
      Arcs nxt{0, 0};
      if (V.x_n > 0 && S.bw_n[b] > t) {  // the string goes on to t+1
        nxt = find_arcs(L, __ldg(T.sym + x.p + 1), d);
        const int32_t ds = pull ? __ldcg(S.dslot + x.p) : -1;
        if (ds >= 0) {
          // a dense token: its value goes to the dense vector and the next
          // position pulls instead
          S.dvec[((int64_t)ds * 2 + (t & 1)) * S.Q + d] = r;
        } else {
          e0 = nxt.pos;
          len = nxt.len;
          nx = PushCtx{x.p + 1, b, r};
        }
      }
      if (!VIT) {
        S.pool_x[j] = nxt.pos;
        S.pool_n[j] = nxt.len;
      }
    }
    if (!VIT) warp_max_by_token(S.mkey, mk_p, mk_key);  // the step maximum m_t
    block_push<VIT>(L, T, S, t + 1, sh, e0, len, nx);
  }
  // pool ranges of position t+1's tokens (with the direction switch, the
  // sum launch of t+1 hands them out, after its pull has staged)
  if (V.x_n > 0 && !pull) {
    StepView Vn = V;
    Vn.t = V.x_t;
    Vn.n = V.x_n;
    Vn.slot0 = V.x_slot0;
    ranges_last_block(T, Vn, S, S.scnt, S.pool_top, S.pool_cap, S.slot_base, S.pool_base, S.pool_cnt,
                      S.step_rng + 2 * Vn.t);
  }
}

__global__ void __launch_bounds__(KT) k_vit_step(LayoutView L, TokenView T, StepView V, FrontierState S) {
  __shared__ BlockScratch<PushCtx> sh;
  chain_enter();
  step_position<true>(L, T, V, S, sh);
}

__global__ void __launch_bounds__(KT) k_fwd_step(LayoutView L, TokenView T, StepView V, FrontierState S) {
  __shared__ BlockScratch<PushCtx> sh;
  chain_enter();
  step_position<false>(L, T, V, S, sh);
}

// ======================================================================
// Direction switch (forward pass, dense accumulators).  The dense tokens of
// position s (DENSE_SLOTS at most, each with its values scattered into a
// dense vector by the forward step of s) pull over the destination-ordered
// slice of w_{s+1} inside the sum launch of s+1: a warp per 128-arc window,
// four consecutive 16-byte records per lane, the source values gathered
// from the dense vector.  The tokens were chosen on symbols whose slice has
// no segment longer than a window, so every destination's arcs lie in one
// window: the warp takes each destination's exact maximum (a forward and a
// backward segmented scan over the window's runs of equal destination),
// its fixed-point terms and their sum (a segmented scan), and writes the
// accumulator and stages the destination itself -- no atomics on the
// accumulators, and the same exact terms as the pushes.
// ======================================================================
// Segmented inclusive scans over a warp's 128 elements, 4 consecutive ones
// per lane: forward (runs start where head is set) and backward (runs end
// where tail is set).  op is associative and commutative (max, sum).
template <class V, class Op>
__device__ __forceinline__ void seg_scan_fwd(V (&a)[4], const bool (&head)[4], Op op) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 1; i < 4; ++i)
    if (!head[i]) a[i] = op(a[i - 1], a[i]);
  V carry = a[3];
  bool flag = head[0] || head[1] || head[2] || head[3];
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const V o = __shfl_up_sync(FULL, carry, dd);
    const bool of = __shfl_up_sync(FULL, flag, dd);
    if (lane >= dd) {
      if (!flag) carry = op(o, carry);
      flag = flag || of;
    }
  }
  const V in = __shfl_up_sync(FULL, carry, 1);
  if (lane > 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (head[i]) break;
      a[i] = op(in, a[i]);
    }
  }
}
template <class V, class Op>
__device__ __forceinline__ void seg_scan_bwd(V (&a)[4], const bool (&tail)[4], Op op) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 2; i >= 0; --i)
    if (!tail[i]) a[i] = op(a[i], a[i + 1]);
  V carry = a[0];
  bool flag = tail[0] || tail[1] || tail[2] || tail[3];
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const V o = __shfl_down_sync(FULL, carry, dd);
    const bool of = __shfl_down_sync(FULL, flag, dd);
    if (lane + dd < 32) {
      if (!flag) carry = op(carry, o);
      flag = flag || of;
    }
  }
  const V in = __shfl_down_sync(FULL, carry, 1);
  if (lane < 31) {
#pragma unroll
    for (int i = 3; i >= 0; --i) {
      if (tail[i]) break;
      a[i] = op(a[i], in);
    }
  }
}

__device__ __forceinline__ void pull_fused(const TokenView& T, const FrontierState& S, const PullView& R,
                                           int32_t s) {
  const int32_t nd = __ldcg(S.dcnt + s);
  if (nd <= 0) return;
  const int lane = threadIdx.x & 31;
  const int32_t t = s + 1;  // the destination position
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;; gw += warps) {
    // the dense token whose windows hold window gw (warp-uniform)
    int32_t k = -1, p = 0;
    int64_t w = 0, acc = 0;
    for (int32_t kk = 0; kk < nd; ++kk) {
      const int32_t pk = __ldcg(S.dlist + (int64_t)s * DENSE_SLOTS + kk);
      const int32_t a = __ldg(T.sym + pk + 1);
      const int64_t w0 = __ldg(R.win + a), nw = __ldg(R.win + a + 1) - w0;
      if (gw < acc + nw) {
        k = kk;
        p = pk;
        w = w0 + (gw - acc);
        break;
      }
      acc += nw;
    }
    if (k < 0) break;
    const int32_t b = __ldg(T.b + p);
    const double* D = S.dvec + ((int64_t)k * 2 + (s & 1)) * S.Q;
    const int64_t i0 = w * WIN + lane * 4;
    int4 r[4];
    float th[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      r[i] = __ldg(R.rec + i0 + i);
      th[i] = __ldg(R.theta + i0 + i);
    }
    double v[4];
    bool live[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (r[i].z >= 0 && !dead32(th[i])) ? __ldcg(D + r[i].x) : -INFINITY;
    unsigned long long fm[4], bm[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      live[i] = !dead64(v[i]);
      if (live[i]) v[i] += (double)th[i];
      fm[i] = bm[i] = live[i] ? dkey(v[i]) : 0ull;
    }
    // runs of equal destination
    const int32_t prev = __shfl_up_sync(FULL, r[3].y, 1), next = __shfl_down_sync(FULL, r[0].y, 1);
    bool head[4], tail[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      head[i] = i == 0 ? (lane == 0 || prev != r[0].y) : r[i].y != r[i - 1].y;
      tail[i] = i == 3 ? (lane == 31 || next != r[3].y) : r[i].y != r[i + 1].y;
    }
    auto mx = [](unsigned long long x, unsigned long long y) { return x > y ? x : y; };
    auto add = [](unsigned long long x, unsigned long long y) { return x + y; };
    seg_scan_fwd(fm, head, mx);
    seg_scan_bwd(bm, tail, mx);
    unsigned long long e[4], M[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      M[i] = mx(fm[i], bm[i]);  // the run's maximum, at every element of the run
      e[i] = live[i] ? fix_exp64(v[i], dkey_inv(M[i])) : 0ull;
    }
    seg_scan_fwd(e, head, add);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // the run's last element writes its destination's accumulator
      const bool want = tail[i] && M[i] != 0ull;
      if (want) {
        const int64_t slot = acc_slot(S, b, t, r[i].y);
        *fwd_max(S, slot) = M[i];
        *fwd_sum(S, slot) = e[i];
      }
      const uint32_t j = warp_stage_index(S.scnt, p + 1, want);
      if (want) fwd_stage(S, t)[__ldg(T.stf + p + 1) + j] = r[i].y;
    }
  }
}

// The fixed-point terms of every thread's segment, VU arcs per thread a
// round: the arcs, then each destination's maximum (compact: the home
// slot's key and maximum in one load), then integer adds that return
// nothing.  All threads of the block call it.
__device__ __forceinline__ void sum_push(const LayoutView& L, const FrontierState& S, int32_t t,
                                         BlockScratch<PushCtx>& sh, int32_t e0, int32_t len, const PushCtx& mine) {
  const int32_t total = block_stage(sh, e0, len, mine);
  const bool cpt = compact(S);
  unsigned long long* tab = htab(S, t);
  const int w = hwords(S);
  for (int32_t a0 = 0; a0 < total; a0 += KT * VU) {
    int oo[VU];
    int4 arc[VU];
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      const int32_t a = a0 + u * KT + (int32_t)threadIdx.x;
      oo[u] = a < total ? block_owner(sh.excl, a) : -1;
      arc[u] = oo[u] >= 0 ? __ldg(L.arcs + sh.e0[oo[u]] + (a - sh.excl[oo[u]])) : make_int4(0, 0, 0, 0);
    }
    double v[VU];
    unsigned long long* dst[VU];  // the sum word
    unsigned long long mk[VU];    // the maximum's order key
    if (cpt) {
      unsigned long long key[VU];
      ulonglong2 kv[VU];
      uint64_t h[VU];
#pragma unroll
      for (int u = 0; u < VU; ++u) {
        v[u] = oo[u] >= 0 ? sh.ctx[oo[u]].r + (double)__int_as_float(arc[u].y) : -INFINITY;
        key[u] = v[u] != -INFINITY ? tab_key(sh.ctx[oo[u]].b, arc[u].x) : 0ull;
        h[u] = tab_home(key[u], S.hmask);
        kv[u] = key[u] ? __ldcg((const ulonglong2*)(tab + h[u] * w)) : make_ulonglong2(0ull, 0ull);
      }
#pragma unroll
      for (int u = 0; u < VU; ++u) {
        dst[u] = nullptr;
        mk[u] = kv[u].y;
        if (key[u] == 0ull) continue;
        int64_t slot = (int64_t)h[u];
        // the step before inserted every destination with a finite value
        if (kv[u].x != key[u]) slot = tab_find(tab, w, S.hmask, key[u], &kv[u]);
        if (slot >= 0) {
          dst[u] = tab + slot * w + 2;
          mk[u] = kv[u].y;
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < VU; ++u) {
        v[u] = oo[u] >= 0 ? sh.ctx[oo[u]].r + (double)__int_as_float(arc[u].y) : -INFINITY;
        dst[u] = nullptr;
        mk[u] = 0ull;
        if (v[u] == -INFINITY) continue;
        const int64_t slot = acc_slot(S, sh.ctx[oo[u]].b, t, arc[u].x);
        dst[u] = fwd_sum(S, slot);
        mk[u] = __ldcg(fwd_max(S, slot));
      }
    }
#pragma unroll
    for (int u = 0; u < VU; ++u)
      if (dst[u]) atomicAdd(dst[u], fix_exp64(v[u], dkey_inv(mk[u])));
  }
  __syncthreads();
}

// Forward sum of position t: with every maximum M_d final, each live arc
// adds exp(r_{t-1}[src] + theta - M_d) to its destination in fixed point.
template <bool PULL>
__device__ __forceinline__ void sum_position(const LayoutView& L, const TokenView& T, const StepView& V,
                                             const FrontierState& S, const PullView& R,
                                             BlockScratch<PushCtx>& sh) {
  const int lane = threadIdx.x & 31;
  const int32_t t = V.t;
  const bool pull = PULL && S.dense_min > 0 && t >= 2;
  // the dense tokens of t-1 by the pull; their entries push nothing here
  if (pull) pull_fused(T, S, R, t - 1);
  int64_t R0, R1;
  source_range(V, S, &R0, &R1);
  for (int64_t cb = R0 + (int64_t)blockIdx.x * KT; cb < R1; cb += (int64_t)gridDim.x * KT) {
    const int64_t c0 = cb + (int64_t)(threadIdx.x & ~31);
    const int64_t j = c0 + lane;
    Owner o{0, 0};
    if (t > 1) o = flat_owner(S.slot_base + V.x_slot0, V.x_n, c0, clamp_entry(j, c0, R1));  // t is uniform
    int32_t e0 = 0, len = 0;
    PushCtx me{0, 0, 0.0};
    if (j < R1) {
      const Source x = source_at(T, V, S, o, j);
      if (x.p >= 0 && !(pull && __ldcg(S.dslot + x.p - 1) >= 0)) {
        const Arcs r = source_arcs(L, T, V, S, x, j);
        e0 = r.pos;
        len = r.len;
        me = PushCtx{x.p, __ldg(T.b + x.p), x.r};
      }
    }
    sum_push(L, S, t, sh, e0, len, me);
  }
  // with the direction switch, this launch hands out the pool ranges of t
  // (the pull staged destinations of t above)
  if (pull) ranges_last_block(T, V, S, S.scnt, S.pool_top, S.pool_cap, S.slot_base, S.pool_base, S.pool_cnt,
                              S.step_rng + 2 * t);
}

__global__ void __launch_bounds__(KT) k_fwd_sum(LayoutView L, TokenView T, StepView V, FrontierState S,
                                                PullView R) {
  __shared__ BlockScratch<PushCtx> sh;
  chain_enter();
  sum_position<true>(L, T, V, S, R, sh);
}

// ======================================================================
// Backward step of position t fused with the posteriors (Alg. 2 backward
// and count loops; Sec. 5.2).  For each live state q of position t-1 and
// its arcs e = q -> q' on w_t:
//   beta_{t-1}[q] = LSE_e theta_e + beta_t[q'] - e_t   (shifted by e_t, the
//                   largest backward value of position t),
//   gamma_t(e)   = exp(alpha_{t-1}[q] + theta_e + beta_t[q'] - log Z),
// the exponent formed in float64 from the stored (shifted) values and the
// float64 running shifts K = C_{t-1} + E_t - log Z.  States that are not
// live in the forward pass are never visited: their posteriors are zero and
// no backward value of theirs is read.
// ======================================================================
__device__ __forceinline__ void add_count(const CountView& C, int32_t id, float g) {
  if (C.batched) {
    atomicAdd(C.cnt64 + id, (double)g);
  } else {
    // compensated float32 summation (one string: one writer per arc and
    // step; read through L2, as a persistent pass meets the same arc at
    // later positions in other blocks)
    const float s0 = __ldcg(C.cnt + id), cmp = __ldcg(C.comp + id);
    const float y = __fsub_rn(g, cmp);
    const float s1 = __fadd_rn(s0, y);
    C.comp[id] = __fsub_rn(__fsub_rn(s1, s0), y);
    C.cnt[id] = s1;
  }
}

struct BwdCtx {
  int32_t b, n;
  float et;     // e_t (0 at the string's last position)
  float gw;     // the string's gradient weight
  double ra;    // r_{t-1}[q]
  double m;     // the segment's maximum (second pass)
  double K;     // C_{t-1} + E_t - log Z - m_{t-1}
};

// Compact accumulators: empty the backward values of the entries of
// position y (their slots in bslot), every block a share.
__device__ __forceinline__ void bwd_clear_position(const FrontierState& S, int32_t y) {
  const int64_t R0 = __ldcg(S.step_rng + 2 * y), R1 = __ldcg(S.step_rng + 2 * y + 1);
  unsigned long long* tab = btab(S, y);
  for (int64_t j = R0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < R1; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t h = __ldcg(S.bslot + j);
    if (h >= 0) *(ulonglong2*)(tab + 2 * (int64_t)h) = make_ulonglong2(0ull, 0ull);
  }
}

// Reduction over each thread's segment of arcs on w_t for the backward
// step.  VU arcs per thread a round: the arcs, then the backward values of
// their destinations (the final weight at the string's last position), the
// loads of a round issued together (compact: the home slot, almost always
// the key's), then term(arc, beta, ctx) folded into the segment owner's
// shared accumulator.
template <class Op, class F>
__device__ __forceinline__ typename Op::T bwd_reduce(BlockScratch<BwdCtx>& sh, const LayoutView& L,
                                                     const FrontierState& S, int32_t t, int32_t e0, int32_t len,
                                                     const BwdCtx& mine, F term) {
  const int32_t total = block_stage(sh, e0, len, mine);
  const bool cpt = compact(S);
  const unsigned long long* tab = cpt ? btab(S, t) : nullptr;
  for (int32_t a0 = 0; a0 < total; a0 += KT * VU) {
    int oo[VU];
    int4 arc[VU];
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      const int32_t a = a0 + u * KT + (int32_t)threadIdx.x;
      oo[u] = a < total ? block_owner(sh.excl, a) : -1;
      arc[u] = oo[u] >= 0 ? __ldg(L.arcs + sh.e0[oo[u]] + (a - sh.excl[oo[u]])) : make_int4(0, 0, 0, 0);
    }
    double ub[VU];
    if (cpt) {
      unsigned long long key[VU];
      ulonglong2 kv[VU];
#pragma unroll
      for (int u = 0; u < VU; ++u) {
        ub[u] = -INFINITY;
        key[u] = 0ull;
        kv[u] = make_ulonglong2(0ull, 0ull);
        if (oo[u] < 0) continue;
        const BwdCtx& c = sh.ctx[oo[u]];
        if (t == c.n) {
          ub[u] = (double)__ldg(S.theta_f + arc[u].x);
        } else {
          key[u] = tab_key(c.b, arc[u].x);
          kv[u] = __ldcg((const ulonglong2*)(tab + 2 * tab_home(key[u], S.hmask)));
        }
      }
#pragma unroll
      for (int u = 0; u < VU; ++u) {
        if (key[u] == 0ull) continue;
        // every destination of a live arc is live at t: absent means a
        // backward value of -inf, which was not stored
        if (kv[u].x != key[u] && kv[u].x != 0ull) tab_find(tab, 2, S.hmask, key[u], &kv[u]);
        if (kv[u].x == key[u]) ub[u] = __longlong_as_double((long long)kv[u].y);
      }
    } else {
#pragma unroll
      for (int u = 0; u < VU; ++u) {
        ub[u] = -INFINITY;
        if (oo[u] < 0) continue;
        const BwdCtx& c = sh.ctx[oo[u]];
        ub[u] = (t == c.n) ? (double)__ldg(S.theta_f + arc[u].x) : __ldcg(S.beta + acc_slot(S, c.b, t, arc[u].x));
      }
    }
#pragma unroll
    for (int u = 0; u < VU; ++u)
      if (oo[u] >= 0) Op::atomic(&sh.acc[oo[u]], Op::key(term(arc[u], ub[u], sh.ctx[oo[u]])));
  }
  __syncthreads();
  const typename Op::T r = Op::value(sh.acc[threadIdx.x]);
  __syncthreads();
  return r;
}

__device__ __forceinline__ void bwd_position(const LayoutView& L, const TokenView& T, const StepView& V,
                                             const FrontierState& S, const CountView& C, BlockScratch<BwdCtx>& sh) {
  const int lane = threadIdx.x & 31;
  const int32_t t = V.t;
  const bool cpt = compact(S);
  // the backward values of position t+1 were last read by the step before
  if (cpt && V.y_t > 0) bwd_clear_position(S, V.y_t);
  int64_t R0, R1;
  source_range(V, S, &R0, &R1);
  for (int64_t cb = R0 + (int64_t)blockIdx.x * KT; cb < R1; cb += (int64_t)gridDim.x * KT) {
    const int64_t c0 = cb + (int64_t)(threadIdx.x & ~31);
    const int64_t j = c0 + lane;
    Owner o{0, 0};
    if (t > 1) o = flat_owner(S.slot_base + V.x_slot0, V.x_n, c0, clamp_entry(j, c0, R1));  // t is uniform
    int32_t e0 = 0, len = 0, q = -1, p = -1;
    BwdCtx me{0, 0, 0.f, 0.f, 0.0, 0.0, 0.0};
    if (j < R1) {
      const Source x = source_at(T, V, S, o, j);
      const int32_t b = x.p >= 0 ? __ldg(T.b + x.p) : 0;
      const double lz = x.p >= 0 ? __ldcg(S.logz + b) : -INFINITY;
      if (lz != -INFINITY) {
        p = x.p;
        q = x.q;
        const int32_t n = S.bw_n[b];
        const float et = (t == n) ? 0.f : decode_max(__ldcg(S.ekey + p));
        const double tE = (t == n) ? 0.0 : __ldcg(S.esum + p + 1) + (double)et;
        if (x.head && t > 1) S.esum[p] = tE;  // E_t, read by the step at t-1
        const float mprev = (t == 1) ? 0.f : decode_max(__ldcg(S.mkey + p - 1));
        if (et != neg_inf()) {
          const Arcs r = source_arcs(L, T, V, S, x, j);
          e0 = r.pos;
          len = r.len;
        }
        me = BwdCtx{b, n, et, S.gweight ? S.gweight[b] : 1.f, x.r, 0.0,
                    (((t == 1) ? 0.0 : __ldcg(S.csum + p - 1)) + tE - lz) - (double)mprev};
      }
    }
    // theta_e + beta_t[q'] - e_t
    me.m = bwd_reduce<RedMaxD>(sh, L, S, t, e0, len, me, [&](const int4& a, double ub, const BwdCtx& c) -> double {
      const float th = __int_as_float(a.y);
      return (th == neg_inf() || ub == -INFINITY) ? -INFINITY : (double)th + (ub - (double)c.et);
    });
    const unsigned long long su = bwd_reduce<RedSum>(
        sh, L, S, t, e0, me.m == -INFINITY ? 0 : len, me, [&](const int4& a, double ub, const BwdCtx& c) {
          const float th = __int_as_float(a.y);
          if (th == neg_inf() || ub == -INFINITY) return 0ull;
          const double v = (double)th + (ub - (double)c.et);
          // the exponent adds terms of either sign and tens in size that
          // cancel to a small number: formed in float64
          const double ex = c.ra + v + c.K;
          add_count(C, a.z, __expf((float)ex) * c.gw);
          return fix_exp64(v, c.m);
        });
    int32_t ek_p = -1;
    uint32_t ek_key = 0u;
    if (cpt && t > 1 && j < R1) {
      // every entry of position t-1 names its slot (or none), so that the
      // step of position t-2 can empty the table behind it
      int32_t h = -1;
      if (q >= 0) {
        const double u = fix_log_sum64(me.m, su);
        if (u != -INFINITY) {
          unsigned long long* tab = btab(S, t - 1);
          bool fresh;
          const int64_t hh = tab_claim(tab, 2, S.hmask, tab_key(me.b, q), &fresh);
          if (hh < 0) {
            atomicOr(S.flags + 1, ERR_POOL);
          } else {
            tab[2 * hh + 1] = (unsigned long long)__double_as_longlong(u);
            h = (int32_t)hh;
          }
          ek_p = p - 1;
          ek_key = fkey64(u);
        }
      }
      S.bslot[j] = h;
    } else if (q >= 0 && t > 1) {
      const double u = fix_log_sum64(me.m, su);
      S.beta[acc_slot(S, me.b, t - 1, q)] = u;
      if (u != -INFINITY) {
        ek_p = p - 1;
        ek_key = fkey64(u);
      }
    } else if (q >= 0 && C.start64) {
      // t = 1: the item is a start state q, log beta_0[q] = u + E_1 and its
      // start posterior is exp(theta_s[q] + log beta_0[q] - log Z)
      const double u = fix_log_sum64(me.m, su);
      if (u != -INFINITY) atomicAdd(C.start64 + q, exp(me.ra + u + me.K) * (double)me.gw);
    }
    warp_max_by_token(S.ekey, ek_p, ek_key);  // the step maximum e_{t-1}
  }
}

__global__ void __launch_bounds__(KT) k_bwd_step(LayoutView L, TokenView T, StepView V, FrontierState S,
                                                 CountView C) {
  __shared__ BlockScratch<BwdCtx> sh;
  chain_enter();
  bwd_position(L, T, V, S, C, sh);
}

// ======================================================================
// Persistent passes: one cooperative launch runs every position of a pass,
// the positions separated by a grid-wide barrier instead of kernel
// boundaries.  The step view of position t is rebuilt on the device from the
// wave's step offsets.  Every wait of the barrier is bounded: past the limit
// it raises ERR_TIMEOUT, every block leaves at its next barrier, and the
// final kernels report FST_ERR_TIMEOUT for each string of the wave.
// ======================================================================
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// All blocks of the grid (G.expected of them) meet; returns false when the
// run was abandoned (this block's wait expired, or another block's did).
// The fences follow the usual grid-synchronisation pattern: writes before
// the barrier are visible to every block after it.
__device__ __forceinline__ bool grid_sync(const GridSync& G, uint32_t* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* gen = G.bar + 1;
    const uint32_t g0 = *gen;
    int good = 1;
    __threadfence();
    const uint32_t arrived = atomicAdd(G.bar, 1u) + 1u;
    if (arrived == G.expected) {
      atomicExch(G.bar, 0u);
      __threadfence();
      atomicAdd(G.bar + 1, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*gen == g0) {
        if (*(volatile uint32_t*)err & ERR_TIMEOUT) { good = 0; break; }
        if (global_ns() - t0 > G.limit_ns) {
          atomicOr(err, ERR_TIMEOUT);
          good = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ StepView step_at(const WaveSteps& D, int32_t t, int32_t x_t) {
  StepView V;
  V.t = t;
  V.slot0 = D.step0[t];
  V.n = D.step0[t + 1] - V.slot0;
  const bool hasx = x_t >= 1 && x_t <= D.tmax;
  V.x_t = hasx ? x_t : 0;
  V.x_slot0 = hasx ? D.step0[x_t] : 0;
  V.x_n = hasx ? D.step0[x_t + 1] - V.x_slot0 : 0;
  V.blocks = (int32_t)gridDim.x;
  V.y_t = 0;
  return V;
}

__global__ void __launch_bounds__(KT) k_vit_persist(LayoutView L, TokenView T, WaveSteps D, FrontierState S,
                                                    GridSync G) {
  __shared__ BlockScratch<PushCtx> sh;
  if (D.tmax < 1) return;
  first_position<true>(L, T, step_at(D, 1, 0), S, sh);
  if (!grid_sync(G, S.flags + 1)) return;
  for (int32_t t = 1; t <= D.tmax; ++t) {
    step_position<true>(L, T, step_at(D, t, t + 1), S, sh);
    if (!grid_sync(G, S.flags + 1)) return;
  }
}

__global__ void __launch_bounds__(KT) k_fwd_persist(LayoutView L, TokenView T, WaveSteps D, FrontierState S,
                                                    GridSync G) {
  __shared__ BlockScratch<PushCtx> sh;
  if (D.tmax < 1) return;
  first_position<false>(L, T, step_at(D, 1, 0), S, sh);
  if (!grid_sync(G, S.flags + 1)) return;
  for (int32_t t = 1; t <= D.tmax; ++t) {
    sum_position<false>(L, T, step_at(D, t, t - 1), S, PullView{nullptr, nullptr, nullptr}, sh);
    if (!grid_sync(G, S.flags + 1)) return;
    step_position<false>(L, T, step_at(D, t, t + 1), S, sh);
    if (!grid_sync(G, S.flags + 1)) return;
  }
}

__global__ void __launch_bounds__(KT) k_bwd_persist(LayoutView L, TokenView T, WaveSteps D, FrontierState S,
                                                    CountView C, GridSync G) {
  __shared__ BlockScratch<BwdCtx> sh;
  // a forward pass that gave up leaves nothing to walk back over
  if (*(volatile uint32_t*)(S.flags + 1) & ERR_TIMEOUT) return;
  for (int32_t t = D.tmax; t >= 1; --t) {
    StepView V = step_at(D, t, t - 1);
    V.y_t = t + 1 < D.tmax ? t + 1 : 0;
    bwd_position(L, T, V, S, C, sh);
    if (!grid_sync(G, S.flags + 1)) return;
  }
  if (compact(S) && D.tmax >= 2) bwd_clear_position(S, 1);
}

__global__ void k_bwd_clear(FrontierState S, int32_t y) { bwd_clear_position(S, y); }

// ======================================================================
// Epilogues: final reductions (Alg. 1 return line; Alg. 2 Z), backtrace
// (Sec. 5.1), and counts back to caller arc order.  A string's candidates
// are the live states of its last position (its pool entries), or the
// start states when it is empty.
// ======================================================================
__global__ void __launch_bounds__(FT) k_vit_final(FrontierState S, float* __restrict__ scores,
                                                  int32_t* __restrict__ jfinal, int32_t* __restrict__ status) {
  __shared__ unsigned long long red[FT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = blockIdx.x;
  const int32_t n = S.bw_n[b];
  const int64_t p = S.bw_off[b] + n - 1;
  // a run that stopped early (pool overflow, barrier timeout) may not have
  // handed out the last position's pool range: read no candidates then
  const uint32_t err = S.flags[1] & (ERR_POOL | ERR_TIMEOUT);
  const int64_t base = (n == 0 || err) ? 0 : S.pool_base[p];
  const int32_t* cand = n == 0 ? S.start_q : S.pool_q + base;
  const int32_t ncand = err ? 0 : (n == 0 ? S.nstart : S.pool_cnt[p]);
  // best (score, lowest state) key; the low word holds ~state, and for the
  // pool entry the search below finds the index
  unsigned long long best = 0ull;
  for (int32_t i = threadIdx.x; i < ncand; i += FT) {
    const int32_t q = cand[i];
    if (q < 0) continue;
    const float a = n == 0 ? __ldg(S.theta_s + q) : S.pool_v[base + i];
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
  best = red[0];
  for (int w = 1; w < FT / 32; ++w) best = red[w] > best ? red[w] : best;
  const bool oom = err != 0u;
  const int32_t qbest = best ? (int32_t)(~(uint32_t)best) : -1;
  if (threadIdx.x == 0) {
    scores[b] = (best && !oom) ? fkey_inv((uint32_t)(best >> 32)) : neg_inf();
    if (status) status[b] = err ? run_error(err) : (best ? FST_OK : FST_ERR_NO_PATH);
    if (!best || oom || n == 0) jfinal[b] = -1;
  }
  // the entry holding the best state (each state appears once per token)
  if (best && !oom && n > 0)
    for (int32_t i = threadIdx.x; i < ncand; i += FT)
      if (cand[i] == qbest) jfinal[b] = (int32_t)(base + i);
}

// One thread per string, from the last position back: each pool entry
// names its best incoming arc and the entry of that arc's source, so the
// path is a chain of loads with no search.
//
// With compact accumulators there is no state map to record predecessor
// entries: a block per string finds each predecessor among the pool entries
// of the previous token (each state is there once), BB at a time.
constexpr int BB = 512;
__global__ void __launch_bounds__(BB) k_backtrace_scan(FrontierState S, const int32_t* __restrict__ olabel_by_id,
                                                       const int32_t* __restrict__ jfinal,
                                                       int32_t* __restrict__ paths, int32_t* __restrict__ olabels) {
  __shared__ int32_t found;
  const int64_t b = blockIdx.x;
  const int32_t n = S.bw_n[b];
  const int64_t off = S.bw_off[b];
  int32_t j = jfinal[b];
  int32_t t = n;
  for (; t >= 1 && j >= 0; --t) {
    const int32_t id = S.pool_x[j];
    if (threadIdx.x == 0) {
      paths[off + t - 1] = id;
      if (olabels) olabels[off + t - 1] = olabel_by_id[id];
      found = -1;
    }
    __syncthreads();
    if (t > 1) {
      const int32_t src = __ldg(S.src_by_id + id);
      const int64_t p = off + t - 2;  // the token of position t-1
      const int64_t base = S.pool_base[p];
      const int32_t cnt = S.pool_cnt[p];
      for (int32_t i0 = 0; i0 < cnt; i0 += BB) {
        const int32_t i = i0 + (int32_t)threadIdx.x;
        const bool hit = i < cnt && S.pool_q[base + i] == src;
        if (hit) found = (int32_t)(base + i);
        if (__syncthreads_or(hit)) break;  // the same answer in every thread
      }
    }
    j = found;  // the predecessor entry (none at the first position)
    __syncthreads();
  }
  for (int32_t u = threadIdx.x; u < t; u += BB) {  // no path (or an entry chain cut short): markers
    paths[off + u] = -1;
    if (olabels) olabels[off + u] = -1;
  }
}

__global__ void k_backtrace(FrontierState S, const int32_t* __restrict__ olabel_by_id, int32_t Bw,
                            const int32_t* __restrict__ jfinal, int32_t* __restrict__ paths,
                            int32_t* __restrict__ olabels) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= Bw) return;
  const int32_t n = S.bw_n[b];
  const int64_t off = S.bw_off[b];
  int32_t j = jfinal[b];
  int32_t t = n;
  for (; t >= 1 && j >= 0; --t) {
    const int32_t id = S.pool_x[j];
    paths[off + t - 1] = id;
    if (olabels) olabels[off + t - 1] = olabel_by_id[id];
    j = S.pool_n[j];
  }
  for (; t >= 1; --t) {  // no path (or an entry chain cut short): markers
    paths[off + t - 1] = -1;
    if (olabels) olabels[off + t - 1] = -1;
  }
}

// log Z of one string (Alg. 2, Z): C_{n-1} + log sum_q exp(r_n[q] + final[q]).
// Warp 0 first writes the running normalisers C_t (a warp scan, float64).
__global__ void __launch_bounds__(FT) k_fb_final(FrontierState S, double* __restrict__ logz,
                                                 int32_t* __restrict__ status) {
  __shared__ double red_m[FT / 32];
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
  // a run that stopped early may not have handed out the last position's
  // pool range: read no candidates then
  const uint32_t err = S.flags[1] & (ERR_POOL | ERR_TIMEOUT);
  const int64_t base = (n == 0 || err) ? 0 : S.pool_base[p];
  const int32_t* cand = n == 0 ? S.start_q : S.pool_q + base;
  const int32_t ncand = err ? 0 : (n == 0 ? S.nstart : S.pool_cnt[p]);
  auto value = [&](int32_t i) -> double {
    const int32_t q = cand[i];
    if (q < 0) return -INFINITY;
    const double a = n == 0 ? (double)__ldg(S.theta_s + q) : S.pool_d[base + i];
    return a + (double)__ldg(S.theta_f + q);
  };
  // the candidates sit in the pool in scheduling order: the sum is made
  // order-independent (bitwise repeatable) by adding exp(v - max) as
  // integers, in units of 2^-62
  double mx = -INFINITY;
  for (int32_t i = threadIdx.x; i < ncand; i += FT) mx = fmax(mx, value(i));
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, d));
  if (lane == 0) red_m[warp] = mx;
  __syncthreads();
  for (int w = 0; w < FT / 32; ++w) mx = fmax(mx, red_m[w]);
  unsigned long long lo = 0ull, hi = 0ull;  // 128-bit accumulator
  if (mx != -INFINITY) {
    for (int32_t i = threadIdx.x; i < ncand; i += FT) {
      const double v = value(i);
      if (v == -INFINITY) continue;
      const unsigned long long u = __double2ull_rn(exp(v - mx) * 4611686018427387904.0);  // 2^62
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
    const double cp = c_prev;
    double lz = -INFINITY;
    if (!err && mx != -INFINITY && cp != -INFINITY) lz = cp + mx + log(sum);
    logz[b] = lz;
    if (status) status[b] = err ? run_error(err) : ((lz == -INFINITY) ? FST_ERR_NO_PATH : FST_OK);
  }
}

// Final-state posteriors: exp(alpha_n[q] + theta_f[q] - log Z) for every
// live state q of a string's last position, alpha_n = r_n + C_{n-1} (Alg. 2
// at t = n); an empty string's path starts and ends in the same state.
__global__ void __launch_bounds__(FT) k_final_post(FrontierState S, CountView C) {
  const int64_t b = blockIdx.x;
  const double lz = S.logz[b];
  if (lz == -INFINITY) return;
  const int32_t n = S.bw_n[b];
  const double g = S.gweight ? (double)S.gweight[b] : 1.0;
  if (n == 0) {
    for (int32_t i = threadIdx.x; i < S.nstart; i += FT) {
      const int32_t q = S.start_q[i];
      const double v = (double)__ldg(S.theta_s + q) + (double)__ldg(S.theta_f + q);
      if (v == -INFINITY) continue;
      const double post = exp(v - lz) * g;
      if (C.final64) atomicAdd(C.final64 + q, post);
      if (C.start64) atomicAdd(C.start64 + q, post);
    }
    return;
  }
  if (!C.final64) return;
  const int64_t p = S.bw_off[b] + n - 1;
  const double cprev = n >= 2 ? S.csum[p - 1] : 0.0;
  const int64_t base = S.pool_base[p];
  const int32_t cnt = S.pool_cnt[p];
  for (int32_t i = threadIdx.x; i < cnt; i += FT) {
    const int32_t q = S.pool_q[base + i];
    const float tf = __ldg(S.theta_f + q);
    if (tf == neg_inf()) continue;
    atomicAdd(C.final64 + q, exp((S.pool_d[base + i] + (double)tf) + cprev - lz) * g);
  }
}

__global__ void k_fill_neg_inf(double* __restrict__ p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = -INFINITY;
}

__global__ void k_to_float(const double* __restrict__ in, int64_t n, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

__global__ void k_counts_out(int64_t A, CountView C, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A) return;
  out[i] = C.batched ? (float)C.cnt64[i] : __fsub_rn(C.cnt[i], C.comp[i]);
}

__global__ void k_clear_if_overflow(const uint32_t* __restrict__ flag, unsigned long long* __restrict__ acc,
                                    int64_t n) {
  if (!(*flag & (ERR_POOL | ERR_TIMEOUT))) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc[i] = 0ull;
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

int g_grid[6] = {0, 0, 0, 0, 0, 0};

// Chained launches are on unless FSTGPU_CHAIN=0.
bool chain_on() {
  static const bool on = [] {
    const char* e = std::getenv("FSTGPU_CHAIN");
    return !(e && e[0] == '0');
  }();
  return on;
}

// Launch a step kernel (KT threads, static shared memory only), chained to
// the previous kernel of its stream when the state asks for it: a chain of
// one stream's positions gains the launch latency; stream-parallel parts
// run unchained, where the early-scheduled blocks of one part would hold
// SM slots that the other parts' running positions need.
template <class... KArgs, class... Args>
int launch_step(void (*kernel)(KArgs...), unsigned grid, cudaStream_t s, const char* what, bool chain,
                Args... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(KT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = chain && chain_on() ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_fail(e, what);
  }
  return check_launch(what);
}

}  // namespace

int launch_vit_first(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                     cudaStream_t s) {
  return launch_step(k_vit_first, step_grid(k_vit_first, &g_grid[0], V), s, "k_vit_first", S.chain != 0, L, T, V, S);
}

int launch_fwd_first(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                     cudaStream_t s) {
  return launch_step(k_fwd_first, step_grid(k_fwd_first, &g_grid[1], V), s, "k_fwd_first", S.chain != 0, L, T, V, S);
}

int launch_vit_step(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                    cudaStream_t s) {
  return launch_step(k_vit_step, step_grid(k_vit_step, &g_grid[2], V), s, "k_vit_step", S.chain != 0, L, T, V, S);
}

int launch_fwd_step(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                    cudaStream_t s) {
  return launch_step(k_fwd_step, step_grid(k_fwd_step, &g_grid[3], V), s, "k_fwd_step", S.chain != 0, L, T, V, S);
}

int launch_fwd_sum(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                   const PullView& R, cudaStream_t s) {
  unsigned g = step_grid(k_fwd_sum, &g_grid[4], V);
  if (S.dense_min > 0) g = std::max(g, (unsigned)std::min(V.blocks * 4, 2048));  // room for the pull's windows
  return launch_step(k_fwd_sum, g, s, "k_fwd_sum", S.chain != 0, L, T, V, S, R);
}

int launch_bwd_step(const LayoutView& L, const TokenView& T, const StepView& V, const FrontierState& S,
                    const CountView& C, cudaStream_t s) {
  return launch_step(k_bwd_step, step_grid(k_bwd_step, &g_grid[5], V), s, "k_bwd_step", S.chain != 0, L, T, V, S, C);
}

// Largest co-resident grid of a persistent kernel on this device.
template <class K>
int persist_capacity(K kernel, int* cache) {
  if (*cache <= 0) {
    int dev = 0, sms = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, KT, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    *cache = sms * nb;
  }
  return *cache;
}
int g_persist_cap[3] = {0, 0, 0};

template <class K, class... Args>
int launch_persist(K kernel, int* cap_cache, int32_t grid, GridSync G, cudaStream_t s, const char* what,
                   Args... args) {
  const int cap = persist_capacity(kernel, cap_cache);
  if (cap <= 0 || grid < 1 || grid > cap) {
    set_error("%s: a grid of %d blocks cannot be co-resident (at most %d)", what, grid, cap);
    return FST_ERR_UNSUPPORTED;
  }
  G.expected += (uint32_t)grid;
  void* argv[sizeof...(Args) + 1];
  int i = 0;
  ((argv[i++] = (void*)&args), ...);
  argv[i] = (void*)&G;
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)kernel, dim3((unsigned)grid), dim3(KT), argv, 0, s);
  if (e != cudaSuccess) return cuda_fail(e, what);
  return FST_OK;
}

int debug_read(int64_t* violations, int32_t* code, int64_t* index, int64_t* bound) {
#ifdef FST_DEBUG
  unsigned long long h[4] = {0, 0, 0, 0};
  FST_CUDA(cudaMemcpyFromSymbol(h, g_dbg, sizeof(h)));
  const unsigned long long z[4] = {0, 0, 0, 0};
  FST_CUDA(cudaMemcpyToSymbol(g_dbg, z, sizeof(z)));
  if (violations) *violations = (int64_t)h[0];
  if (code) *code = (int32_t)h[1];
  if (index) *index = (int64_t)h[2];
  if (bound) *bound = (int64_t)h[3];
  return FST_OK;
#else
  (void)violations; (void)code; (void)index; (void)bound;
  set_error("this library was built without FST_DEBUG (no bounds checks)");
  return FST_ERR_UNSUPPORTED;
#endif
}

int persist_grid_limit(int which) {
  switch (which) {
    case 0: return persist_capacity(k_vit_persist, &g_persist_cap[0]);
    case 1: return persist_capacity(k_fwd_persist, &g_persist_cap[1]);
    default: return persist_capacity(k_bwd_persist, &g_persist_cap[2]);
  }
}

int launch_vit_persist(const LayoutView& L, const TokenView& T, const WaveSteps& D, const FrontierState& S,
                       int32_t grid, const GridSync& G, cudaStream_t s) {
  return launch_persist(k_vit_persist, &g_persist_cap[0], grid, G, s, "k_vit_persist", L, T, D, S);
}

int launch_fwd_persist(const LayoutView& L, const TokenView& T, const WaveSteps& D, const FrontierState& S,
                       int32_t grid, const GridSync& G, cudaStream_t s) {
  return launch_persist(k_fwd_persist, &g_persist_cap[1], grid, G, s, "k_fwd_persist", L, T, D, S);
}

int launch_bwd_persist(const LayoutView& L, const TokenView& T, const WaveSteps& D, const FrontierState& S,
                       const CountView& C, int32_t grid, const GridSync& G, cudaStream_t s) {
  return launch_persist(k_bwd_persist, &g_persist_cap[2], grid, G, s, "k_bwd_persist", L, T, D, S, C);
}

int launch_vit_final(const FrontierState& S, int32_t Bw, float* scores, int32_t* jfinal, int32_t* status,
                     cudaStream_t s) {
  if (Bw <= 0) return FST_OK;
  k_vit_final<<<(unsigned)Bw, FT, 0, s>>>(S, scores, jfinal, status);
  return check_launch("k_vit_final");
}

int launch_backtrace(const FrontierState& S, const int32_t* olabel_by_id, int32_t Bw, const int32_t* jfinal,
                     int32_t* paths, int32_t* olabels, cudaStream_t s) {
  if (Bw <= 0) return FST_OK;
  if (S.hmask != 0ull) {
    k_backtrace_scan<<<(unsigned)Bw, BB, 0, s>>>(S, olabel_by_id, jfinal, paths, olabels);
    return check_launch("k_backtrace_scan");
  }
  k_backtrace<<<(unsigned)((Bw + 127) / 128), 128, 0, s>>>(S, olabel_by_id, Bw, jfinal, paths, olabels);
  return check_launch("k_backtrace");
}

int launch_bwd_clear(const FrontierState& S, int32_t pos, int num_sms, cudaStream_t s) {
  if (S.hmask == 0ull || pos < 1) return FST_OK;
  k_bwd_clear<<<(unsigned)std::max(num_sms, 1) * 2, 256, 0, s>>>(S, pos);
  return check_launch("k_bwd_clear");
}

int launch_fb_final(const FrontierState& S, int32_t Bw, double* logz, int32_t* status, cudaStream_t s) {
  if (Bw <= 0) return FST_OK;
  k_fb_final<<<(unsigned)Bw, FT, 0, s>>>(S, logz, status);
  return check_launch("k_fb_final");
}

int launch_counts_out(int64_t A, const CountView& C, float* out, cudaStream_t s) {
  if (A <= 0) return FST_OK;
  k_counts_out<<<(unsigned)((A + 255) / 256), 256, 0, s>>>(A, C, out);
  return check_launch("k_counts_out");
}

int launch_final_posteriors(const FrontierState& S, int32_t Bw, const CountView& C, cudaStream_t s) {
  if (Bw <= 0 || (!C.final64 && !C.start64)) return FST_OK;
  k_final_post<<<(unsigned)Bw, FT, 0, s>>>(S, C);
  return check_launch("k_final_post");
}

int launch_fill_neg_inf(double* p, int64_t n, cudaStream_t s) {
  if (n <= 0) return FST_OK;
  k_fill_neg_inf<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(p, n);
  return check_launch("k_fill_neg_inf");
}

int launch_to_float(const double* in, int64_t n, float* out, cudaStream_t s) {
  if (n <= 0) return FST_OK;
  k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, n, out);
  return check_launch("k_to_float");
}

int launch_clear_if_overflow(const uint32_t* flag, unsigned long long* acc, int64_t n, int num_sms, cudaStream_t s) {
  if (n <= 0) return FST_OK;
  const int64_t blocks = std::min<int64_t>((int64_t)std::max(num_sms, 1) * 8, (n + 255) / 256);
  k_clear_if_overflow<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(flag, acc, n);
  return check_launch("k_clear_if_overflow");
}

}  // namespace fstgpu
