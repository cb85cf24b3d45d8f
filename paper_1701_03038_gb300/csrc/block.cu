// block.cu -- one string on a small FST in one thread block.
//
// The paper relaxes the slice delta[w_t] of every input position with one
// thread per arc and one kernel launch per position (Sec. 5).  On a small
// FST (a thousand states, a few hundred arcs per slice) the launches, not
// the arcs, take the time: each position costs a launch and a round trip
// through global memory for a microsecond of work.  Here the position loop
// runs inside one block of 1024 threads: the values of every state at t-1
// and the accumulators of t sit in shared memory, the slice's arcs are
// read from L2, collisions on a destination go to shared-memory atomics,
// and __syncthreads() separates the positions.
//
//   Viterbi  -- the packed (order-preserving score bits << 32 | ~index)
//               atomicMax of Sec. 5.1, the index that of the arc in its
//               destination-ordered slice (lowest arc id on ties, as the
//               frontier kernels), a backpointer {arc, source} per state
//               and position in global memory (the sources also in shared
//               memory when the string's rows fit), the backtrace by one
//               thread, the path gathered by all;
//   forward  -- two sweeps of the slice per position: the exact float64
//               maximum of the arc values into each destination, then
//               exp(value - maximum) added in 2^-40 fixed point, both
//               order-independent; alpha_t in float64 to global memory;
//   backward -- the same two sweeps into each arc's source, beta_t in
//               shared memory and global memory.  The backward recursion
//               does not depend on alpha, so it runs in a second block at
//               the same time as the forward one;
//   posteriors -- once both have finished, a kernel over (position, slice
//               arc) pairs adds each arc's posterior (Alg. 2) in 2^-40 fixed
//               point (exact integer sums, bitwise repeatable).
//
// Values are kept unshifted in float64 (no per-position rescaling: float64
// holds the sums of log-probabilities of any string length used here).
// The float64 pipe of this part is narrow: a float64 exponential or
// logarithm costs the warp that holds a position's live arcs on the order of
// a microsecond, which the other warps wait out at the barrier.  The terms
// and logarithms of the log-sums stay float64 (their accuracy carries over
// hundreds of positions); a posterior term is exponentiated in float32 from
// a float64 argument, as in the batched kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <vector>

#include "fst_internal.cuh"

using namespace fstgpu;

namespace {

// threads of the block (a build-time tuning knob)
#ifndef FST_BLOCK_THREADS
#define FST_BLOCK_THREADS 1024
#endif
constexpr int BT = FST_BLOCK_THREADS;

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

// The padded slice of symbol a: positions [sym_win[a], sym_win[a+1]) x WIN.
struct Slice {
  int64_t i0, i1;
};
__device__ __forceinline__ Slice slice_of(const int64_t* __restrict__ sym_win, int32_t a) {
  return Slice{__ldg(sym_win + a) * WIN, __ldg(sym_win + a + 1) * WIN};
}

// Block-wide maximum of a 64-bit key (all threads get it).
__device__ __forceinline__ unsigned long long block_max_key(unsigned long long k, unsigned long long* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(FULL, k, d);
    k = o > k ? o : k;
  }
  __syncthreads();
  if (lane == 0) red[warp] = k;
  __syncthreads();
  k = red[0];
  for (int w = 1; w < BT / 32; ++w) k = red[w] > k ? red[w] : k;
  return k;
}

// Block-wide sum of a float64, in a fixed order (all threads get it).
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = 0.0;
  for (int w = 0; w < BT / 32; ++w) v += red[w];
  return v;
}

// The first KR * BT arcs of a slice, KR per thread, are held in registers
// for every sweep over the slice at a position; they are loaded one
// position ahead, so the loads of t+1 are in flight while t is relaxed.
// Arcs past them (slices longer than KR * BT) are read where they are used.
#ifndef FST_BLOCK_REG_ARCS
#define FST_BLOCK_REG_ARCS 2
#endif
constexpr int KR = FST_BLOCK_REG_ARCS;
struct ArcRegs {
  int4 r[KR];  // {source, destination, caller id (< 0: none), 0}
  float th[KR];
};
__device__ __forceinline__ void load_arcs(ArcRegs& R, const int4* __restrict__ arcs,
                                          const float* __restrict__ theta, const Slice& sl) {
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const int64_t i = sl.i0 + k * BT + threadIdx.x;
    R.r[k] = i < sl.i1 ? __ldg(arcs + i) : make_int4(0, 0, -1, 0);
    R.th[k] = i < sl.i1 ? __ldg(theta + i) : 0.f;
  }
}
__device__ __forceinline__ Slice slice_at(const int64_t* __restrict__ sym_win, const int32_t* __restrict__ ids,
                                          int32_t n, int32_t t) {
  return (t >= 1 && t <= n) ? slice_of(sym_win, __ldg(ids + t - 1)) : Slice{0, 0};
}

// ======================================================================
// Viterbi (Alg. 1, Sec. 5.1).  The slice records are the destination-
// ordered ones, where the arcs into a state sit in caller-id order, so the
// packed key carries the arc's index within the slice: the lowest index
// into a destination is its lowest arc id.  Shared: key[Q] (packed best
// arc into each state at t), v[Q] (float32 score of each state at t-1),
// rec[KR BT] ({caller id, source} of the register arcs, for the readout).
// bp[(t-1) Q + q] = {best arc, its source} of state q at position t.
// ======================================================================
__global__ void __launch_bounds__(BT, 1) k_block_viterbi(const int4* __restrict__ arcs,
                                                         const float* __restrict__ theta,
                                                         const int64_t* __restrict__ sym_win,
                                                         const int32_t* __restrict__ ids, int32_t n, int32_t Q,
                                                         const float* __restrict__ theta_s,
                                                         const float* __restrict__ theta_f,
                                                         const int32_t* __restrict__ olabel, int2* __restrict__ bp,
                                                         float* __restrict__ score, int32_t* __restrict__ path,
                                                         int32_t* __restrict__ olab, int32_t* __restrict__ status,
                                                         int32_t keep) {
  extern __shared__ unsigned long long smem[];
  __shared__ unsigned long long red[BT / 32];
  __shared__ int2 rec[KR * BT];
  unsigned long long* key = smem;
  float* v = (float*)(smem + Q);
  // keep: the state path qs[n + 1] and each position's best sources
  // src[(t - 1) Q + q] (0xffff: none; Q <= 8192) also in shared memory, so
  // that the backtrace walks shared rather than global memory
  int32_t* qs = (int32_t*)(v + Q);
  uint16_t* src = (uint16_t*)(qs + n + 1);
  for (int32_t q = threadIdx.x; q < Q; q += BT) {
    key[q] = 0ull;
    v[q] = __ldg(theta_s + q);
  }
  ArcRegs cur, nxt;
  load_arcs(cur, arcs, theta, slice_at(sym_win, ids, n, 1));
  __syncthreads();
  for (int32_t t = 1; t <= n; ++t) {
    const Slice sl = slice_at(sym_win, ids, n, t);
    load_arcs(nxt, arcs, theta, slice_at(sym_win, ids, n, t + 1));
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const int4 r = cur.r[k];
      rec[k * BT + threadIdx.x] = make_int2(r.z, r.x);
      if (r.z < 0) continue;  // padding, or past the slice
      const float x = v[r.x];
      if (x == neg_inf()) continue;
      const float c = __fadd_rn(x, cur.th[k]);
      if (c == neg_inf()) continue;
      atomicMax(key + r.y, ((unsigned long long)fkey(c) << 32) | (unsigned long long)(~(uint32_t)(k * BT + threadIdx.x)));
    }
    for (int64_t i = sl.i0 + KR * BT + threadIdx.x; i < sl.i1; i += BT) {
      const int4 r = __ldg(arcs + i);
      if (r.z < 0) continue;
      const float x = v[r.x];
      if (x == neg_inf()) continue;
      const float c = __fadd_rn(x, __ldg(theta + i));
      if (c == neg_inf()) continue;
      atomicMax(key + r.y, ((unsigned long long)fkey(c) << 32) | (unsigned long long)(~(uint32_t)(i - sl.i0)));
    }
    __syncthreads();
    int2* row = bp + (int64_t)(t - 1) * Q;
    for (int32_t q = threadIdx.x; q < Q; q += BT) {
      const unsigned long long k = key[q];
      int2 e = make_int2(-1, -1);
      if (k) {
        const int64_t j = (int64_t)(~(uint32_t)k);
        if (j < KR * BT) {
          e = rec[j];
        } else {
          const int4 r = __ldg(arcs + sl.i0 + j);
          e = make_int2(r.z, r.x);
        }
      }
      row[q] = e;
      if (keep) src[(int64_t)(t - 1) * Q + q] = e.y < 0 ? (uint16_t)0xffff : (uint16_t)e.y;
      v[q] = k ? fkey_inv((uint32_t)(k >> 32)) : neg_inf();
      key[q] = 0ull;
    }
    __syncthreads();
    cur = nxt;
  }
  // the best final state (lowest state id on ties)
  unsigned long long best = 0ull;
  for (int32_t q = threadIdx.x; q < Q; q += BT) {
    const float c = __fadd_rn(v[q], __ldg(theta_f + q));
    if (c == neg_inf()) continue;
    const unsigned long long k = ((unsigned long long)fkey(c) << 32) | (unsigned long long)(~(uint32_t)q);
    best = k > best ? k : best;
  }
  best = block_max_key(best, red);
  if (threadIdx.x == 0) {
    *score = best ? fkey_inv((uint32_t)(best >> 32)) : neg_inf();
    *status = best ? FST_OK : FST_ERR_NO_PATH;
  }
  if (keep) {
    if (threadIdx.x == 0) {
      int32_t q = best ? (int32_t)(~(uint32_t)best) : -1;
      for (int32_t t = n; t >= 1; --t) {
        qs[t] = q;
        const uint16_t p = q >= 0 ? src[(int64_t)(t - 1) * Q + q] : (uint16_t)0xffff;
        q = p == 0xffff ? -1 : (int32_t)p;
      }
    }
    __syncthreads();
    for (int32_t t = 1 + (int32_t)threadIdx.x; t <= n; t += BT) {
      const int32_t q = qs[t];
      const int2 e = q >= 0 ? bp[(int64_t)(t - 1) * Q + q] : make_int2(-1, -1);
      path[t - 1] = e.x;
      if (olab) olab[t - 1] = e.x >= 0 ? __ldg(olabel + e.x) : -1;
    }
    return;
  }
  if (threadIdx.x != 0) return;
  int32_t q = best ? (int32_t)(~(uint32_t)best) : -1;
  for (int32_t t = n; t >= 1; --t) {
    const int2 e = q >= 0 ? bp[(int64_t)(t - 1) * Q + q] : make_int2(-1, -1);
    path[t - 1] = e.x;
    if (olab) olab[t - 1] = e.x >= 0 ? __ldg(olabel + e.x) : -1;
    q = e.y;
  }
}

// ======================================================================
// Forward-backward (Alg. 2, Sec. 5.2).  Block 0 runs the forward pass and
// block 1 (when posteriors are wanted) the backward pass, each with its own
// shared mx[Q] (order key of the float64 maximum into each state), sm[Q]
// (fixed-point sum) and a[Q] (float64 values of the previous position).
// alpha[t Q + q] = alpha_t[q] and beta[t Q + q] = beta_t[q], t = 0..n.
// ======================================================================
__device__ __forceinline__ double state_value(unsigned long long m, unsigned long long s) {
  return m ? fix_log_sum64(dkey_inv(m), s) : -INFINITY;
}

// The forward pass (block 0): alpha_0 = theta_s, then alpha_t of every
// position; log Z and the status at the end.
__device__ void block_forward(const int4* __restrict__ arcs, const float* __restrict__ theta,
                              const int64_t* __restrict__ sym_win, const int32_t* __restrict__ ids, int32_t n,
                              int32_t Q, const float* __restrict__ theta_s, const float* __restrict__ theta_f,
                              double* __restrict__ alpha, double* __restrict__ logz, int32_t* __restrict__ status,
                              unsigned long long* mx, unsigned long long* sm, double* a, double* redd,
                              unsigned long long* redk) {
  for (int32_t q = threadIdx.x; q < Q; q += BT) {
    mx[q] = sm[q] = 0ull;
    a[q] = (double)__ldg(theta_s + q);
    alpha[q] = a[q];
  }
  ArcRegs cur, nxt;
  load_arcs(cur, arcs, theta, slice_at(sym_win, ids, n, 1));
  __syncthreads();
  for (int32_t t = 1; t <= n; ++t) {
    const Slice sl = slice_at(sym_win, ids, n, t);
    load_arcs(nxt, arcs, theta, slice_at(sym_win, ids, n, t + 1));
    // an arc counts when its source is live and its weight finite (then
    // the sum is finite too)
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      if (cur.r[k].z < 0 || dead32(cur.th[k])) continue;
      const double as = a[cur.r[k].x];
      if (dead64(as)) continue;
      atomicMax(mx + cur.r[k].y, dkey(as + (double)cur.th[k]));
    }
    for (int64_t i = sl.i0 + KR * BT + threadIdx.x; i < sl.i1; i += BT) {
      const int4 r = __ldg(arcs + i);
      const float th = __ldg(theta + i);
      if (r.z < 0 || dead32(th)) continue;
      const double as = a[r.x];
      if (dead64(as)) continue;
      atomicMax(mx + r.y, dkey(as + (double)th));
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      if (cur.r[k].z < 0 || dead32(cur.th[k])) continue;
      const double as = a[cur.r[k].x];
      if (dead64(as)) continue;
      atomicAdd(sm + cur.r[k].y, fix_exp64(as + (double)cur.th[k], dkey_inv(mx[cur.r[k].y])));
    }
    for (int64_t i = sl.i0 + KR * BT + threadIdx.x; i < sl.i1; i += BT) {
      const int4 r = __ldg(arcs + i);
      const float th = __ldg(theta + i);
      if (r.z < 0 || dead32(th)) continue;
      const double as = a[r.x];
      if (dead64(as)) continue;
      atomicAdd(sm + r.y, fix_exp64(as + (double)th, dkey_inv(mx[r.y])));
    }
    __syncthreads();
    double* row = alpha + (int64_t)t * Q;
    for (int32_t q = threadIdx.x; q < Q; q += BT) {
      a[q] = state_value(mx[q], sm[q]);
      row[q] = a[q];
      mx[q] = sm[q] = 0ull;
    }
    __syncthreads();
    cur = nxt;
  }
  // log Z = log sum_q exp(alpha_n[q] + theta_f[q]): exact maximum, then a
  // float64 sum in a fixed order
  unsigned long long mk = 0ull;
  for (int32_t q = threadIdx.x; q < Q; q += BT) {
    const float tf = __ldg(theta_f + q);
    if (dead64(a[q]) || dead32(tf)) continue;
    const unsigned long long k = dkey(a[q] + (double)tf);
    mk = k > mk ? k : mk;
  }
  mk = block_max_key(mk, redk);
  const double m = mk ? dkey_inv(mk) : -INFINITY;
  double part = 0.0;
  if (mk)
    for (int32_t q = threadIdx.x; q < Q; q += BT) {
      const float tf = __ldg(theta_f + q);
      if (dead64(a[q]) || dead32(tf)) continue;
      part += exp((a[q] + (double)tf) - m);
    }
  const double lz = mk ? m + log(block_sum(part, redd)) : -INFINITY;
  if (threadIdx.x == 0) {
    *logz = lz;
    *status = mk ? FST_OK : FST_ERR_NO_PATH;
  }
}

// The backward pass (block 1): beta_n = theta_f, then beta_{t-1} of every
// position from the slice of w_t, the log-sum taken into each arc's source.
__device__ void block_backward(const int4* __restrict__ arcs, const float* __restrict__ theta,
                               const int64_t* __restrict__ sym_win, const int32_t* __restrict__ ids, int32_t n,
                               int32_t Q, const float* __restrict__ theta_f, double* __restrict__ beta,
                               unsigned long long* mx, unsigned long long* sm, double* a) {
  for (int32_t q = threadIdx.x; q < Q; q += BT) {
    mx[q] = sm[q] = 0ull;
    a[q] = (double)__ldg(theta_f + q);
    beta[(int64_t)n * Q + q] = a[q];
  }
  ArcRegs cur, nxt;
  load_arcs(cur, arcs, theta, slice_at(sym_win, ids, n, n));
  __syncthreads();
  for (int32_t t = n; t >= 1; --t) {
    const Slice sl = slice_at(sym_win, ids, n, t);
    load_arcs(nxt, arcs, theta, slice_at(sym_win, ids, n, t - 1));
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      if (cur.r[k].z < 0 || dead32(cur.th[k])) continue;
      const double b = a[cur.r[k].y];
      if (dead64(b)) continue;
      atomicMax(mx + cur.r[k].x, dkey((double)cur.th[k] + b));
    }
    for (int64_t i = sl.i0 + KR * BT + threadIdx.x; i < sl.i1; i += BT) {
      const int4 r = __ldg(arcs + i);
      const float th = __ldg(theta + i);
      if (r.z < 0 || dead32(th)) continue;
      const double b = a[r.y];
      if (dead64(b)) continue;
      atomicMax(mx + r.x, dkey((double)th + b));
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      if (cur.r[k].z < 0 || dead32(cur.th[k])) continue;
      const double b = a[cur.r[k].y];
      if (dead64(b)) continue;
      atomicAdd(sm + cur.r[k].x, fix_exp64((double)cur.th[k] + b, dkey_inv(mx[cur.r[k].x])));
    }
    for (int64_t i = sl.i0 + KR * BT + threadIdx.x; i < sl.i1; i += BT) {
      const int4 r = __ldg(arcs + i);
      const float th = __ldg(theta + i);
      if (r.z < 0 || dead32(th)) continue;
      const double b = a[r.y];
      if (dead64(b)) continue;
      atomicAdd(sm + r.x, fix_exp64((double)th + b, dkey_inv(mx[r.x])));
    }
    __syncthreads();
    double* row = beta + (int64_t)(t - 1) * Q;
    for (int32_t q = threadIdx.x; q < Q; q += BT) {
      a[q] = state_value(mx[q], sm[q]);
      row[q] = a[q];
      mx[q] = sm[q] = 0ull;
    }
    __syncthreads();
    cur = nxt;
  }
}

// Block 0: the forward pass; block 1 (launched when posteriors are wanted):
// the backward pass, which also zeroes the fixed-point counts cnt [A].
__global__ void __launch_bounds__(BT, 1) k_block_fb(const int4* __restrict__ arcs, const float* __restrict__ theta,
                                                    const int64_t* __restrict__ sym_win,
                                                    const int32_t* __restrict__ ids, int32_t n, int32_t Q,
                                                    int64_t A, const float* __restrict__ theta_s,
                                                    const float* __restrict__ theta_f, double* __restrict__ alpha,
                                                    double* __restrict__ beta, unsigned long long* __restrict__ cnt,
                                                    double* __restrict__ logz, int32_t* __restrict__ status) {
  extern __shared__ unsigned long long smem[];
  __shared__ double redd[BT / 32];
  __shared__ unsigned long long redk[BT / 32];
  unsigned long long* mx = smem;
  unsigned long long* sm = smem + Q;
  double* a = (double*)(smem + 2 * Q);
  if (blockIdx.x == 0) {
    block_forward(arcs, theta, sym_win, ids, n, Q, theta_s, theta_f, alpha, logz, status, mx, sm, a, redd, redk);
  } else {
    for (int64_t i = threadIdx.x; i < A; i += BT) cnt[i] = 0ull;
    block_backward(arcs, theta, sym_win, ids, n, Q, theta_f, beta, mx, sm, a);
  }
}

// The posteriors of position t (block t - 1): for each arc of the slice of
// w_t, gamma = exp(alpha_{t-1}[src] + theta + beta_t[dst] - log Z) added to
// its arc's count in 2^-40 fixed point (gamma <= 1, fewer than 2^24
// positions: no overflow).  Nothing for a string without a path.
__global__ void __launch_bounds__(256) k_block_post(const int4* __restrict__ arcs, const float* __restrict__ theta,
                                                    const int64_t* __restrict__ sym_win,
                                                    const int32_t* __restrict__ ids, int32_t n, int32_t Q,
                                                    const double* __restrict__ alpha,
                                                    const double* __restrict__ beta,
                                                    const double* __restrict__ logz,
                                                    const int32_t* __restrict__ status,
                                                    unsigned long long* __restrict__ cnt) {
  if (*status != FST_OK) return;
  const int32_t t = (int32_t)blockIdx.x + 1;
  const Slice sl = slice_at(sym_win, ids, n, t);
  const double lz = *logz;
  const double* al = alpha + (int64_t)(t - 1) * Q;
  const double* be = beta + (int64_t)t * Q;
  for (int64_t i = sl.i0 + threadIdx.x; i < sl.i1; i += blockDim.x) {
    const int4 r = __ldg(arcs + i);
    const float th = __ldg(theta + i);
    if (r.z < 0 || dead32(th)) continue;
    const double x = al[r.x];
    if (dead64(x)) continue;
    const double b = be[r.y];
    if (dead64(b)) continue;
    const double u = (double)th + b;
    const float g = __expf((float)((x + u) - lz));
    atomicAdd(cnt + r.z, (unsigned long long)__float2ull_rn(g * 1099511627776.0f));  // 2^40
  }
}

// out[i] = cnt[i] / 2^40 as float32.
__global__ void k_block_post_out(const unsigned long long* __restrict__ cnt, int64_t A, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)((double)cnt[i] * 0x1p-40);
}

}  // namespace

namespace fstgpu {

bool block_fits(const fst_s* f) { return f->Q >= 1 && f->Q <= BLOCK_QMAX; }

// Grow a device buffer of T to at least `need` elements (doubling).
template <class T>
static int grow(T** p, int64_t* cap, int64_t need) {
  if (need <= *cap) return FST_OK;
  const int64_t c = std::max<int64_t>(need, 2 * *cap);
  dfree(*p);
  *cap = 0;
  const int rc = dalloc(p, c);
  if (rc) return rc;
  *cap = c;
  return FST_OK;
}

// Working memory of the block kernels: the string, its outputs, and n Q
// backpointers or (n + 1) Q forward values (in 8-byte words).
static int block_reserve(fst_s* f, int32_t n, int64_t words) {
  int rc;
  if ((rc = grow(&f->block_ids, &f->block_ids_cap, 3 * (int64_t)std::max(n, 1) + 4)) ||
      (rc = grow(&f->block_ws, &f->block_ws_cap, words)))
    return rc;
  return FST_OK;
}

// The dynamic shared memory a kernel may take, set once per device.
template <class K>
static int block_launch_setup(K kernel, int slot, size_t smem) {
  static int done[2][64];
  int dev = 0;
  FST_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && done[slot][dev]) return FST_OK;
  FST_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((size_t)BLOCK_QMAX * 24)));
  if (dev >= 0 && dev < 64) done[slot][dev] = 1;
  (void)smem;
  return FST_OK;
}

int viterbi_block_run(fst_s* f, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path,
                      int32_t* olabels, int32_t* status) {
  if (!block_fits(f)) {
    set_error("the one-block kernels hold at most %d states (this FST has %d)", BLOCK_QMAX, f->Q);
    return FST_ERR_UNSUPPORTED;
  }
  int rc;
  cudaStream_t s = 0;
  // the destination-ordered records, whichever order the slice kernels use
  SliceView sv;
  const int32_t order = f->slice_order;
  f->slice_order = FST_SLICE_BY_DESTINATION;
  rc = slice_view(f, s, &sv);
  f->slice_order = order;
  if (rc) return rc;
  const Layout& L = f->fwd;
  // block_ids: the string, then the path, the output labels, the score and
  // the status, read back with one copy
  if ((rc = block_reserve(f, n, (int64_t)std::max(n, 1) * f->Q))) return rc;
  const int64_t n1 = std::max(n, 1);
  int32_t* d_ids = f->block_ids;
  int32_t* d_path = d_ids + n1;
  int32_t* d_olab = d_ids + 2 * n1;
  float* d_score = (float*)(d_ids + 3 * n1);
  int32_t* d_status = d_ids + 3 * n1 + 1;
  if (n > 0) FST_CUDA(cudaMemcpyAsync(d_ids, ids, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  // the backtrace rows in shared memory when they fit the block's limit
  const size_t base = (size_t)f->Q * 12;
  const size_t kept = base + 4 * ((size_t)n + 1) + 2 * (size_t)n * (size_t)f->Q;
  const int32_t keep = kept <= (size_t)BLOCK_QMAX * 24 ? 1 : 0;
  const size_t smem = keep ? kept : base;
  if ((rc = block_launch_setup(k_block_viterbi, 0, smem))) return rc;
  k_block_viterbi<<<1, BT, smem, s>>>(sv.arcs, L.theta, L.sym_win, d_ids, n, f->Q, f->theta_s, f->theta_f,
                                      f->olabel, (int2*)f->block_ws, d_score, d_path, olabels ? d_olab : nullptr,
                                      d_status, keep);
  FST_CUDA(cudaGetLastError());
  std::vector<int32_t> h((size_t)(2 * n1 + 2));
  FST_CUDA(cudaMemcpy(h.data(), d_path, h.size() * 4, cudaMemcpyDeviceToHost));
  memcpy(best_score, &h[2 * n1], 4);
  *status = h[2 * n1 + 1];
  if (n > 0) {
    memcpy(arc_path, h.data(), (size_t)n * 4);
    if (olabels) memcpy(olabels, h.data() + n1, (size_t)n * 4);
  }
  return FST_OK;
}

int fb_block_run(fst_s* f, const int32_t* ids, int32_t n, float* arc_posteriors, double* log_z, int32_t* status) {
  if (!block_fits(f)) {
    set_error("the one-block kernels hold at most %d states (this FST has %d)", BLOCK_QMAX, f->Q);
    return FST_ERR_UNSUPPORTED;
  }
  int rc;
  cudaStream_t s = 0;
  SliceView sv;
  const int32_t order = f->slice_order;
  f->slice_order = FST_SLICE_BY_DESTINATION;
  rc = slice_view(f, s, &sv);
  f->slice_order = order;
  if (rc) return rc;
  const Layout& L = f->fwd;
  // block_ws: the posteriors [A floats], log Z and the status (read back
  // with one copy), the fixed-point counts [A], then the forward and the
  // backward values [(n + 1) Q] each
  const int64_t A = f->A;
  const int64_t Q = f->Q;
  const int64_t head = (A + 1) / 2 + 2;  // 8-byte words before the counts
  const int64_t rows = ((int64_t)n + 1) * Q;
  if ((rc = block_reserve(f, n, head + A + 2 * rows))) return rc;
  int32_t* d_ids = f->block_ids;
  float* d_out = (float*)f->block_ws;
  double* d_logz = (double*)(f->block_ws + head - 2);
  int32_t* d_status = (int32_t*)(f->block_ws + head - 1);
  unsigned long long* d_cnt = f->block_ws + head;
  double* d_alpha = (double*)(f->block_ws + head + A);
  double* d_beta = d_alpha + rows;
  if (n > 0) FST_CUDA(cudaMemcpyAsync(d_ids, ids, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  const size_t smem = (size_t)Q * 24;
  if ((rc = block_launch_setup(k_block_fb, 1, smem))) return rc;
  // block 0 the forward pass, block 1 the backward pass (posteriors only)
  k_block_fb<<<arc_posteriors ? 2 : 1, BT, smem, s>>>(sv.arcs, L.theta, L.sym_win, d_ids, n, f->Q, A, f->theta_s,
                                                      f->theta_f, d_alpha, d_beta, d_cnt, d_logz, d_status);
  FST_CUDA(cudaGetLastError());
  if (arc_posteriors) {
    if (n > 0)
      k_block_post<<<(unsigned)n, 256, 0, s>>>(sv.arcs, L.theta, L.sym_win, d_ids, n, f->Q, d_alpha, d_beta, d_logz,
                                               d_status, d_cnt);
    if (A > 0)
      k_block_post_out<<<(unsigned)std::min<int64_t>((A + 255) / 256, 4096), 256, 0, s>>>(d_cnt, A, d_out);
    FST_CUDA(cudaGetLastError());
    std::vector<unsigned long long> h((size_t)head);
    FST_CUDA(cudaMemcpy(h.data(), f->block_ws, (size_t)head * 8, cudaMemcpyDeviceToHost));
    memcpy(arc_posteriors, h.data(), (size_t)A * 4);
    memcpy(log_z, &h[head - 2], 8);
    memcpy(status, &h[head - 1], 4);
  } else {
    unsigned long long h[2];
    FST_CUDA(cudaMemcpy(h, f->block_ws + head - 2, 16, cudaMemcpyDeviceToHost));
    memcpy(log_z, &h[0], 8);
    memcpy(status, &h[1], 4);
  }
  return FST_OK;
}

}  // namespace fstgpu
