// prefix.cu -- the weight of a string by a parallel product over time.
//
// Eq. 1 is a product of the matrices delta[w_1] ... delta[w_n] between the
// start and final vectors.  Instead of a sweep over the positions, the
// matrices can be multiplied pairwise in parallel, and the products again,
// until one matrix is left (the parallel prefix approach of Sec. 6.1, which
// the paper leaves for future work).  Each product costs Q^3 instead of the
// Q^2 of a matrix-vector step, so this pays only for small dense FSTs and
// long strings: it takes log2(n) dependent rounds instead of n.
//
// Matrices are dense Q x Q log-weights (-inf = no arc), one per symbol of
// the string (parallel arcs combined: log-sum for the weight, max for the
// best path).  A product entry is log sum_k exp(A[i][k] + B[k][j]) (an
// online log-sum-exp over k, in float32) or max_k A[i][k] + B[k][j].  The
// Viterbi score so obtained is the best path's weight with its float32
// additions associated in tree order rather than left to right.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <vector>

#include "fst_internal.cuh"

using namespace fstgpu;

namespace {

constexpr int TB = 256;
constexpr int TILE = 16;  // output tile TILE x TILE, one thread per entry
constexpr int KC = 16;    // k chunk staged in shared memory
constexpr int PREFIX_MAX_STATES = 512;

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

__global__ void k_fill(float* __restrict__ p, int64_t n, float v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// log(e^a + e^b) with -inf handled.
__device__ __forceinline__ float log_add(float a, float b) {
  if (a == neg_inf()) return b;
  if (b == neg_inf()) return a;
  const float hi = fmaxf(a, b), lo = fminf(a, b);
  return hi + log1pf(expf(lo - hi));
}

// The dense matrices of one symbol: every arc of its slice adds into
// M[src][dst] (log-sum: a compare-and-swap loop; max: order keys).
__global__ void k_dense(const int4* __restrict__ arcs, const float* __restrict__ theta, int64_t i0, int64_t np,
                        int32_t Q, float* __restrict__ msum, uint32_t* __restrict__ mmax) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int4 a = __ldg(arcs + i0 + i);
  if (a.z < 0) return;
  const float th = __ldg(theta + i0 + i);
  if (th == neg_inf()) return;
  const int64_t e = (int64_t)a.x * Q + a.y;
  atomicMax(mmax + e, fkey(th));
  unsigned int* u = (unsigned int*)(msum + e);
  unsigned int old = *u, seen;
  do {
    seen = old;
    const float r = log_add(__uint_as_float(seen), th);
    if (__float_as_uint(r) == seen) break;
    old = atomicCAS(u, seen, __float_as_uint(r));
  } while (old != seen);
}

// Order keys (0 = no arc) to float32 values.
__global__ void k_keys_to_values(const uint32_t* __restrict__ k, int64_t n, float* __restrict__ v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = k[i] ? fkey_inv(k[i]) : neg_inf();
}

// out[p] = lhs[p] (x) rhs[p] for every pair p (blockIdx.y), one TILE x TILE
// tile of the result per block (blockIdx.x); MAXPLUS picks the semiring.
template <bool MAXPLUS>
__global__ void __launch_bounds__(TILE * TILE) k_mul(const float* const* __restrict__ lhs,
                                                     const float* const* __restrict__ rhs,
                                                     float* __restrict__ out, int32_t Q) {
  __shared__ float As[TILE][KC + 1];
  __shared__ float Bs[KC][TILE + 1];
  const int32_t tiles = (Q + TILE - 1) / TILE;
  const int32_t ti = blockIdx.x / tiles, tj = blockIdx.x % tiles;
  const int32_t r = threadIdx.x / TILE, c = threadIdx.x % TILE;
  const int32_t i = ti * TILE + r, j = tj * TILE + c;
  const float* A = lhs[blockIdx.y];
  const float* B = rhs[blockIdx.y];
  float m = neg_inf(), s = 0.f;  // log-sum: running max and sum of exp(v - m); max-plus: m
  for (int32_t k0 = 0; k0 < Q; k0 += KC) {
    // stage A[ti rows][k0..k0+KC) and B[k0..k0+KC)[tj cols]
    {
      const int32_t rr = threadIdx.x / KC, kk = threadIdx.x % KC;  // TILE * KC == blockDim
      const int32_t ai = ti * TILE + rr, ak = k0 + kk;
      As[rr][kk] = (ai < Q && ak < Q) ? A[(int64_t)ai * Q + ak] : neg_inf();
      const int32_t bk = k0 + threadIdx.x / TILE, bj = tj * TILE + threadIdx.x % TILE;
      Bs[threadIdx.x / TILE][threadIdx.x % TILE] = (bk < Q && bj < Q) ? B[(int64_t)bk * Q + bj] : neg_inf();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      const float a = As[r][kk], b = Bs[kk][c];
      if (a == neg_inf() || b == neg_inf()) continue;
      const float v = a + b;
      if (MAXPLUS) {
        m = fmaxf(m, v);
      } else if (v > m) {
        s = s * expf(m - v) + 1.f;  // m == -inf gives s * 0 + 1
        m = v;
      } else {
        s += expf(v - m);
      }
    }
    __syncthreads();
  }
  if (i < Q && j < Q)
    out[((int64_t)blockIdx.y * Q + i) * Q + j] = MAXPLUS ? m : (m == neg_inf() ? m : m + logf(s));
}

// log Z = LSE_{i,j}(theta_s[i] + P[i][j] + theta_f[j]) (float64) and the
// best score max_{i,j} fl(fl(theta_s[i] + V[i][j]) + theta_f[j]); one block.
// P == nullptr: the empty string (P and V the identity of their semiring).
__global__ void k_close(const float* __restrict__ P, const float* __restrict__ V, int32_t Q,
                        const float* __restrict__ ts, const float* __restrict__ tf, double* __restrict__ logz,
                        float* __restrict__ best) {
  __shared__ double red[TB / 32];
  __shared__ float redf[TB / 32];
  const int64_t QQ = (int64_t)Q * Q;
  auto val = [&](int64_t e, bool vit) -> float {
    const int32_t i = (int32_t)(e / Q), j = (int32_t)(e % Q);
    const float m = P ? (vit ? V[e] : P[e]) : (i == j ? 0.f : neg_inf());
    if (ts[i] == neg_inf() || m == neg_inf() || tf[j] == neg_inf()) return neg_inf();
    return __fadd_rn(__fadd_rn(ts[i], m), tf[j]);
  };
  double mx = -INFINITY;
  float bf = neg_inf();
  for (int64_t e = threadIdx.x; e < QQ; e += TB) {
    const int32_t i = (int32_t)(e / Q), j = (int32_t)(e % Q);
    const float m = P ? P[e] : (i == j ? 0.f : neg_inf());
    if (ts[i] != neg_inf() && m != neg_inf() && tf[j] != neg_inf())
      mx = fmax(mx, (double)ts[i] + (double)m + (double)tf[j]);
    bf = fmaxf(bf, val(e, true));
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(FULL, mx, d));
    bf = fmaxf(bf, __shfl_xor_sync(FULL, bf, d));
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = mx;
    redf[threadIdx.x >> 5] = bf;
  }
  __syncthreads();
  mx = red[0];
  bf = redf[0];
  for (int w = 1; w < TB / 32; ++w) {
    mx = fmax(mx, red[w]);
    bf = fmaxf(bf, redf[w]);
  }
  __syncthreads();
  double sum = 0.0;
  if (mx != -INFINITY)
    for (int64_t e = threadIdx.x; e < QQ; e += TB) {
      const int32_t i = (int32_t)(e / Q), j = (int32_t)(e % Q);
      const float m = P ? P[e] : (i == j ? 0.f : neg_inf());
      if (ts[i] != neg_inf() && m != neg_inf() && tf[j] != neg_inf())
        sum += exp((double)ts[i] + (double)m + (double)tf[j] - mx);
    }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) sum += __shfl_xor_sync(FULL, sum, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < TB / 32; ++w) t += red[w];
    *logz = mx == -INFINITY ? -INFINITY : mx + log(t);
    *best = bf;
  }
}

struct DevMem {
  std::vector<void*> p;
  template <class T>
  int get(T** out, int64_t n) {
    int rc = dalloc(out, n);
    if (!rc) p.push_back((void*)*out);
    return rc;
  }
  ~DevMem() {
    for (void* x : p) cudaFree(x);
  }
};

struct DevGuard {
  int old = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&old) != cudaSuccess) old = -1;
    if (old != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    if (old >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != old) cudaSetDevice(old);
  }
};

inline unsigned nb(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + TB - 1) / TB); }

}  // namespace

extern "C" int fst_prefix_log_z(fst_t* f, const int32_t* ids, int32_t n, double* log_z, float* best_score) {
  if (!f || n < 0 || (n > 0 && !ids) || !log_z || !best_score) {
    set_error("fst_prefix_log_z: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  if (f->Q > PREFIX_MAX_STATES) {
    set_error("fst_prefix_log_z: %d states; the dense product is for at most %d", f->Q, PREFIX_MAX_STATES);
    return FST_ERR_UNSUPPORTED;
  }
  for (int32_t i = 0; i < n; ++i)
    if (ids[i] < 0 || ids[i] >= f->m) {
      set_error("symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
      return FST_ERR_INVALID_ARG;
    }
  DevGuard g(f->device);
  cudaStream_t s = 0;
  const int64_t Q = f->Q, QQ = Q * Q;
  DevMem mem;
  int rc;
  double* d_logz = nullptr;
  float* d_best = nullptr;
  if ((rc = mem.get(&d_logz, 1)) || (rc = mem.get(&d_best, 1))) return rc;
  if (n == 0) {
    k_close<<<1, TB, 0, s>>>(nullptr, nullptr, f->Q, f->theta_s, f->theta_f, d_logz, d_best);
  } else {
    SliceView sv;
    if ((rc = slice_view(f, s, &sv))) return rc;
    // one dense pair (log-sum, max) per distinct symbol
    std::map<int32_t, int32_t> slot;
    for (int32_t i = 0; i < n; ++i) slot.emplace(ids[i], (int32_t)slot.size());
    const int64_t U = (int64_t)slot.size(), half = (n + 1) / 2;
    float *dsum = nullptr, *dmax = nullptr, *bufs[4] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t* keys = nullptr;
    const float** d_ptr = nullptr;
    if ((rc = mem.get(&dsum, U * QQ)) || (rc = mem.get(&dmax, U * QQ)) || (rc = mem.get(&keys, U * QQ)) ||
        (rc = mem.get(&bufs[0], half * QQ)) || (rc = mem.get(&bufs[1], half * QQ)) ||
        (rc = mem.get(&bufs[2], half * QQ)) || (rc = mem.get(&bufs[3], half * QQ)) ||
        (rc = mem.get(&d_ptr, 2 * half)))
      return rc;
    k_fill<<<nb(U * QQ), TB, 0, s>>>(dsum, U * QQ, -INFINITY);
    FST_CUDA(cudaMemsetAsync(keys, 0, (size_t)(U * QQ) * 4, s));
    for (const auto& kv : slot) {
      const int32_t a = kv.first;
      const int64_t i0 = sv.h_sym_win[a] * WIN, np = (sv.h_sym_win[a + 1] - sv.h_sym_win[a]) * WIN;
      if (np)
        k_dense<<<nb(np), TB, 0, s>>>(sv.arcs, sv.theta, i0, np, f->Q, dsum + kv.second * QQ,
                                      keys + kv.second * QQ);
    }
    k_keys_to_values<<<nb(U * QQ), TB, 0, s>>>(keys, U * QQ, dmax);
    FST_CUDA(cudaGetLastError());
    // the product tree, both semirings side by side: level by level,
    // adjacent pairs multiplied, an odd last matrix carried up
    std::vector<const float*> cur_s(n), cur_m(n);
    for (int32_t i = 0; i < n; ++i) {
      cur_s[i] = dsum + slot[ids[i]] * QQ;
      cur_m[i] = dmax + slot[ids[i]] * QQ;
    }
    int parity = 0;
    const int32_t tiles = (int32_t)((Q + TILE - 1) / TILE);
    while (cur_s.size() > 1) {
      const int64_t pairs = (int64_t)cur_s.size() / 2;
      float* out_s = bufs[parity];
      float* out_m = bufs[2 + parity];
      for (int sem = 0; sem < 2; ++sem) {
        const std::vector<const float*>& cur = sem ? cur_m : cur_s;
        std::vector<const float*> h(2 * pairs);
        for (int64_t p = 0; p < pairs; ++p) {
          h[p] = cur[2 * p];
          h[pairs + p] = cur[2 * p + 1];
        }
        FST_CUDA(cudaMemcpyAsync(d_ptr, h.data(), (size_t)(2 * pairs) * sizeof(float*), cudaMemcpyHostToDevice, s));
        for (int64_t p0 = 0; p0 < pairs; p0 += 65535) {
          const int64_t cnt = std::min<int64_t>(65535, pairs - p0);
          const dim3 grid((unsigned)(tiles * tiles), (unsigned)cnt);
          float* out = (sem ? out_m : out_s) + p0 * QQ;
          if (sem)
            k_mul<true><<<grid, TILE * TILE, 0, s>>>(d_ptr + p0, d_ptr + pairs + p0, out, f->Q);
          else
            k_mul<false><<<grid, TILE * TILE, 0, s>>>(d_ptr + p0, d_ptr + pairs + p0, out, f->Q);
        }
        FST_CUDA(cudaGetLastError());
        // the pointer table is rewritten for the other semiring only after
        // these launches have read it
        FST_CUDA(cudaStreamSynchronize(s));
      }
      std::vector<const float*> nxt_s(pairs), nxt_m(pairs);
      for (int64_t p = 0; p < pairs; ++p) {
        nxt_s[p] = out_s + p * QQ;
        nxt_m[p] = out_m + p * QQ;
      }
      if (cur_s.size() % 2) {
        // carry the odd one into this level's buffer (the buffer it sits in
        // is overwritten by the next level's products)
        FST_CUDA(cudaMemcpyAsync(out_s + pairs * QQ, cur_s.back(), (size_t)QQ * 4, cudaMemcpyDeviceToDevice, s));
        FST_CUDA(cudaMemcpyAsync(out_m + pairs * QQ, cur_m.back(), (size_t)QQ * 4, cudaMemcpyDeviceToDevice, s));
        nxt_s.push_back(out_s + pairs * QQ);
        nxt_m.push_back(out_m + pairs * QQ);
      }
      cur_s.swap(nxt_s);
      cur_m.swap(nxt_m);
      parity ^= 1;
    }
    k_close<<<1, TB, 0, s>>>(cur_s[0], cur_m[0], f->Q, f->theta_s, f->theta_f, d_logz, d_best);
  }
  FST_CUDA(cudaGetLastError());
  FST_CUDA(cudaMemcpy(log_z, d_logz, 8, cudaMemcpyDeviceToHost));
  FST_CUDA(cudaMemcpy(best_score, d_best, 4, cudaMemcpyDeviceToHost));
  if (*log_z == -INFINITY) {
    set_error("no accepting path");
    return FST_ERR_NO_PATH;
  }
  return FST_OK;
}
