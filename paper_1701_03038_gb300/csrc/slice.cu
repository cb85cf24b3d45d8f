// slice.cu -- the paper's own relaxation, kept for comparison.
//
// At each input position the paper relaxes every arc of the slice
// delta[w_t] (the arcs R[w_t] .. R[w_t+1]-1 of Fig. 2), one thread per arc,
// whether or not its source holds a finite value, and resolves collisions on
// a destination with a packed 64-bit atomicMax (Sec. 5.1).  fst_viterbi_slice
// decodes one string this way, so that the frontier-driven kernels can be
// measured against it on the same inputs.  The packed key is the one the
// frontier kernels use (order-preserving score bits << 32 | ~arc id), so the
// two give bit-identical results; the arcs are read as the paper lays them
// out: symbol-major, one record per arc (source, destination, id) and the
// weight array beside it.
//
// fst_forward_backward_slice is the paper's forward-backward the same way
// (Sec. 5.2): every arc of the slice adds its value into its destination's
// forward value (its source's backward value) with an atomic log-add-exp,
// a compare-and-swap loop over Eq. 3, in float32 as the paper keeps its
// log-probabilities; log Z and the per-arc posteriors follow Alg. 2.
//
// Within a slice the arcs can be ordered by destination (column-major, the
// CSC reading of Sec. 4) or by source (row-major, CSR; the paper sorts by
// source and notes that sorting by target helps its backward pass):
// fst_set_slice_order picks which, for the layout study.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "fst_internal.cuh"

using namespace fstgpu;

namespace {

constexpr int TB = 256;

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

// Slice records in the destination-segmented layout's padded order: the
// padding gets id -1.
__global__ void k_slice_pad(int4* __restrict__ arcs, int64_t P) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) arcs[i] = make_int4(0, 0, -1, 0);
}
// Records {source, destination, id} of a layout's segments: the segment
// state is the destination (by_source = false) or the source.
__global__ void k_slice_fill(const int32_t* __restrict__ seg_state, const int32_t* __restrict__ seg_pos,
                             const int32_t* __restrict__ seg_len, const int32_t* __restrict__ other,
                             const int32_t* __restrict__ arc_id, int64_t nseg, bool by_source,
                             int4* __restrict__ arcs) {
  const int64_t sg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sg >= nseg) return;
  const int32_t st = seg_state[sg], p0 = seg_pos[sg];
  for (int32_t i = 0; i < seg_len[sg]; ++i)
    arcs[p0 + i] = by_source ? make_int4(st, other[p0 + i], arc_id[p0 + i], 0)
                             : make_int4(other[p0 + i], st, arc_id[p0 + i], 0);
}

__global__ void k_fill_f32(float* __restrict__ p, int64_t n, float v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// *p = log(exp(*p) + exp(a)) atomically, a > -inf: the compare-and-swap
// loop of the paper's atomic log-add (Eq. 3: b + log1p(exp(a - b)) with
// a <= b), with -inf + a = a (reading of Eq. 3 for an empty sum).
__device__ __forceinline__ void atomic_log_add(float* p, float a) {
  unsigned int* u = (unsigned int*)p;
  unsigned int old = *u, seen;
  do {
    seen = old;
    const float b = __uint_as_float(seen);
    float r;
    if (b == neg_inf()) {
      r = a;
    } else {
      const float hi = fmaxf(a, b), lo = fminf(a, b);
      r = hi + log1pf(expf(lo - hi));
    }
    if (__float_as_uint(r) == seen) return;
    old = atomicCAS(u, seen, __float_as_uint(r));
  } while (old != seen);
}

// Forward, one position: alpha_t[dst] (+)= alpha_{t-1}[src] + theta.
__global__ void k_slice_fwd(const int4* __restrict__ arcs, const float* __restrict__ theta, int64_t i0, int64_t np,
                            const float* __restrict__ prev, float* __restrict__ cur) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int4 a = __ldg(arcs + i0 + i);
  if (a.z < 0) return;
  const float v = prev[a.x] + __ldg(theta + i0 + i);
  if (v == neg_inf()) return;
  atomic_log_add(cur + a.y, v);
}

// Backward, one position: beta_{t-1}[src] (+)= theta + beta_t[dst].
__global__ void k_slice_bwd(const int4* __restrict__ arcs, const float* __restrict__ theta, int64_t i0, int64_t np,
                            const float* __restrict__ next, float* __restrict__ cur) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int4 a = __ldg(arcs + i0 + i);
  if (a.z < 0) return;
  const float v = __ldg(theta + i0 + i) + next[a.y];
  if (v == neg_inf()) return;
  atomic_log_add(cur + a.x, v);
}

// log Z = log sum_q exp(alpha_n[q] + theta_f[q]), in float64 (one block).
__global__ void k_slice_logz(const float* __restrict__ alpha_n, const float* __restrict__ theta_f, int32_t Q,
                             double* __restrict__ logz) {
  __shared__ double red[TB / 32];
  double m = -INFINITY;
  for (int32_t q = threadIdx.x; q < Q; q += TB) m = fmax(m, (double)alpha_n[q] + (double)theta_f[q]);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) m = fmax(m, __shfl_xor_sync(FULL, m, d));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
  for (int w = 1; w < TB / 32; ++w) m = fmax(m, red[w]);
  __syncthreads();
  double sum = 0.0;
  if (m != -INFINITY)
    for (int32_t q = threadIdx.x; q < Q; q += TB) {
      const double v = (double)alpha_n[q] + (double)theta_f[q];
      if (v != -INFINITY) sum += exp(v - m);
    }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) sum += __shfl_xor_sync(FULL, sum, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < TB / 32; ++w) tot += red[w];
    *logz = (m == -INFINITY) ? -INFINITY : m + log(tot);
  }
}

// Posteriors of one position (Alg. 2's count loop, per arc):
// count[id] += exp(alpha_{t-1}[src] + theta + beta_t[dst] - log Z).
__global__ void k_slice_post(const int4* __restrict__ arcs, const float* __restrict__ theta, int64_t i0, int64_t np,
                             const float* __restrict__ prev, const float* __restrict__ next,
                             const double* __restrict__ logz, float* __restrict__ counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int4 a = __ldg(arcs + i0 + i);
  if (a.z < 0) return;
  const float al = prev[a.x], be = next[a.y], th = __ldg(theta + i0 + i);
  const double lz = *logz;
  if (al == neg_inf() || be == neg_inf() || th == neg_inf() || lz == -INFINITY) return;
  atomicAdd(counts + a.z, (float)exp((double)al + (double)th + (double)be - lz));
}

// One position: every arc of the slice [i0, i0 + np) of the padded layout.
// keys_prev == nullptr: the first position, sources valued by theta_s.
__global__ void k_slice_relax(const int4* __restrict__ arcs, const float* __restrict__ theta, int64_t i0,
                              int64_t np, const unsigned long long* __restrict__ keys_prev,
                              const float* __restrict__ theta_s, unsigned long long* __restrict__ keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int4 a = __ldg(arcs + i0 + i);
  if (a.z < 0) return;  // padding
  float v;
  if (keys_prev) {
    const unsigned long long k = keys_prev[a.x];
    if (!k) return;  // the source is -inf at t-1
    v = fkey_inv((uint32_t)(k >> 32));
  } else {
    v = __ldg(theta_s + a.x);
  }
  const float c = __fadd_rn(v, __ldg(theta + i0 + i));
  if (c == neg_inf()) return;
  atomicMax(keys + a.y, ((unsigned long long)fkey(c) << 32) | (unsigned long long)(~(uint32_t)a.z));
}

// Best final state (lowest id on ties), then the backtrace by thread 0.
__global__ void k_slice_final(const unsigned long long* __restrict__ keys, int32_t n, int32_t Q,
                              const float* __restrict__ theta_s, const float* __restrict__ theta_f,
                              const int32_t* __restrict__ src_by_id, float* __restrict__ score,
                              int32_t* __restrict__ path) {
  __shared__ unsigned long long red[TB / 32];
  const unsigned long long* last = keys + (int64_t)n * Q;
  unsigned long long best = 0ull;
  for (int32_t q = threadIdx.x; q < Q; q += TB) {
    float v;
    if (n == 0) {
      v = theta_s[q];
    } else {
      const unsigned long long k = last[q];
      v = k ? fkey_inv((uint32_t)(k >> 32)) : neg_inf();
    }
    const float c = __fadd_rn(v, theta_f[q]);
    if (c == neg_inf()) continue;
    const unsigned long long key = ((unsigned long long)fkey(c) << 32) | (unsigned long long)(~(uint32_t)q);
    best = key > best ? key : best;
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(FULL, best, d);
    best = o > best ? o : best;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < TB / 32; ++w) best = red[w] > best ? red[w] : best;
  best = red[0] > best ? red[0] : best;
  *score = best ? fkey_inv((uint32_t)(best >> 32)) : neg_inf();
  int32_t q = best ? (int32_t)(~(uint32_t)best) : -1;
  for (int32_t t = n; t >= 1; --t) {
    if (q < 0) {
      path[t - 1] = -1;
      continue;
    }
    const int32_t id = (int32_t)(~(uint32_t)keys[(int64_t)t * Q + q]);
    path[t - 1] = id;
    q = src_by_id[id];
  }
}

// The layout whose order the slice kernels read, and its records.
const Layout& slice_layout(const fst_s* f) { return f->slice_order == FST_SLICE_BY_SOURCE ? f->bwd : f->fwd; }
int4* slice_arcs(const fst_s* f) { return f->slice_order == FST_SLICE_BY_SOURCE ? f->slice_arcs_src : f->slice_arcs; }

// The slice records of the current order, built on first use.
int slice_records(fst_s* f, cudaStream_t s) {
  const bool by_src = f->slice_order == FST_SLICE_BY_SOURCE;
  int4** rec = by_src ? &f->slice_arcs_src : &f->slice_arcs;
  if (*rec) return FST_OK;
  const Layout& L = slice_layout(f);
  int rc;
  if ((rc = dalloc(rec, L.P))) return rc;
  if (L.P > 0) k_slice_pad<<<(unsigned)((L.P + TB - 1) / TB), TB, 0, s>>>(*rec, L.P);
  if (L.nseg > 0)
    k_slice_fill<<<(unsigned)((L.nseg + TB - 1) / TB), TB, 0, s>>>(L.seg_state, L.seg_pos, L.seg_len, L.other,
                                                                   L.arc_id, L.nseg, by_src, *rec);
  FST_CUDA(cudaGetLastError());
  return FST_OK;
}

inline unsigned nb(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + TB - 1) / TB); }

__global__ void k_gather_olabels(const int32_t* __restrict__ path, int32_t n, const int32_t* __restrict__ olabel,
                                 int32_t* __restrict__ out) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = path[i] >= 0 ? olabel[path[i]] : -1;
}

}  // namespace

namespace fstgpu {
int slice_records_dst(fst_s* f, cudaStream_t s) {
  const int32_t order = f->slice_order;
  f->slice_order = FST_SLICE_BY_DESTINATION;
  const int rc = slice_records(f, s);
  f->slice_order = order;
  return rc;
}

int slice_view(fst_s* f, cudaStream_t s, SliceView* out) {
  int rc = slice_records(f, s);
  if (rc) return rc;
  const Layout& L = slice_layout(f);
  *out = SliceView{slice_arcs(f), L.theta, L.h_sym_win};
  return FST_OK;
}
}  // namespace fstgpu

extern "C" int fst_set_slice_order(fst_t* f, int32_t order) {
  if (!f || (order != FST_SLICE_BY_DESTINATION && order != FST_SLICE_BY_SOURCE)) {
    set_error("fst_set_slice_order: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  f->slice_order = order;
  return FST_OK;
}

extern "C" int fst_forward_backward_slice(fst_t* f, const int32_t* ids, int32_t n, double* log_z,
                                          float* arc_posteriors) {
  if (!f || n < 0 || (n > 0 && !ids) || !log_z) {
    set_error("fst_forward_backward_slice: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  for (int32_t i = 0; i < n; ++i)
    if (ids[i] < 0 || ids[i] >= f->m) {
      set_error("symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
      return FST_ERR_INVALID_ARG;
    }
  const Layout& L = slice_layout(f);
  const int64_t Q = f->Q;
  cudaStream_t s = 0;
  int rc;
  if ((rc = slice_records(f, s))) return rc;
  const int4* arcs = slice_arcs(f);
  // forward and backward tables, (n+1) x Q each
  const int64_t need = 2 * (int64_t)(n + 1) * Q;
  if (need > f->slice_fb_cap) {
    dfree(f->slice_fb);
    f->slice_fb_cap = 0;
    if ((rc = dalloc(&f->slice_fb, need))) return rc;
    f->slice_fb_cap = need;
  }
  float* alpha = f->slice_fb;
  float* beta = f->slice_fb + (int64_t)(n + 1) * Q;
  double* d_logz = nullptr;
  float* d_cnt = nullptr;
  if ((rc = dalloc(&d_logz, 1))) return rc;
  if (arc_posteriors && (rc = dalloc(&d_cnt, std::max<int64_t>(f->A, 1)))) {
    dfree(d_logz);
    return rc;
  }
  const float NEG_INF = -INFINITY;
  // alpha_0 = theta_s, beta_n = theta_f, every other entry -inf
  k_fill_f32<<<nb(need), TB, 0, s>>>(f->slice_fb, need, NEG_INF);
  cudaError_t e = cudaMemcpyAsync(alpha, f->theta_s, (size_t)Q * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(beta + (int64_t)n * Q, f->theta_f, (size_t)Q * 4, cudaMemcpyDeviceToDevice, s);
  for (int32_t t = 1; t <= n && e == cudaSuccess; ++t) {
    const int32_t a = ids[t - 1];
    const int64_t i0 = L.h_sym_win[a] * WIN, np = (L.h_sym_win[a + 1] - L.h_sym_win[a]) * WIN;
    if (np) k_slice_fwd<<<nb(np), TB, 0, s>>>(arcs, L.theta, i0, np, alpha + (int64_t)(t - 1) * Q, alpha + (int64_t)t * Q);
  }
  for (int32_t t = n; t >= 1 && e == cudaSuccess; --t) {
    const int32_t a = ids[t - 1];
    const int64_t i0 = L.h_sym_win[a] * WIN, np = (L.h_sym_win[a + 1] - L.h_sym_win[a]) * WIN;
    if (np) k_slice_bwd<<<nb(np), TB, 0, s>>>(arcs, L.theta, i0, np, beta + (int64_t)t * Q, beta + (int64_t)(t - 1) * Q);
  }
  if (e == cudaSuccess) {
    k_slice_logz<<<1, TB, 0, s>>>(alpha + (int64_t)n * Q, f->theta_f, f->Q, d_logz);
    if (d_cnt) {
      e = cudaMemsetAsync(d_cnt, 0, (size_t)std::max<int64_t>(f->A, 1) * 4, s);
      for (int32_t t = 1; t <= n && e == cudaSuccess; ++t) {
        const int32_t a = ids[t - 1];
        const int64_t i0 = L.h_sym_win[a] * WIN, np = (L.h_sym_win[a + 1] - L.h_sym_win[a]) * WIN;
        if (np)
          k_slice_post<<<nb(np), TB, 0, s>>>(arcs, L.theta, i0, np, alpha + (int64_t)(t - 1) * Q,
                                             beta + (int64_t)t * Q, d_logz, d_cnt);
      }
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(log_z, d_logz, 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && d_cnt && f->A > 0)
    e = cudaMemcpy(arc_posteriors, d_cnt, (size_t)f->A * 4, cudaMemcpyDeviceToHost);
  dfree(d_logz);
  dfree(d_cnt);
  if (e != cudaSuccess) return cuda_fail(e, "fst_forward_backward_slice");
  if (*log_z == -INFINITY) {
    set_error("no accepting path");
    return FST_ERR_NO_PATH;
  }
  return FST_OK;
}

namespace fstgpu {
// Viterbi of one string by the slice-wide relaxation; host outputs (olabels
// may be NULL).  The score, path and output labels equal fst_viterbi's.
int viterbi_slice_run(fst_s* f, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path,
                      int32_t* olabels) {
  for (int32_t i = 0; i < n; ++i)
    if (ids[i] < 0 || ids[i] >= f->m) {
      set_error("symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
      return FST_ERR_INVALID_ARG;
    }
  const Layout& L = slice_layout(f);
  const int64_t Q = f->Q;
  int rc;
  cudaStream_t s = 0;
  if ((rc = slice_records(f, s))) return rc;
  const int64_t need = (int64_t)(n + 1) * Q;
  if (need > f->slice_cap) {
    dfree(f->slice_keys);
    f->slice_cap = 0;
    if ((rc = dalloc(&f->slice_keys, need))) return rc;
    f->slice_cap = need;
  }
  // output buffers kept by the handle: score, path and output labels
  if (n + 2 > f->slice_out_cap) {
    dfree(f->slice_out);
    f->slice_out_cap = 0;
    const int64_t c = std::max<int64_t>(2 * (int64_t)n + 4, 2 * f->slice_out_cap);
    if ((rc = dalloc(&f->slice_out, 2 * c + 1))) return rc;
    f->slice_out_cap = c;
  }
  float* d_score = (float*)f->slice_out;
  int32_t* d_path = f->slice_out + 1;
  int32_t* d_olab = f->slice_out + 1 + f->slice_out_cap;
  FST_CUDA(cudaMemsetAsync(f->slice_keys, 0, (size_t)need * 8, s));
  for (int32_t t = 1; t <= n; ++t) {
    const int32_t a = ids[t - 1];
    const int64_t i0 = L.h_sym_win[a] * WIN, np = (L.h_sym_win[a + 1] - L.h_sym_win[a]) * WIN;
    if (np == 0) continue;
    k_slice_relax<<<(unsigned)((np + TB - 1) / TB), TB, 0, s>>>(
        slice_arcs(f), L.theta, i0, np, t == 1 ? nullptr : f->slice_keys + (int64_t)(t - 1) * Q, f->theta_s,
        f->slice_keys + (int64_t)t * Q);
  }
  k_slice_final<<<1, TB, 0, s>>>(f->slice_keys, n, f->Q, f->theta_s, f->theta_f, f->src_by_id, d_score, d_path);
  if (olabels && n > 0) k_gather_olabels<<<nb(n), TB, 0, s>>>(d_path, n, f->olabel, d_olab);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(best_score, d_score, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(arc_path, d_path, (size_t)n * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && olabels && n > 0) e = cudaMemcpy(olabels, d_olab, (size_t)n * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "slice Viterbi");
  if (*best_score == -INFINITY) {
    set_error("no accepting path");
    return FST_ERR_NO_PATH;
  }
  return FST_OK;
}
}  // namespace fstgpu

extern "C" int fst_viterbi_slice(fst_t* f, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path) {
  if (!f || n < 0 || (n > 0 && (!ids || !arc_path)) || !best_score) {
    set_error("fst_viterbi_slice: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  return viterbi_slice_run(f, ids, n, best_score, arc_path, nullptr);
}
