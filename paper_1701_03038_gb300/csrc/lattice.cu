// lattice.cu -- an acyclic input lattice composed with the FST.
//
// The paper decodes input strings and names input lattices as the general
// case its approach extends to (Sec. 6.1).  A lattice here is a DAG whose
// nodes are numbered in a topological order: node 0 is the start, node N-1
// the end, and edge e goes from from[e] to to[e] > from[e], reads symbol
// label[e] and carries the log-weight weight[e].  Its paths replace the one
// path of a string; the FST reads the symbols along them.  The recursions
// run node by node, and each edge relaxes every arc of its symbol's slice
// (the paper's slice-wide relaxation, Sec. 5) into dense per-node tables:
//   Viterbi  V[v][q'] = max over edges e = (u -> v) and arcs k = (q -> q') of
//            fl(fl(V[u][q] + theta_k) + w_e), packed 64-bit keys
//            (score << 32 | ~arc id) so that ties go to the lowest arc id;
//            the backtrace takes the lowest edge id among the edges that
//            reach the same score with that arc;
//   forward  alpha[v][q'] = log-sum-exp of alpha[u][q] + w_e + theta_k in
//            float64: an exact maximum (64-bit order keys), then exp(value -
//            maximum) summed in 2^-40 fixed point, as in the step kernels;
//   backward beta[u][q] likewise from the end node; log Z, and the
//            posterior of each arc (summed over the edges reading its
//            symbol) and of each edge (summed over its arcs).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "fst_internal.cuh"

using namespace fstgpu;

namespace {

constexpr int TB = 256;
inline unsigned nb(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + TB - 1) / TB); }

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

// Start node: the start weights as keys (no incoming arc: low word 0).
__global__ void k_lat_vit_init(const float* __restrict__ theta_s, int32_t Q, unsigned long long* __restrict__ keys0) {
  const int32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const float v = theta_s[q];
  keys0[q] = v == neg_inf() ? 0ull : ((unsigned long long)fkey(v) << 32);
}

// One edge u -> v: every arc of its slice with a live source.
__global__ void k_lat_vit_edge(const int4* __restrict__ arcs, const float* __restrict__ theta, int64_t i0, int64_t np,
                               const unsigned long long* __restrict__ keys_u, float w,
                               unsigned long long* __restrict__ keys_v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int4 a = __ldg(arcs + i0 + i);
  if (a.z < 0) return;
  const unsigned long long kp = keys_u[a.x];
  if (!kp) return;
  const float c = __fadd_rn(__fadd_rn(fkey_inv((uint32_t)(kp >> 32)), __ldg(theta + i0 + i)), w);
  if (c == neg_inf()) return;
  atomicMax(keys_v + a.y, ((unsigned long long)fkey(c) << 32) | (unsigned long long)(~(uint32_t)a.z));
}

__device__ __forceinline__ float key_score(unsigned long long k) {
  return k ? fkey_inv((uint32_t)(k >> 32)) : neg_inf();
}

// Best end state (lowest id on ties), then the backtrace by thread 0: at
// node v in state q the key names the best arc k; the edge is the lowest id
// into v that reads k's symbol and reaches the same score through it.  At
// most N-1 steps (each moves to a lower node).
__global__ void k_lat_vit_final(const unsigned long long* __restrict__ keys, int32_t N, int32_t Q,
                                const float* __restrict__ theta_f, const int32_t* __restrict__ in_off,
                                const int32_t* __restrict__ in_edge, const int32_t* __restrict__ efrom,
                                const int32_t* __restrict__ elabel, const float* __restrict__ eweight,
                                const int32_t* __restrict__ il_by_id, const float* __restrict__ th_by_id,
                                const int32_t* __restrict__ src_by_id, float* __restrict__ score,
                                int32_t* __restrict__ edge_path, int32_t* __restrict__ arc_path,
                                int32_t* __restrict__ path_len) {
  __shared__ unsigned long long red[TB / 32];
  const unsigned long long* last = keys + (int64_t)(N - 1) * Q;
  unsigned long long best = 0ull;
  for (int32_t q = threadIdx.x; q < Q; q += TB) {
    const float c = __fadd_rn(key_score(last[q]), theta_f[q]);
    if (c == neg_inf()) continue;
    const unsigned long long k = ((unsigned long long)fkey(c) << 32) | (unsigned long long)(~(uint32_t)q);
    best = k > best ? k : best;
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(FULL, best, d);
    best = o > best ? o : best;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 0; w < TB / 32; ++w) best = red[w] > best ? red[w] : best;
  *score = best ? fkey_inv((uint32_t)(best >> 32)) : neg_inf();
  int32_t len = 0;
  if (best) {
    int32_t v = N - 1, q = (int32_t)(~(uint32_t)best);
    for (int32_t step = 0; step < N - 1 && v != 0; ++step) {
      const unsigned long long kv = keys[(int64_t)v * Q + q];
      const int32_t k = (int32_t)(~(uint32_t)kv);
      if (!kv || k < 0) { len = -1; break; }
      const float s = key_score(kv);
      const int32_t src = src_by_id[k];
      int32_t e_best = -1;
      for (int32_t j = in_off[v]; j < in_off[v + 1]; ++j) {  // edges into v, by increasing id
        const int32_t e = in_edge[j];
        if (elabel[e] != il_by_id[k]) continue;
        const float vu = key_score(keys[(int64_t)efrom[e] * Q + src]);
        if (vu == neg_inf()) continue;
        if (__fadd_rn(__fadd_rn(vu, th_by_id[k]), eweight[e]) == s) { e_best = e; break; }
      }
      if (e_best < 0) { len = -1; break; }
      edge_path[len] = e_best;
      arc_path[len] = k;
      ++len;
      v = efrom[e_best];
      q = src;
    }
  }
  *path_len = len;
}

// Forward and backward relaxations of one edge (float64 values), in two
// phases: the exact maximum of each target, then the fixed-point sum.
// fwd: target = destination, value = tab_u[src] + w + theta;
// bwd: target = source, value = w + theta + tab_v[dst].
template <bool FWD, bool SUM>
__global__ void k_lat_lse_edge(const int4* __restrict__ arcs, const float* __restrict__ theta, int64_t i0, int64_t np,
                               const double* __restrict__ tab, double w, unsigned long long* __restrict__ maxk,
                               unsigned long long* __restrict__ sum) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int4 a = __ldg(arcs + i0 + i);
  if (a.z < 0) return;
  const double x = tab[FWD ? a.x : a.y];
  const float th = __ldg(theta + i0 + i);
  if (x == -INFINITY || th == neg_inf()) return;
  const double v = x + w + (double)th;
  const int32_t tgt = FWD ? a.y : a.x;
  if (!SUM)
    atomicMax(maxk + tgt, dkey(v));
  else
    atomicAdd(sum + tgt, fix_exp64(v, dkey_inv(maxk[tgt])));
}

// tab[q] = max + log(sum) (or -inf), and the accumulators back to zero.
__global__ void k_lat_lse_finish(unsigned long long* __restrict__ maxk, unsigned long long* __restrict__ sum,
                                 int32_t Q, double* __restrict__ tab) {
  const int32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const unsigned long long m = maxk[q];
  tab[q] = m ? fix_log_sum64(dkey_inv(m), sum[q]) : -INFINITY;
  maxk[q] = 0ull;
  sum[q] = 0ull;
}

__global__ void k_lat_from_f32(const float* __restrict__ in, int32_t Q, double* __restrict__ out) {
  const int32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < Q) out[q] = (double)in[q];
}

// log Z = LSE_q(alpha_end[q] + theta_f[q]) in float64 (one block).
__global__ void k_lat_logz(const double* __restrict__ alpha_end, const float* __restrict__ theta_f, int32_t Q,
                           double* __restrict__ logz) {
  __shared__ double red[TB / 32];
  double m = -INFINITY;
  for (int32_t q = threadIdx.x; q < Q; q += TB) m = fmax(m, alpha_end[q] + (double)theta_f[q]);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) m = fmax(m, __shfl_xor_sync(FULL, m, d));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
  for (int w = 1; w < TB / 32; ++w) m = fmax(m, red[w]);
  __syncthreads();
  double s = 0.0;
  if (m != -INFINITY)
    for (int32_t q = threadIdx.x; q < Q; q += TB) {
      const double v = alpha_end[q] + (double)theta_f[q];
      if (v != -INFINITY) s += exp(v - m);
    }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) s += __shfl_xor_sync(FULL, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < TB / 32; ++w) t += red[w];
    *logz = m == -INFINITY ? -INFINITY : m + log(t);
  }
}

// Posteriors through edge e: exp(alpha[u][src] + w + theta + beta[v][dst] - log Z)
// to each arc's count and to the edge's posterior.
__global__ void k_lat_post(const int4* __restrict__ arcs, const float* __restrict__ theta, int64_t i0, int64_t np,
                           const double* __restrict__ alpha_u, const double* __restrict__ beta_v, double w,
                           const double* __restrict__ logz, double* __restrict__ cnt, double* __restrict__ epost) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double g = 0.0;
  if (i < np) {
    const int4 a = __ldg(arcs + i0 + i);
    const float th = a.z >= 0 ? __ldg(theta + i0 + i) : neg_inf();
    const double lz = *logz;
    if (a.z >= 0 && th != neg_inf() && lz != -INFINITY) {
      const double al = alpha_u[a.x], be = beta_v[a.y];
      if (al != -INFINITY && be != -INFINITY) {
        g = exp(al + w + (double)th + be - lz);
        atomicAdd(cnt + a.z, g);
      }
    }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) g += __shfl_xor_sync(FULL, g, d);
  if ((threadIdx.x & 31) == 0 && g != 0.0) atomicAdd(epost, g);
}

__global__ void k_lat_to_f32(const double* __restrict__ in, int64_t n, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
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

// A validated lattice on the host: edges grouped by destination and by
// source node, each group in increasing edge id.
struct HostLattice {
  int32_t N = 0, E = 0;
  std::vector<int32_t> in_off, in_edge, out_off, out_edge;
};

int check_lattice(const fst_s* f, int32_t N, int32_t E, const int32_t* from, const int32_t* to, const int32_t* label,
                  const float* weight, HostLattice* L) {
  if (N < 1 || E < 0 || (E > 0 && (!from || !to || !label || !weight))) {
    set_error("lattice: bad sizes or NULL arrays");
    return FST_ERR_INVALID_ARG;
  }
  for (int32_t e = 0; e < E; ++e) {
    if (from[e] < 0 || to[e] <= from[e] || to[e] >= N) {
      set_error("lattice edge %d goes from node %d to node %d: edges must go to a higher node id below %d", e,
                from[e], to[e], N);
      return FST_ERR_INVALID_ARG;
    }
    if (label[e] < 0 || label[e] >= f->m) {
      set_error("lattice edge %d reads symbol %d outside [0, %d)", e, label[e], f->m);
      return FST_ERR_INVALID_ARG;
    }
    if (isnan(weight[e]) || weight[e] == INFINITY) {
      set_error("lattice edge %d has weight NaN or +inf", e);
      return FST_ERR_INVALID_ARG;
    }
  }
  L->N = N;
  L->E = E;
  L->in_off.assign(N + 1, 0);
  L->out_off.assign(N + 1, 0);
  for (int32_t e = 0; e < E; ++e) {
    ++L->in_off[to[e] + 1];
    ++L->out_off[from[e] + 1];
  }
  for (int32_t v = 0; v < N; ++v) {
    L->in_off[v + 1] += L->in_off[v];
    L->out_off[v + 1] += L->out_off[v];
  }
  L->in_edge.assign(std::max(E, 1), 0);
  L->out_edge.assign(std::max(E, 1), 0);
  std::vector<int32_t> fi(L->in_off.begin(), L->in_off.end() - 1), fo(L->out_off.begin(), L->out_off.end() - 1);
  for (int32_t e = 0; e < E; ++e) {
    L->in_edge[fi[to[e]]++] = e;
    L->out_edge[fo[from[e]]++] = e;
  }
  return FST_OK;
}

template <class T>
int upload(DevMem& mem, T** d, const T* h, int64_t n) {
  int rc = mem.get(d, n);
  if (rc) return rc;
  if (n > 0) FST_CUDA(cudaMemcpy(*d, h, (size_t)n * sizeof(T), cudaMemcpyHostToDevice));
  return FST_OK;
}

}  // namespace

extern "C" int fst_lattice_viterbi(fst_t* f, int32_t num_nodes, int32_t num_edges, const int32_t* from,
                                   const int32_t* to, const int32_t* label, const float* weight, float* best_score,
                                   int32_t* edge_path, int32_t* arc_path, int32_t* path_len) {
  if (!f || !best_score || !path_len || (num_nodes > 1 && (!edge_path || !arc_path))) {
    set_error("fst_lattice_viterbi: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  HostLattice H;
  int rc = check_lattice(f, num_nodes, num_edges, from, to, label, weight, &H);
  if (rc) return rc;
  DevGuard g(f->device);
  cudaStream_t s = 0;
  SliceView sv;
  if ((rc = slice_view(f, s, &sv))) return rc;
  const int64_t Q = f->Q, N = num_nodes, E = num_edges;
  DevMem mem;
  unsigned long long* keys = nullptr;
  int32_t *d_in_off = nullptr, *d_in_edge = nullptr, *d_from = nullptr, *d_label = nullptr, *il = nullptr;
  int32_t *d_epath = nullptr, *d_apath = nullptr, *d_len = nullptr;
  float *d_w = nullptr, *th = nullptr, *d_score = nullptr;
  if ((rc = mem.get(&keys, N * Q)) || (rc = mem.get(&il, std::max<int64_t>(f->A, 1))) ||
      (rc = mem.get(&th, std::max<int64_t>(f->A, 1))) || (rc = mem.get(&d_score, 1)) || (rc = mem.get(&d_len, 1)) ||
      (rc = mem.get(&d_epath, std::max<int64_t>(N - 1, 1))) || (rc = mem.get(&d_apath, std::max<int64_t>(N - 1, 1))) ||
      (rc = upload(mem, &d_in_off, H.in_off.data(), N + 1)) ||
      (rc = upload(mem, &d_in_edge, H.in_edge.data(), std::max<int64_t>(E, 1))) ||
      (rc = upload(mem, &d_from, from, E)) || (rc = upload(mem, &d_label, label, E)) ||
      (rc = upload(mem, &d_w, weight, E)))
    return rc;
  if ((rc = arcs_by_id(f, il, nullptr, th, s))) return rc;
  FST_CUDA(cudaMemsetAsync(keys, 0, (size_t)(N * Q) * 8, s));
  k_lat_vit_init<<<nb(Q), TB, 0, s>>>(f->theta_s, f->Q, keys);
  // node by node: every edge into v, in increasing id
  for (int32_t v = 1; v < N; ++v)
    for (int32_t j = H.in_off[v]; j < H.in_off[v + 1]; ++j) {
      const int32_t e = H.in_edge[j], a = label[e];
      const int64_t i0 = sv.h_sym_win[a] * WIN, np = (sv.h_sym_win[a + 1] - sv.h_sym_win[a]) * WIN;
      if (np)
        k_lat_vit_edge<<<nb(np), TB, 0, s>>>(sv.arcs, sv.theta, i0, np, keys + (int64_t)from[e] * Q, weight[e],
                                             keys + (int64_t)v * Q);
    }
  k_lat_vit_final<<<1, TB, 0, s>>>(keys, num_nodes, f->Q, f->theta_f, d_in_off, d_in_edge, d_from, d_label, d_w, il,
                                   th, f->src_by_id, d_score, d_epath, d_apath, d_len);
  FST_CUDA(cudaGetLastError());
  int32_t len = 0;
  FST_CUDA(cudaMemcpy(best_score, d_score, 4, cudaMemcpyDeviceToHost));
  FST_CUDA(cudaMemcpy(&len, d_len, 4, cudaMemcpyDeviceToHost));
  if (len < 0) {
    set_error("fst_lattice_viterbi: the backtrace found no edge reaching the recorded score");
    return FST_ERR_STATE;
  }
  // the path was recorded from the end node back: reverse it
  std::vector<int32_t> he(std::max(len, 1)), ha(std::max(len, 1));
  if (len > 0) {
    FST_CUDA(cudaMemcpy(he.data(), d_epath, (size_t)len * 4, cudaMemcpyDeviceToHost));
    FST_CUDA(cudaMemcpy(ha.data(), d_apath, (size_t)len * 4, cudaMemcpyDeviceToHost));
  }
  for (int32_t i = 0; i < len; ++i) {
    edge_path[i] = he[len - 1 - i];
    arc_path[i] = ha[len - 1 - i];
  }
  *path_len = len;
  if (*best_score == -INFINITY) {
    set_error("no accepting path");
    return FST_ERR_NO_PATH;
  }
  return FST_OK;
}

extern "C" int fst_lattice_forward_backward(fst_t* f, int32_t num_nodes, int32_t num_edges, const int32_t* from,
                                            const int32_t* to, const int32_t* label, const float* weight,
                                            double* log_z, float* arc_posteriors, float* edge_posteriors) {
  if (!f || !log_z) {
    set_error("fst_lattice_forward_backward: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  HostLattice H;
  int rc = check_lattice(f, num_nodes, num_edges, from, to, label, weight, &H);
  if (rc) return rc;
  DevGuard g(f->device);
  cudaStream_t s = 0;
  SliceView sv;
  if ((rc = slice_view(f, s, &sv))) return rc;
  const int64_t Q = f->Q, N = num_nodes, E = num_edges, A = std::max<int64_t>(f->A, 1);
  DevMem mem;
  double *alpha = nullptr, *beta = nullptr, *d_logz = nullptr, *cnt = nullptr, *epost = nullptr;
  unsigned long long *maxk = nullptr, *sum = nullptr;
  if ((rc = mem.get(&alpha, N * Q)) || (rc = mem.get(&beta, N * Q)) || (rc = mem.get(&d_logz, 1)) ||
      (rc = mem.get(&maxk, Q)) || (rc = mem.get(&sum, Q)) || (rc = mem.get(&cnt, A)) ||
      (rc = mem.get(&epost, std::max<int64_t>(E, 1))))
    return rc;
  FST_CUDA(cudaMemsetAsync(maxk, 0, (size_t)Q * 8, s));
  FST_CUDA(cudaMemsetAsync(sum, 0, (size_t)Q * 8, s));
  FST_CUDA(cudaMemsetAsync(cnt, 0, (size_t)A * 8, s));
  FST_CUDA(cudaMemsetAsync(epost, 0, (size_t)std::max<int64_t>(E, 1) * 8, s));
  auto slice = [&](int32_t a, int64_t* i0, int64_t* np) {
    *i0 = sv.h_sym_win[a] * WIN;
    *np = (sv.h_sym_win[a + 1] - sv.h_sym_win[a]) * WIN;
  };
  // forward, node by node
  k_lat_from_f32<<<nb(Q), TB, 0, s>>>(f->theta_s, f->Q, alpha);
  for (int32_t v = 1; v < N; ++v) {
    for (int ph = 0; ph < 2; ++ph)
      for (int32_t j = H.in_off[v]; j < H.in_off[v + 1]; ++j) {
        const int32_t e = H.in_edge[j];
        int64_t i0, np;
        slice(label[e], &i0, &np);
        if (!np) continue;
        const double* tu = alpha + (int64_t)from[e] * Q;
        if (ph == 0)
          k_lat_lse_edge<true, false><<<nb(np), TB, 0, s>>>(sv.arcs, sv.theta, i0, np, tu, weight[e], maxk, sum);
        else
          k_lat_lse_edge<true, true><<<nb(np), TB, 0, s>>>(sv.arcs, sv.theta, i0, np, tu, weight[e], maxk, sum);
      }
    k_lat_lse_finish<<<nb(Q), TB, 0, s>>>(maxk, sum, f->Q, alpha + (int64_t)v * Q);
  }
  k_lat_logz<<<1, TB, 0, s>>>(alpha + (N - 1) * Q, f->theta_f, f->Q, d_logz);
  // backward, from the end node
  k_lat_from_f32<<<nb(Q), TB, 0, s>>>(f->theta_f, f->Q, beta + (N - 1) * Q);
  for (int32_t v = (int32_t)N - 2; v >= 0; --v) {
    for (int ph = 0; ph < 2; ++ph)
      for (int32_t j = H.out_off[v]; j < H.out_off[v + 1]; ++j) {
        const int32_t e = H.out_edge[j];
        int64_t i0, np;
        slice(label[e], &i0, &np);
        if (!np) continue;
        const double* tv = beta + (int64_t)to[e] * Q;
        if (ph == 0)
          k_lat_lse_edge<false, false><<<nb(np), TB, 0, s>>>(sv.arcs, sv.theta, i0, np, tv, weight[e], maxk, sum);
        else
          k_lat_lse_edge<false, true><<<nb(np), TB, 0, s>>>(sv.arcs, sv.theta, i0, np, tv, weight[e], maxk, sum);
      }
    k_lat_lse_finish<<<nb(Q), TB, 0, s>>>(maxk, sum, f->Q, beta + (int64_t)v * Q);
  }
  // posteriors
  for (int32_t e = 0; e < num_edges; ++e) {
    int64_t i0, np;
    slice(label[e], &i0, &np);
    if (np)
      k_lat_post<<<nb(np), TB, 0, s>>>(sv.arcs, sv.theta, i0, np, alpha + (int64_t)from[e] * Q,
                                       beta + (int64_t)to[e] * Q, weight[e], d_logz, cnt, epost + e);
  }
  FST_CUDA(cudaGetLastError());
  FST_CUDA(cudaMemcpy(log_z, d_logz, 8, cudaMemcpyDeviceToHost));
  if (arc_posteriors && f->A > 0) {
    float* tmp = nullptr;
    if ((rc = mem.get(&tmp, f->A))) return rc;
    k_lat_to_f32<<<nb(f->A), TB, 0, s>>>(cnt, f->A, tmp);
    FST_CUDA(cudaMemcpy(arc_posteriors, tmp, (size_t)f->A * 4, cudaMemcpyDeviceToHost));
  }
  if (edge_posteriors && E > 0) {
    float* tmp = nullptr;
    if ((rc = mem.get(&tmp, E))) return rc;
    k_lat_to_f32<<<nb(E), TB, 0, s>>>(epost, E, tmp);
    FST_CUDA(cudaMemcpy(edge_posteriors, tmp, (size_t)E * 4, cudaMemcpyDeviceToHost));
  }
  if (*log_z == -INFINITY) {
    set_error("no accepting path");
    return FST_ERR_NO_PATH;
  }
  return FST_OK;
}
