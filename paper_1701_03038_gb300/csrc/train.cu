// train.cu -- what training needs beyond the expected counts.
//
// The expected counts of Alg. 2 serve training by expectation-maximisation
// (Sec. 4).  fst_em_update is the M-step: every state's outgoing arcs form
// one categorical distribution, re-estimated from the counts.  A
// conditional (CRF-style) likelihood also needs the numerator log Z(x, y),
// the weight of the paths that read x AND write y; fst_create_clamped builds
// the FST in which arc k reads the pair (ilabel_k, olabel_k), so that log
// Z(x, y) is the ordinary forward pass over the string of pairs, with the
// same arc ids, weights and kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fst_internal.cuh"

using namespace fstgpu;

namespace {

constexpr int TB = 256;
inline unsigned nblk(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + TB - 1) / TB); }

// Symbol, destination and log-weight of every arc by caller id, read back
// from the source-segmented layout: position i lies in the windows of the
// symbol a with sym_win[a] <= i / WIN < sym_win[a + 1]; padding has id -1.
__global__ void k_by_id(const int32_t* __restrict__ arc_id, const int32_t* __restrict__ other,
                        const float* __restrict__ theta, const int64_t* __restrict__ sym_win, int32_t m, int64_t P,
                        int32_t* __restrict__ il_out, int32_t* __restrict__ dst_out, float* __restrict__ th_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const int32_t id = arc_id[i];
  if (id < 0) return;
  const int64_t w = i / WIN;
  int32_t lo = 0, hi = m;  // last a with sym_win[a] <= w
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (sym_win[mid] <= w) lo = mid; else hi = mid;
  }
  if (il_out) il_out[id] = lo;
  if (dst_out) dst_out[id] = other[i];
  if (th_out) th_out[id] = theta[i];
}

// M-step: total[q] = sum over the arcs out of q of (count + alpha) ...
__global__ void k_em_totals(const float* __restrict__ counts, const int32_t* __restrict__ src, int64_t A,
                            double alpha, double* __restrict__ total, unsigned int* __restrict__ err) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= A) return;
  const float c = counts[k];
  if (!(c >= 0.f) || isinf(c)) {  // negative, NaN or infinite count
    atomicOr(err, 1u);
    return;
  }
  atomicAdd(total + src[k], (double)c + alpha);
}

// ... and theta'_k = log((count_k + alpha) / total[src_k]); a state with a
// zero total keeps its arcs' old log-weights.
__global__ void k_em_theta(const float* __restrict__ counts, const int32_t* __restrict__ src,
                           const float* __restrict__ theta_old, const double* __restrict__ total, int64_t A,
                           double alpha, float* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= A) return;
  const double t = total[src[k]];
  out[k] = t > 0.0 ? (float)log(((double)counts[k] + alpha) / t) : theta_old[k];
}

// (input label, output label) key of every arc, with its id, for the sort.
__global__ void k_pair_keys(const int32_t* __restrict__ il, const int32_t* __restrict__ ol, int64_t A,
                            uint64_t* __restrict__ keys, uint32_t* __restrict__ ids) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= A) return;
  keys[k] = ((uint64_t)(uint32_t)il[k] << 32) | (uint64_t)(uint32_t)ol[k];
  ids[k] = (uint32_t)k;
}

__global__ void k_pair_heads(const uint64_t* __restrict__ keys, int64_t A, int64_t* __restrict__ head) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A) head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// pair id of every arc (by id) and the distinct keys in pair order.
__global__ void k_pair_ids(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ids,
                           const int64_t* __restrict__ head, const int64_t* __restrict__ excl, int64_t A,
                           int32_t* __restrict__ pair_by_id, uint64_t* __restrict__ ukeys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A) return;
  const int64_t pid = excl[i] + head[i] - 1;
  pair_by_id[ids[i]] = (int32_t)pid;
  if (head[i]) ukeys[pid] = keys[i];
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

}  // namespace

namespace fstgpu {
int arcs_by_id(fst_s* f, int32_t* il, int32_t* dst, float* th, cudaStream_t s) {
  const Layout& L = f->bwd;
  if (L.P > 0)
    k_by_id<<<nblk(L.P), TB, 0, s>>>(L.arc_id, L.other, L.theta, L.sym_win, f->m, L.P, il, dst, th);
  FST_CUDA(cudaGetLastError());
  return FST_OK;
}
}  // namespace fstgpu

extern "C" int fst_em_update(fst_t* f, const float* counts, float pseudo_count, float* theta_out, int32_t flags) {
  if (!f || (f->A > 0 && (!counts || !theta_out)) || !(pseudo_count >= 0.f) || isinf(pseudo_count) ||
      (flags & ~(FST_FLAG_DEVICE_PTRS | FST_EM_APPLY))) {
    set_error("fst_em_update: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  DevGuard g(f->device);
  const int64_t A = f->A;
  if (A == 0) return FST_OK;
  const bool dev = (flags & FST_FLAG_DEVICE_PTRS) != 0;
  cudaStream_t s = 0;
  DevMem mem;
  float *d_counts = nullptr, *d_out = nullptr, *d_old = nullptr;
  double* total = nullptr;
  unsigned int* err = nullptr;
  int rc;
  if ((rc = mem.get(&d_old, A)) || (rc = mem.get(&total, f->Q)) || (rc = mem.get(&err, 1))) return rc;
  if (dev) {
    d_counts = (float*)counts;
    d_out = theta_out;
  } else {
    if ((rc = mem.get(&d_counts, A)) || (rc = mem.get(&d_out, A))) return rc;
    FST_CUDA(cudaMemcpy(d_counts, counts, (size_t)A * 4, cudaMemcpyHostToDevice));
  }
  FST_CUDA(cudaMemsetAsync(total, 0, (size_t)f->Q * 8, s));
  FST_CUDA(cudaMemsetAsync(err, 0, 4, s));
  if ((rc = arcs_by_id(f, nullptr, nullptr, d_old, s))) return rc;
  k_em_totals<<<nblk(A), TB, 0, s>>>(d_counts, f->src_by_id, A, (double)pseudo_count, total, err);
  FST_CUDA(cudaGetLastError());
  unsigned int h_err = 0;
  FST_CUDA(cudaMemcpy(&h_err, err, 4, cudaMemcpyDeviceToHost));
  if (h_err) {
    set_error("fst_em_update: a count is negative, NaN or infinite");
    return FST_ERR_INVALID_ARG;
  }
  k_em_theta<<<nblk(A), TB, 0, s>>>(d_counts, f->src_by_id, d_old, total, A, (double)pseudo_count, d_out);
  FST_CUDA(cudaGetLastError());
  if (flags & FST_EM_APPLY) {
    if ((rc = set_layout_weights(f, d_out, s))) return rc;
  }
  if (!dev) FST_CUDA(cudaMemcpy(theta_out, d_out, (size_t)A * 4, cudaMemcpyDeviceToHost));
  FST_CUDA(cudaStreamSynchronize(s));
  return FST_OK;
}

extern "C" int fst_create_clamped(const fst_t* fc, fst_t** out, int32_t* num_pairs) {
  if (!out) { set_error("out is NULL"); return FST_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!fc) { set_error("fst is NULL"); return FST_ERR_INVALID_ARG; }
  fst_s* f = const_cast<fst_s*>(fc);
  DevGuard g(f->device);
  const int64_t A = f->A;
  cudaStream_t s = 0;
  DevMem mem;
  int32_t *il = nullptr, *dst = nullptr, *pair = nullptr;
  float* th = nullptr;
  uint64_t *keys = nullptr, *ukeys = nullptr;
  uint32_t* ids = nullptr;
  int64_t *head = nullptr, *excl = nullptr;
  int rc;
  const int64_t n = std::max<int64_t>(A, 1);
  if ((rc = mem.get(&il, n)) || (rc = mem.get(&dst, n)) || (rc = mem.get(&th, n)) || (rc = mem.get(&pair, n)) ||
      (rc = mem.get(&keys, n)) || (rc = mem.get(&ids, n)) || (rc = mem.get(&head, n)) || (rc = mem.get(&excl, n)) ||
      (rc = mem.get(&ukeys, n)))
    return rc;
  if ((rc = arcs_by_id(f, il, dst, th, s))) return rc;
  int64_t npairs = 0;
  if (A > 0) {
    k_pair_keys<<<nblk(A), TB, 0, s>>>(il, f->olabel, A, keys, ids);
    FST_CUDA(cudaGetLastError());
    if ((rc = radix_sort_pairs(keys, ids, A, 64, s))) return rc;
    k_pair_heads<<<nblk(A), TB, 0, s>>>(keys, A, head);
    FST_CUDA(cudaGetLastError());
    if ((rc = exclusive_scan_i64(head, excl, A, &npairs, s))) return rc;
    k_pair_ids<<<nblk(A), TB, 0, s>>>(keys, ids, head, excl, A, pair, ukeys);
    FST_CUDA(cudaGetLastError());
  }
  if (npairs >= INT32_MAX) { set_error("too many label pairs"); return FST_ERR_UNSUPPORTED; }
  std::vector<uint64_t> h_keys((size_t)std::max<int64_t>(npairs, 1));
  if (npairs > 0) FST_CUDA(cudaMemcpy(h_keys.data(), ukeys, (size_t)npairs * 8, cudaMemcpyDeviceToHost));
  FST_CUDA(cudaStreamSynchronize(s));
  // the pairs are the input symbols; one more symbol, without arcs, stands
  // for every pair that no arc carries
  fst_t* c = nullptr;
  rc = fst_create(f->Q, A, f->src_by_id, dst, pair, f->olabel, th, FST_WEIGHT_LOG, f->theta_s, f->theta_f,
                  (int32_t)npairs + 1, FST_FLAG_DEVICE_PTRS, &c);
  if (rc) return rc;
  c->pair_keys = new std::vector<uint64_t>(h_keys.begin(), h_keys.begin() + npairs);
  *out = c;
  if (num_pairs) *num_pairs = (int32_t)npairs;
  return FST_OK;
}

extern "C" int fst_clamp_labels(const fst_t* c, const int32_t* ids, const int32_t* olabels, int64_t n,
                                int32_t* pair_ids) {
  if (!c || n < 0 || (n > 0 && (!ids || !olabels || !pair_ids))) {
    set_error("fst_clamp_labels: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  if (!c->pair_keys) { set_error("fst_clamp_labels: the FST was not made by fst_create_clamped"); return FST_ERR_STATE; }
  const std::vector<uint64_t>& K = *c->pair_keys;
  const int32_t absent = (int32_t)K.size();
  for (int64_t t = 0; t < n; ++t) {
    const uint64_t key = ((uint64_t)(uint32_t)ids[t] << 32) | (uint64_t)(uint32_t)olabels[t];
    auto it = std::lower_bound(K.begin(), K.end(), key);
    pair_ids[t] = (it != K.end() && *it == key) ? (int32_t)(it - K.begin()) : absent;
  }
  return FST_OK;
}
