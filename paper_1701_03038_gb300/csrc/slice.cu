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
__global__ void k_slice_fill(const int32_t* __restrict__ seg_state, const int32_t* __restrict__ seg_pos,
                             const int32_t* __restrict__ seg_len, const int32_t* __restrict__ other,
                             const int32_t* __restrict__ arc_id, int64_t nseg, int4* __restrict__ arcs) {
  const int64_t sg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sg >= nseg) return;
  const int32_t d = seg_state[sg], p0 = seg_pos[sg];
  for (int32_t i = 0; i < seg_len[sg]; ++i) arcs[p0 + i] = make_int4(other[p0 + i], d, arc_id[p0 + i], 0);
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

}  // namespace

extern "C" int fst_viterbi_slice(fst_t* f, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path) {
  if (!f || n < 0 || (n > 0 && (!ids || !arc_path)) || !best_score) {
    set_error("fst_viterbi_slice: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  for (int32_t i = 0; i < n; ++i)
    if (ids[i] < 0 || ids[i] >= f->m) {
      set_error("symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
      return FST_ERR_INVALID_ARG;
    }
  const Layout& L = f->fwd;
  const int64_t Q = f->Q;
  int rc;
  cudaStream_t s = 0;
  if (!f->slice_arcs) {  // the slice records, built on first use
    if ((rc = dalloc(&f->slice_arcs, L.P))) return rc;
    if (L.P > 0) k_slice_pad<<<(unsigned)((L.P + TB - 1) / TB), TB, 0, s>>>(f->slice_arcs, L.P);
    if (L.nseg > 0)
      k_slice_fill<<<(unsigned)((L.nseg + TB - 1) / TB), TB, 0, s>>>(L.seg_state, L.seg_pos, L.seg_len, L.other,
                                                                     L.arc_id, L.nseg, f->slice_arcs);
    FST_CUDA(cudaGetLastError());
  }
  const int64_t need = (int64_t)(n + 1) * Q;
  if (need > f->slice_cap) {
    dfree(f->slice_keys);
    f->slice_cap = 0;
    if ((rc = dalloc(&f->slice_keys, need))) return rc;
    f->slice_cap = need;
  }
  float* d_score = nullptr;
  int32_t* d_path = nullptr;
  if ((rc = dalloc(&d_score, 1)) || (rc = dalloc(&d_path, std::max(n, 1)))) {
    dfree(d_score);
    return rc;
  }
  FST_CUDA(cudaMemsetAsync(f->slice_keys, 0, (size_t)need * 8, s));
  for (int32_t t = 1; t <= n; ++t) {
    const int32_t a = ids[t - 1];
    const int64_t i0 = L.h_sym_win[a] * WIN, np = (L.h_sym_win[a + 1] - L.h_sym_win[a]) * WIN;
    if (np == 0) continue;
    k_slice_relax<<<(unsigned)((np + TB - 1) / TB), TB, 0, s>>>(
        f->slice_arcs, L.theta, i0, np, t == 1 ? nullptr : f->slice_keys + (int64_t)(t - 1) * Q, f->theta_s,
        f->slice_keys + (int64_t)t * Q);
  }
  k_slice_final<<<1, TB, 0, s>>>(f->slice_keys, n, f->Q, f->theta_s, f->theta_f, f->src_by_id, d_score, d_path);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(best_score, d_score, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(arc_path, d_path, (size_t)n * 4, cudaMemcpyDeviceToHost);
  dfree(d_score);
  dfree(d_path);
  if (e != cudaSuccess) return cuda_fail(e, "fst_viterbi_slice");
  if (*best_score == -INFINITY) {
    set_error("no accepting path");
    return FST_ERR_NO_PATH;
  }
  return FST_OK;
}
