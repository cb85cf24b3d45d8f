// fd64.cu -- log Z of one string in float64 on the GPU (plain method).
//
// The forward recursion of Alg. 2 in the log domain, every value and every
// arc weight in float64.  It exists for finite-difference checks of the
// float32 gradient (d log Z / d theta = expected arc counts): a central
// difference with h = 1e-6 needs log Z to ~1e-12, which float32 cannot give.
// One launch per position over the windows of the symbol's slice; segments
// are reduced with a max-shifted (max, sum) pair scan as in the float32
// kernels.  The dense frontier is refilled with -inf before each position.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "fst_internal.cuh"
#include "kernels.cuh"

using namespace fstgpu;

namespace {

constexpr int TB = 256;

__device__ __forceinline__ double2 lse64_combine(double2 a, double2 b) {
  if (a.x < b.x) { double2 c = a; a = b; b = c; }
  if (b.x == -INFINITY) return a;
  return make_double2(a.x, a.y + b.y * exp(b.x - a.x));
}

__device__ __forceinline__ double2 shfl_up2(double2 v, int d) {
  return make_double2(__shfl_up_sync(FULL, v.x, d), __shfl_up_sync(FULL, v.y, d));
}

__global__ void k_fill64(double* p, int64_t n, double v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// One position: out[q'] = LSE_{arcs of the slice into q'} (in[src] + theta64).
// Segments longer than a window are combined with an ordered serial pass by
// the lane that owns the segment's last window (long segments are rare in
// the small FSTs this serves; correctness over speed).
__global__ void k_fwd64_step(const int32_t* __restrict__ other, const double* __restrict__ theta64,
                             const WinMeta* __restrict__ win, const int32_t* __restrict__ seg_state,
                             const int32_t* __restrict__ seg_pos, int64_t w0, int64_t nwin,
                             const double* __restrict__ in, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (item >= nwin) return;
  const int64_t w = w0 + item;
  const WinMeta m = win[w];
  if (m.lseg >= 0) {
    // long segment: the warp of its first window sums every window in order
    const int64_t first = seg_pos[m.seg] / WIN;
    if (w != first) return;
    double2 acc = make_double2(-INFINITY, 0.0);
    for (int64_t j = 0; j < (int64_t)m.lcnt * WIN; j += 32) {
      const int64_t pos = first * WIN + j + lane;
      const double v = in[other[pos]] + theta64[pos];
      double2 e = (v == -INFINITY) ? make_double2(-INFINITY, 0.0) : make_double2(v, 1.0);
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) {
        double2 o = make_double2(__shfl_xor_sync(FULL, e.x, d), __shfl_xor_sync(FULL, e.y, d));
        e = (lane & d) ? lse64_combine(o, e) : lse64_combine(e, o);
      }
      acc = lse64_combine(acc, e);
    }
    if (lane == 0) out[seg_state[m.seg]] = acc.x == -INFINITY ? -INFINITY : acc.x + log(acc.y);
    return;
  }
  const uint32_t word = (lane >> 3) == 0 ? m.mask[0] : (lane >> 3) == 1 ? m.mask[1] : (lane >> 3) == 2 ? m.mask[2] : m.mask[3];
  const int sh = (lane & 7) * 4;
  const uint32_t h = (word >> sh) & 0xFu;
  int hb = __popc(word & ((1u << sh) - 1u));
  for (int k = 0; k < 3; ++k)
    if (k < (lane >> 3)) hb += __popc(m.mask[k]);
  double2 p[APL];
  for (int k = 0; k < APL; ++k) {
    const int64_t pos = w * WIN + lane * APL + k;
    const double v = in[other[pos]] + theta64[pos];
    const double2 e = (v == -INFINITY) ? make_double2(-INFINITY, 0.0) : make_double2(v, 1.0);
    p[k] = (k == 0 || ((h >> k) & 1u)) ? e : lse64_combine(p[k - 1], e);
  }
  // segmented scan over lanes of each lane's last partial segment
  const uint32_t hm = __ballot_sync(FULL, h != 0u);
  const uint32_t le = hm & (0xffffffffu >> (31 - lane));
  const int start = le ? 31 - __clz(le) : 0;
  double2 agg = p[APL - 1];
  for (int d = 1; d < 32; d <<= 1) {
    const double2 o = shfl_up2(agg, d);
    if (lane - d >= start) agg = lse64_combine(o, agg);
  }
  double2 carry = shfl_up2(agg, 1);
  if (lane == 0) carry = make_double2(-INFINITY, 0.0);
  const int firsth = h ? __ffs(h) - 1 : APL;
  const uint32_t hn = __shfl_down_sync(FULL, h, 1);
  int cum = hb;
  for (int k = 0; k < APL; ++k) {
    cum += (h >> k) & 1u;
    const double2 full = (k < firsth) ? lse64_combine(carry, p[k]) : p[k];
    const bool tail = (k < APL - 1) ? ((h >> (k + 1)) & 1u) : (lane == 31 || (hn & 1u));
    if (tail) {
      const int32_t s = m.seg + cum - 1;
      out[seg_state[s]] = full.x == -INFINITY ? -INFINITY : full.x + log(full.y);
    }
  }
}

// log Z = LSE_q (alpha_n[q] + final[q]) in one block.
__global__ void k_logz64(const double* __restrict__ a, const float* __restrict__ fin, int32_t Q, double* out) {
  __shared__ double red[TB];
  double mx = -INFINITY;
  for (int32_t q = threadIdx.x; q < Q; q += blockDim.x) mx = fmax(mx, a[q] + (double)fin[q]);
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int d = TB / 2; d >= 1; d >>= 1) {
    if ((int)threadIdx.x < d) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + d]);
    __syncthreads();
  }
  mx = red[0];
  __syncthreads();
  double sm = 0.0;
  if (mx != -INFINITY)
    for (int32_t q = threadIdx.x; q < Q; q += blockDim.x) {
      const double v = a[q] + (double)fin[q];
      if (v != -INFINITY) sm += exp(v - mx);
    }
  red[threadIdx.x] = sm;
  __syncthreads();
  for (int d = TB / 2; d >= 1; d >>= 1) {
    if ((int)threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (mx == -INFINITY) ? -INFINITY : mx + log(red[0]);
}

__global__ void k_start64(const float* __restrict__ ts, int32_t Q, double* out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < Q) out[q] = (double)ts[q];
}

}  // namespace

extern "C" int fst_log_z_f64(fst_t* f, const double* theta, const int32_t* ids, int32_t n, double* log_z) {
  if (!f || n < 0 || (n > 0 && !ids) || !log_z) {
    set_error("fst_log_z_f64: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  for (int32_t i = 0; i < n; ++i)
    if (ids[i] < 0 || ids[i] >= f->m) {
      set_error("fst_log_z_f64: symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
      return FST_ERR_INVALID_ARG;
    }
  int rc;
  cudaStream_t s = 0;
  if (theta) {
    double* d_th = nullptr;
    if ((rc = dalloc(&d_th, f->A))) return rc;
    cudaError_t e = cudaMemcpy(d_th, theta, (size_t)std::max<int64_t>(f->A, 1) * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) rc = set_layout_weights64(f, d_th, s);
    else rc = cuda_fail(e, "fst_log_z_f64 copy");
    cudaError_t e2 = cudaDeviceSynchronize();
    dfree(d_th);
    if (rc) return rc;
    if (e2 != cudaSuccess) return cuda_fail(e2, "fst_log_z_f64 weights");
  } else if (!f->fwd.theta64) {
    set_error("fst_log_z_f64: no float64 weights set yet (pass theta)");
    return FST_ERR_STATE;
  }
  const int64_t Q = f->Q;
  double *a0 = nullptr, *a1 = nullptr, *d_lz = nullptr;
  if ((rc = dalloc(&a0, Q)) || (rc = dalloc(&a1, Q)) || (rc = dalloc(&d_lz, 1))) {
    dfree(a0); dfree(a1); dfree(d_lz);
    return rc;
  }
  const unsigned qb = (unsigned)((Q + TB - 1) / TB);
  k_start64<<<qb, TB, 0, s>>>(f->theta_s, f->Q, a0);
  for (int32_t t = 1; t <= n; ++t) {
    const int32_t a = ids[t - 1];
    const int64_t w0 = f->fwd.h_sym_win[a], nw = f->fwd.h_sym_win[a + 1] - w0;
    k_fill64<<<qb, TB, 0, s>>>(a1, Q, -INFINITY);
    if (nw > 0)
      k_fwd64_step<<<(unsigned)((nw * 32 + TB - 1) / TB), TB, 0, s>>>(f->fwd.other, f->fwd.theta64, f->fwd.win,
                                                                      f->fwd.seg_state, f->fwd.seg_pos, w0, nw, a0, a1);
    std::swap(a0, a1);
  }
  k_logz64<<<1, TB, 0, s>>>(a0, f->theta_f, f->Q, d_lz);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(log_z, d_lz, 8, cudaMemcpyDeviceToHost);
  dfree(a0); dfree(a1); dfree(d_lz);
  if (e != cudaSuccess) return cuda_fail(e, "fst_log_z_f64");
  return FST_OK;
}
