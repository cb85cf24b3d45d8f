// sort_scan.cu -- device primitives used when an FST or a plan is built:
// exclusive prefix sums and a stable LSD radix sort of (u64 key, u32 value)
// pairs.  They sort the arcs into the symbol-major slices of Sec. 4 / Fig. 2
// (the R offsets are a prefix sum of the per-symbol arc counts).  Written
// for this library; no external sort or scan library.
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fst_internal.cuh"

namespace fstgpu {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ __forceinline__ T warp_incl_sum(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x += o;
  }
  return x;
}

// Exclusive scan of a thread's SCAN_ITEMS values across the block; returns
// the block total.  Values are in blocked order (thread t owns items
// t*SCAN_ITEMS .. t*SCAN_ITEMS+SCAN_ITEMS-1).
template <class T>
__device__ T block_exclusive(T (&v)[SCAN_ITEMS]) {
  __shared__ T wsum[SCAN_THREADS / 32];
  T local = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    T x = v[i];
    v[i] = local;
    local += x;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = warp_incl_sum(local);
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  T woff = 0, total = 0;
#pragma unroll
  for (int w = 0; w < SCAN_THREADS / 32; ++w) {
    if (w < warp) woff += wsum[w];
    total += wsum[w];
  }
  const T excl = woff + incl - local;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) v[i] += excl;
  __syncthreads();
  return total;
}

template <class T>
__global__ void scan_partials(const T* __restrict__ in, int64_t n, T* __restrict__ part) {
  T v[SCAN_ITEMS];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) v[i] = (base + i < n) ? in[base + i] : T(0);
  T tot = block_exclusive(v);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <class T>
__global__ void scan_apply(const T* in, int64_t n, const T* __restrict__ part_excl, T* out) {
  T v[SCAN_ITEMS];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) v[i] = (base + i < n) ? in[base + i] : T(0);
  block_exclusive(v);
  const T off = part_excl ? part_excl[blockIdx.x] : T(0);
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i)
    if (base + i < n) out[base + i] = v[i] + off;
}

template <class T>
int scan_impl(const T* in, T* out, int64_t n, T* total_dev, cudaStream_t s) {
  if (n <= 0) {
    if (total_dev) FST_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(T), s));
    return FST_OK;
  }
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  T* part = nullptr;
  int rc = dalloc(&part, nb + 1);
  if (rc) return rc;
  scan_partials<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, part);
  if (nb > 1) {
    // part[nb] receives the grand total
    rc = scan_impl<T>(part, part, nb, part + nb, s);
    if (rc) { dfree(part); return rc; }
    scan_apply<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, part, out);
    if (total_dev) FST_CUDA(cudaMemcpyAsync(total_dev, part + nb, sizeof(T), cudaMemcpyDeviceToDevice, s));
  } else {
    if (total_dev) FST_CUDA(cudaMemcpyAsync(total_dev, part, sizeof(T), cudaMemcpyDeviceToDevice, s));
    scan_apply<T><<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out);
  }
  cudaError_t e = cudaGetLastError();
  // the scan kernels are stream-ordered; free after the stream drains
  cudaError_t e2 = cudaStreamSynchronize(s);
  dfree(part);
  if (e != cudaSuccess) return cuda_fail(e, "scan kernels");
  if (e2 != cudaSuccess) return cuda_fail(e2, "scan sync");
  return FST_OK;
}

// ------------------------------------------------------------ radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_BINS = 256;

__global__ void rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                        uint32_t* __restrict__ hist, int64_t ntiles) {
  __shared__ uint32_t h[RS_BINS];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: elements of a tile are visited in index order (round by
// round, lane by lane); each element's rank among equal digits comes from
// __match_any_sync within the warp plus per-warp counts of earlier warps.
__global__ void rs_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                           int64_t n, int shift, const uint32_t* __restrict__ offs, int64_t ntiles,
                           uint64_t* __restrict__ kout, uint32_t* __restrict__ vout) {
  __shared__ uint32_t s_base[RS_BINS];
  __shared__ uint32_t s_wcnt[RS_THREADS / 32][RS_BINS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  s_base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
#pragma unroll
  for (int w = 0; w < RS_THREADS / 32; ++w) s_wcnt[w][tid] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const uint32_t lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t i = base + r * RS_THREADS + tid;
    const bool valid = i < n;
    uint64_t k = 0;
    uint32_t v = 0, d = RS_BINS;  // invalid lanes form their own group
    if (valid) {
      k = kin[i];
      v = vin[i];
      d = (uint32_t)(k >> shift) & 255u;
    }
    const uint32_t peers = __match_any_sync(FULL, d);
    const uint32_t rank = __popc(peers & lt);
    if (valid && rank == 0) s_wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pos = s_base[d] + rank;
      for (int w = 0; w < warp; ++w) pos += s_wcnt[w][d];
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
    uint32_t add = 0;
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) {
      add += s_wcnt[w][tid];
      s_wcnt[w][tid] = 0;
    }
    s_base[tid] += add;
    __syncthreads();
  }
}

}  // namespace

int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, cudaStream_t s) {
  int64_t* tot = nullptr;
  int rc = dalloc(&tot, 1);
  if (rc) return rc;
  rc = scan_impl<long long>((const long long*)in, (long long*)out, n, (long long*)tot, s);
  if (!rc && total) {
    cudaError_t e = cudaMemcpy(total, tot, sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "scan total");
  }
  dfree(tot);
  return rc;
}

int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
  return scan_impl<unsigned int>((const unsigned int*)in, (unsigned int*)out, n, nullptr, s);
}

int radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return FST_OK;
  if (n >= (int64_t)1 << 32) {
    set_error("radix sort of %lld elements is beyond 2^32", (long long)n);
    return FST_ERR_UNSUPPORTED;
  }
  const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  uint64_t* k2 = nullptr;
  uint32_t* v2 = nullptr;
  uint32_t* hist = nullptr;
  int rc = dalloc(&k2, n);
  if (!rc) rc = dalloc(&v2, n);
  if (!rc) rc = dalloc(&hist, ntiles * RS_BINS);
  if (rc) { dfree(k2); dfree(v2); dfree(hist); return rc; }
  uint64_t *ka = keys, *kb = k2;
  uint32_t *va = vals, *vb = v2;
  const int passes = (bits + 7) / 8;
  for (int p = 0; p < passes && !rc; ++p) {
    const int shift = 8 * p;
    rs_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, n, shift, hist, ntiles);
    rc = exclusive_scan_u32(hist, hist, ntiles * RS_BINS, s);
    if (rc) break;
    rs_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, va, n, shift, hist, ntiles, kb, vb);
    uint64_t* tk = ka; ka = kb; kb = tk;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  if (!rc && ka != keys) {
    cudaError_t e = cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vals, va, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "radix sort copy-back");
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "radix sort");
  dfree(k2); dfree(v2); dfree(hist);
  return rc;
}

}  // namespace fstgpu
