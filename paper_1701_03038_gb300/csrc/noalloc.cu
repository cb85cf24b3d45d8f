// noalloc.cu -- fst_viterbi_noalloc: the plain Viterbi decode of one string
// (Alg. 1, Sec. 5.1, with the frontier-driven steps of the other
// single-string calls) with every piece of per-call working memory taken
// from one fixed, file-scope device array instead of cudaMalloc.  The paper
// has no counterpart: this is a deployment variant.
//
// Some callers cannot allocate device memory at decode time: a host
// application whose memory manager owns every allocation, code that must not
// take the implicit device synchronisation of cudaMalloc/cudaFree inside a
// latency-critical loop, or a process running under a hard device-memory
// cap.  For them this entry point uses only the FST (built earlier by
// fst_create), the caller's output buffers and the array below.
//
// The array is NOALLOC_SCRATCH_BYTES (32 MiB) per device and stays resident
// for as long as the library is loaded.  Its device address is looked up
// once per device, with that device current, by the first call on it: make
// that first call before any stream capture.  All calls share the array and
// it keeps the previous call's contents, so each call first clears the parts
// that must start at zero; calls that overlap on the GPU (two host threads,
// or two streams, at once) race on it and must be serialised by the caller.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "fst_internal.cuh"
#include "kernels.cuh"

using namespace fstgpu;

#define NOALLOC_SCRATCH_BYTES (32ull << 20)
#define NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_setup_mutex;
void* g_scratch_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device; host code must not use the symbol itself as an address).
int scratch_address(void** out) {
  int dev = 0;
  FST_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    set_error("fst_viterbi_noalloc: device %d is beyond the %d devices it supports", dev, NOALLOC_MAX_DEVICES);
    return FST_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FST_OK;
}

// Carves 256-byte aligned pieces out of the scratch array.
struct Carver {
  unsigned char* base;
  size_t used = 0;
  template <class T>
  T* take(int64_t n) {
    const size_t bytes = ((size_t)(n > 0 ? n : 1) * sizeof(T) + 255) & ~(size_t)255;
    T* p = (T*)(base + used);
    used += bytes;
    return p;
  }
};

// The step list is the identity (token t-1 is the only slot of position t).
__global__ void k_noalloc_iota(int32_t* __restrict__ iota, int32_t n) {
  const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i < n) iota[i] = i;
}

}  // namespace

extern "C" int fst_viterbi_noalloc(fst_t* f, const int32_t* ids, int32_t n, float* d_score, int32_t* d_path,
                                   int32_t* d_olabels, void* stream) {
  if (!f || n < 0 || (n > 0 && (!ids || !d_path)) || !d_score) {
    set_error("fst_viterbi_noalloc: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  // the FST's memory, the scratch array's address and the caller's stream
  // all belong to the FST's device: a call made while another device is
  // current is refused before anything is launched or looked up
  int cur = -1;
  FST_CUDA(cudaGetDevice(&cur));
  if (cur != f->device) {
    set_error("fst_viterbi_noalloc: device %d is current but the FST lives on device %d (make it current and "
              "pass a stream of that device)", cur, f->device);
    return FST_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // sizes first, from host data only
  int64_t pool = 0, dmax = 1;
  for (int32_t i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= f->m) {
      set_error("fst_viterbi_noalloc: symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
      return FST_ERR_INVALID_ARG;
    }
    const int64_t D = f->fwd.h_sym_seg[ids[i] + 1] - f->fwd.h_sym_seg[ids[i]];
    pool += D;
    dmax = std::max(dmax, D);
  }
  const int64_t Q = f->Q, nn = std::max(n, 1);
  auto rnd = [](int64_t bytes) { return ((bytes > 0 ? bytes : 1) + 255) & ~(int64_t)255; };
  const int64_t need = rnd(2 * Q * 8) + rnd(2 * Q * 4) + 5 * rnd(nn * 4) + 3 * rnd(nn * 8) + 2 * rnd(dmax * 4) +
                       4 * rnd(pool * 4) + rnd(2 * (nn + 2) * 8) + 6 * rnd(8);
  if (need > (int64_t)NOALLOC_SCRATCH_BYTES) {
    set_error("fst_viterbi_noalloc: this string needs %lld bytes of working memory, beyond the fixed %llu bytes "
              "(shorter strings or fewer states fit; fst_viterbi has no such limit)",
              (long long)need, (unsigned long long)NOALLOC_SCRATCH_BYTES);
    return FST_ERR_UNSUPPORTED;
  }
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  Carver c{(unsigned char*)base};
  unsigned long long* acc = c.take<unsigned long long>(2 * Q);
  int32_t* vmap = c.take<int32_t>(2 * Q);
  int32_t* tok_sym = c.take<int32_t>(nn);
  int32_t* tok_b = c.take<int32_t>(nn);
  int32_t* iota = c.take<int32_t>(nn);
  int64_t* slot_base = c.take<int64_t>(nn);
  int64_t* step_rng = c.take<int64_t>(2 * (nn + 2));
  uint32_t* scnt = c.take<uint32_t>(nn);
  int32_t* pool_cnt = c.take<int32_t>(nn);
  int64_t* zero64 = c.take<int64_t>(nn);
  int64_t* pool_base = c.take<int64_t>(nn);
  int32_t* stage = c.take<int32_t>(dmax);
  int32_t* stage_b = c.take<int32_t>(dmax);
  int32_t* pool_q = c.take<int32_t>(pool);
  int32_t* pool_x = c.take<int32_t>(pool);
  float* pool_v = c.take<float>(pool);
  int32_t* pool_n = c.take<int32_t>(pool);
  int64_t* pool_top = c.take<int64_t>(1);
  uint32_t* flags = c.take<uint32_t>(2);
  int32_t* jfinal = c.take<int32_t>(1);
  int32_t* bw_n = c.take<int32_t>(1);
  int64_t* bw_off = c.take<int64_t>(1);
  int32_t* status = c.take<int32_t>(1);

  // what must start at zero: the accumulators, the string index and staging
  // offsets of every token, staging counts, the pool counter and the error
  // flags
  FST_CUDA(cudaMemsetAsync(acc, 0, (size_t)(2 * Q * 8), s));
  FST_CUDA(cudaMemsetAsync(tok_b, 0, (size_t)nn * 4, s));
  FST_CUDA(cudaMemsetAsync(scnt, 0, (size_t)nn * 4, s));
  FST_CUDA(cudaMemsetAsync(zero64, 0, (size_t)nn * 8, s));
  FST_CUDA(cudaMemsetAsync(pool_top, 0, 8, s));
  FST_CUDA(cudaMemsetAsync(flags, 0, 8, s));
  FST_CUDA(cudaMemsetAsync(bw_off, 0, 8, s));
  if (n > 0) FST_CUDA(cudaMemcpyAsync(tok_sym, ids, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  FST_CUDA(cudaMemcpyAsync(bw_n, &n, 4, cudaMemcpyHostToDevice, s));
  k_noalloc_iota<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(iota, n);
  FST_CUDA(cudaGetLastError());

  FrontierState S;
  memset(&S, 0, sizeof(S));
  S.Q = f->Q;
  S.acc = acc;
  S.acc_stride = 1;
  S.vmap = vmap;
  S.src_by_id = f->src_by_id;
  S.pool_n = pool_n;
  S.stage = stage;
  S.stage_b = stage_b;
  S.stage_cap = dmax;
  S.Bw = 1;
  S.chain = 1;
  S.scnt = scnt;
  S.pool_q = pool_q;
  S.pool_x = pool_x;
  S.pool_v = pool_v;
  S.pool_base = pool_base;
  S.pool_cnt = pool_cnt;
  S.slot_base = slot_base;
  S.step_rng = step_rng;
  S.pool_top = pool_top;
  S.pool_cap = pool;
  S.flags = flags;
  S.theta_s = f->theta_s;
  S.theta_f = f->theta_f;
  S.start_q = f->start_q;
  S.nstart = f->nstart;
  S.bw_n = bw_n;
  S.bw_off = bw_off;
  const TokenView T{iota, tok_sym, tok_b, zero64};
  const LayoutView L = view_of(f->bwd);
  auto step = [&](int32_t t, int32_t x_t) {
    StepView V;
    V.t = t;
    V.n = 1;
    V.slot0 = t - 1;
    const bool hasx = x_t >= 1 && x_t <= n;
    V.x_t = hasx ? x_t : 0;
    V.x_n = hasx ? 1 : 0;
    V.x_slot0 = hasx ? x_t - 1 : 0;
    V.blocks = f->num_sms * 4;
    return V;
  };
  if (n >= 1 && (rc = launch_vit_first(L, T, step(1, 0), S, s))) return rc;
  for (int32_t t = 1; t <= n; ++t)
    if ((rc = launch_vit_step(L, T, step(t, t + 1), S, s))) return rc;
  if ((rc = launch_vit_final(S, 1, d_score, jfinal, status, s))) return rc;
  if ((rc = launch_backtrace(S, f->olabel, 1, jfinal, d_path, d_olabels, s))) return rc;
  return FST_OK;
}
