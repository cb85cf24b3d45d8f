// noalloc.cu -- fst_viterbi_noalloc: the plain Viterbi decode of one string
// with every piece of per-call working memory taken from one fixed,
// file-scope device array instead of cudaMalloc.
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

// Token tables of one string: position t, compact backpointer base (prefix
// sum of destination segments per symbol).  One thread; n is at most a few
// thousand here.
__global__ void k_noalloc_tokens(const int32_t* __restrict__ ids, int32_t n, const int64_t* __restrict__ sym_seg,
                                 const int64_t* __restrict__ sym_win, int32_t* __restrict__ tok_t,
                                 int64_t* __restrict__ cbase, int64_t* __restrict__ wbase,
                                 uint32_t* __restrict__ epoch) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t acc = 0, wacc = 0;
  for (int32_t i = 0; i < n; ++i) {
    tok_t[i] = i + 1;
    cbase[i] = acc;
    wbase[i] = wacc;
    acc += sym_seg[ids[i] + 1] - sym_seg[ids[i]];
    wacc += sym_win[ids[i] + 1] - sym_win[ids[i]];
  }
  epoch[0] = 1u;  // tags of this call are 1 + position; the cleared frontier holds tag 0
  epoch[1] = 0u;
}

}  // namespace

extern "C" int fst_viterbi_noalloc(fst_t* f, const int32_t* ids, int32_t n, float* d_score, int32_t* d_path,
                                   int32_t* d_olabels, void* stream) {
  if (!f || n < 0 || (n > 0 && (!ids || !d_path)) || !d_score) {
    set_error("fst_viterbi_noalloc: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // sizes first, from host data only
  int64_t store = 0, max_lseg = 0, nwins = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= f->m) {
      set_error("fst_viterbi_noalloc: symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
      return FST_ERR_INVALID_ARG;
    }
    store += f->fwd.h_sym_seg[ids[i] + 1] - f->fwd.h_sym_seg[ids[i]];
    nwins += f->fwd.h_sym_win[ids[i] + 1] - f->fwd.h_sym_win[ids[i]];
  }
  for (int32_t a = 0; a < f->m; ++a)
    max_lseg = std::max<int64_t>(max_lseg, f->fwd.h_sym_lseg[a + 1] - f->fwd.h_sym_lseg[a]);
  const int64_t Q = f->Q, W = f->W;
  auto rnd = [](int64_t bytes) { return ((bytes > 0 ? bytes : 1) + 255) & ~(int64_t)255; };
  const int64_t need = rnd(2 * Q * 8) + rnd(3 * W * 4) + rnd((int64_t)n * f->Ws * 4) + rnd(nwins) + rnd((int64_t)n * 8) + 3 * rnd((int64_t)n * 4) + 2 * rnd((int64_t)n * 8) +
                       rnd(store * 4) + rnd(max_lseg * 8) + rnd(max_lseg * 4) + 5 * rnd(8) + rnd(4) + rnd(8);
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
  unsigned long long* alpha = c.take<unsigned long long>(2 * Q);
  uint32_t* abm = c.take<uint32_t>(3 * W);
  uint32_t* tsum = c.take<uint32_t>((int64_t)n * f->Ws);
  int32_t* tok_sym = c.take<int32_t>(n);
  int32_t* tok_b = c.take<int32_t>(n);
  int32_t* tok_t = c.take<int32_t>(n);
  int64_t* cbase = c.take<int64_t>(n);
  int64_t* zero64 = c.take<int64_t>(n);
  int64_t* wbase = c.take<int64_t>(n);
  uint8_t* fin = c.take<uint8_t>(nwins);
  int32_t* bp = c.take<int32_t>(store);
  unsigned long long* skey = c.take<unsigned long long>(max_lseg);
  uint32_t* scnt = c.take<uint32_t>(max_lseg);
  uint32_t* epoch = c.take<uint32_t>(2);
  int32_t* qfinal = c.take<int32_t>(1);
  int32_t* bw_n = c.take<int32_t>(1);
  int64_t* bw_off = c.take<int64_t>(1);
  int32_t* status = c.take<int32_t>(1);

  // what must start at zero: the tagged frontier (tag 0 is never valid), the
  // string index and scratch bases of every token, the long-segment slots
  FST_CUDA(cudaMemsetAsync(alpha, 0, (size_t)(2 * Q * 8), s));
  FST_CUDA(cudaMemsetAsync(tok_b, 0, (size_t)std::max(n, 1) * 4, s));
  FST_CUDA(cudaMemsetAsync(zero64, 0, (size_t)std::max(n, 1) * 8, s));
  FST_CUDA(cudaMemsetAsync(skey, 0, (size_t)std::max<int64_t>(max_lseg, 1) * 8, s));
  FST_CUDA(cudaMemsetAsync(scnt, 0, (size_t)std::max<int64_t>(max_lseg, 1) * 4, s));
  FST_CUDA(cudaMemsetAsync(bw_off, 0, 8, s));
  FST_CUDA(cudaMemsetAsync(tsum, 0, (size_t)std::max<int64_t>((int64_t)n * f->Ws, 1) * 4, s));
  if (n > 0) FST_CUDA(cudaMemcpyAsync(tok_sym, ids, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  FST_CUDA(cudaMemcpyAsync(bw_n, &n, 4, cudaMemcpyHostToDevice, s));
  FST_CUDA(cudaMemsetAsync(fin, 0, (size_t)std::max<int64_t>(nwins, 1), s));
  k_noalloc_tokens<<<1, 1, 0, s>>>(tok_sym, n, f->fwd.sym_seg, f->fwd.sym_win, tok_t, cbase, wbase, epoch);
  FST_CUDA(cudaGetLastError());

  WaveState S;
  memset(&S, 0, sizeof(S));
  S.Q = f->Q;
  S.epoch = epoch;
  S.tok0 = 0;
  S.alpha = alpha;
  S.bp = bp;
  S.skey = skey;
  S.scnt = scnt;
  S.theta_s = f->theta_s;
  S.theta_f = f->theta_f;
  S.bw_n = bw_n;
  S.bw_off = bw_off;
  S.abm = abm;
  S.bm_start = f->bm_start;
  S.bm_final = f->bm_final;
  S.W = f->W;
  S.bm_rot = f->W;
  S.tsum = tsum;
  S.fin = fin;
  S.bin = nullptr;
  S.b_seg_state = f->bwd.seg_state;
  S.b_seg_pos = f->bwd.seg_pos;
  S.b_seg_len = f->bwd.seg_len;
  S.b_sym_seg = f->bwd.sym_seg;
  S.b_sym_win = f->bwd.sym_win;
  S.b_fwin = f->bwd.fwin;
  S.f_sym_win = f->fwd.sym_win;
  S.sum_start = f->sum_start;
  S.sum_final = f->sum_final;
  S.Ws = f->Ws;
  S.sum_rot = f->Ws;
  const TokenView T{tok_sym, tok_b, tok_t, cbase, zero64, zero64, zero64, zero64, wbase, zero64};
  const LayoutView Lf = view_of(f->fwd);
  for (int32_t t = 1; t <= n; ++t) {
    const int32_t a = ids[t - 1];
    WorkView V;
    memset(&V, 0, sizeof(V));
    V.single = 1;
    V.p0 = t - 1;
    V.sym0 = a;
    V.nitems = f->fwd.h_sym_win[a + 1] - f->fwd.h_sym_win[a];
    FST_CUDA(cudaMemsetAsync(abm + (int64_t)(t % 3) * W, 0, (size_t)W * 4, s));
    if ((rc = launch_vit_step(Lf, T, V, S, f->num_sms, s))) return rc;
  }
  if ((rc = launch_vit_final(S, 1, d_score, qfinal, status, s))) return rc;
  if ((rc = launch_backtrace(Lf, tok_sym, cbase, S, f->olabel, f->fwd.arc_id, 1, qfinal, d_path, d_olabels, s)))
    return rc;
  return FST_OK;
}
