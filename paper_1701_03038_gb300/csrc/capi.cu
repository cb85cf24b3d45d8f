// capi.cu -- the C ABI: FST handles, the plain per-string driver (the
// paper's host loop over positions, Sec. 5) and batch plans (all strings of
// a batch advanced together, one launch per position, graph-capturable).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fst_internal.cuh"
#include "kernels.cuh"

using namespace fstgpu;

// ====================================================================== errors
namespace {
thread_local char g_err[1024] = "";
}

namespace fstgpu {
void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return FST_ERR_CUDA;
}
int grid_for(int64_t work_warps, int block_threads, int num_sms, int max_blocks_per_sm) {
  const int64_t wpb = block_threads / 32;
  int64_t need = (work_warps + wpb - 1) / wpb;
  const int64_t cap = (int64_t)num_sms * max_blocks_per_sm;
  if (need > cap) need = cap;
  return (int)(need < 1 ? 1 : need);
}
}  // namespace fstgpu

extern "C" const char* fst_last_error(void) { return g_err; }

namespace {

constexpr int TB = 256;
inline unsigned nblk(int64_t n, int tb = TB) { return (unsigned)std::max<int64_t>(1, (n + tb - 1) / tb); }

// ============================================================== validation
__global__ void k_convert_arcs(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                               const int32_t* __restrict__ il, const float* __restrict__ w, int64_t A,
                               int32_t Q, int32_t m, int kind, float* __restrict__ theta,
                               unsigned int* __restrict__ err) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= A) return;
  unsigned e = 0;
  if (src && (src[k] < 0 || src[k] >= Q)) e |= 1u;
  if (dst && (dst[k] < 0 || dst[k] >= Q)) e |= 2u;
  if (il && (il[k] < 0 || il[k] >= m)) e |= 4u;
  float th = kind == FST_WEIGHT_COST ? -w[k] : w[k];
  if (isnan(th) || th == INFINITY) e |= 8u;
  theta[k] = __fadd_rn(th, 0.0f);  // -0 -> +0
  if (e) atomicOr(err, e);
}

__global__ void k_convert_states(const float* __restrict__ w, int32_t Q, int kind, float* __restrict__ out,
                                 unsigned int* __restrict__ err) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const float th = kind == FST_WEIGHT_COST ? -w[q] : w[q];
  if (isnan(th) || th == INFINITY) atomicOr(err, 16u);
  out[q] = __fadd_rn(th, 0.0f);
}

// bit q of word q / 32 is set when w[q] is finite
__global__ void k_finite_bitmap(const float* __restrict__ w, int32_t Q, uint32_t* __restrict__ bm, int32_t W) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= W) return;
  uint32_t m = 0;
  for (int k = 0; k < 32; ++k) {
    const int64_t q = i * 32 + k;
    if (q < Q && w[q] != -INFINITY) m |= 1u << k;
  }
  bm[i] = m;
}

// bit j of summary word i is set when bitmap word 32 i + j is nonzero
__global__ void k_bitmap_summary(const uint32_t* __restrict__ bm, int32_t W, uint32_t* __restrict__ sum, int32_t Ws) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Ws) return;
  uint32_t m = 0;
  for (int k = 0; k < 32; ++k) {
    const int64_t w = i * 32 + k;
    if (w < W && bm[w] != 0u) m |= 1u << k;
  }
  sum[i] = m;
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_check_ids(const int32_t* __restrict__ ids, int64_t n, int32_t m, unsigned int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (ids[i] < 0 || ids[i] >= m)) atomicOr(err, 32u);
}

// Run epochs: epoch[0] is the first tag of the current run and epoch[1]
// the number of tags that run uses.  The next run starts past them; when the
// 32-bit range would run out it restarts at 1 and the frontiers are cleared
// (tag 0, left by the clear, is never a valid tag).
__global__ void k_epoch_advance(uint32_t* epoch, uint32_t span, uint32_t* clear) {
  const uint64_t next = (uint64_t)epoch[0] + (uint64_t)epoch[1] + 1ull;
  if (next + (uint64_t)span + 1ull >= 0xffffffffull) {
    epoch[0] = 1u;
    *clear = 1u;
  } else {
    epoch[0] = (uint32_t)next;
    *clear = 0u;
  }
  epoch[1] = span;
}

__global__ void k_clear_if(const uint32_t* clear, unsigned long long* p, int64_t n) {
  if (!*clear) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0ull;
}

template <class T>
int to_device(const T* h, T** d, int64_t n) {
  int rc = dalloc(d, n);
  if (rc) return rc;
  if (n > 0) FST_CUDA(cudaMemcpy(*d, h, (size_t)n * sizeof(T), cudaMemcpyHostToDevice));
  return FST_OK;
}

int read_err_flag(unsigned int* d_err, const char* what) {
  unsigned int e = 0;
  FST_CUDA(cudaMemcpy(&e, d_err, sizeof(e), cudaMemcpyDeviceToHost));
  if (e) {
    set_error("%s: invalid input (flags 0x%x: 1=src 2=dst 4=ilabel 8=arc weight 16=start/final weight 32=symbol)",
              what, e);
    return FST_ERR_INVALID_ARG;
  }
  return FST_OK;
}

// ================================================================= RAII
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

}  // namespace

// ======================================================== plain workspace
struct PlainWs {
  int64_t cap_n = 0, cap_store = 0;
  unsigned long long* alpha = nullptr;  // [2][Q]
  unsigned long long* beta = nullptr;
  int32_t *tok_sym = nullptr, *tok_b = nullptr, *tok_t = nullptr;
  int64_t *cbase = nullptr, *zero64 = nullptr, *wbase = nullptr, *bwbase = nullptr;
  int32_t* bp = nullptr;
  uint8_t *wlive = nullptr, *fin = nullptr, *bin = nullptr, *bmk = nullptr;
  int64_t cap_wlive = 0, cap_bin = 0;
  float* rc = nullptr;
  uint32_t *mkey = nullptr, *ekey = nullptr;
  double *csum = nullptr, *esum = nullptr;
  unsigned long long* skey = nullptr;
  uint32_t* scnt = nullptr;
  float2* spart = nullptr;
  float *cnt = nullptr, *comp = nullptr, *counts_out = nullptr;
  int32_t *paths = nullptr, *olabels = nullptr, *qfinal = nullptr, *status = nullptr;
  float* score = nullptr;
  double* logz = nullptr;
  int32_t* bw_n = nullptr;
  int64_t* bw_off = nullptr;
  uint32_t *epoch = nullptr, *clear = nullptr;
  uint32_t *abm = nullptr, *bbm = nullptr;  // [3][W] live-state bitmaps
  uint32_t *tsum = nullptr, *bsum = nullptr;  // per-token forward summaries [n][Ws]; backward [3][Ws]
  int64_t cap_tsum = 0;
  int64_t max_lseg = 0, max_lwin = 0;
  ~PlainWs() {
    dfree(abm); dfree(bbm); dfree(tsum); dfree(bsum); dfree(wbase); dfree(wlive); dfree(bwbase); dfree(fin); dfree(bin); dfree(bmk);
    dfree(alpha); dfree(beta); dfree(tok_sym); dfree(tok_b); dfree(tok_t); dfree(cbase); dfree(zero64);
    dfree(bp); dfree(rc); dfree(mkey); dfree(ekey); dfree(csum); dfree(esum); dfree(skey); dfree(scnt);
    dfree(spart); dfree(cnt); dfree(comp); dfree(counts_out); dfree(paths); dfree(olabels); dfree(qfinal);
    dfree(status); dfree(score); dfree(logz); dfree(bw_n); dfree(bw_off); dfree(epoch); dfree(clear);
  }
};

namespace {

int64_t max_diff(const int64_t* h, int32_t m) {
  int64_t mx = 0;
  for (int32_t a = 0; a < m; ++a) mx = std::max(mx, h[a + 1] - h[a]);
  return mx;
}

int plain_init(fst_s* f) {
  if (f->plain) return FST_OK;
  PlainWs* w = new PlainWs();
  f->plain = w;
  const int64_t Q = f->Q;
  int rc;
  w->max_lseg = std::max(max_diff(f->fwd.h_sym_lseg, f->m), max_diff(f->bwd.h_sym_lseg, f->m));
  w->max_lwin = std::max(max_diff(f->fwd.h_sym_lwin, f->m), max_diff(f->bwd.h_sym_lwin, f->m));
  if ((rc = dalloc(&w->alpha, 2 * Q)) || (rc = dalloc(&w->beta, 2 * Q)) || (rc = dalloc(&w->skey, w->max_lseg)) ||
      (rc = dalloc(&w->scnt, w->max_lseg)) || (rc = dalloc(&w->spart, w->max_lwin)) ||
      (rc = dalloc(&w->qfinal, 1)) || (rc = dalloc(&w->status, 1)) || (rc = dalloc(&w->score, 1)) ||
      (rc = dalloc(&w->logz, 1)) || (rc = dalloc(&w->bw_n, 1)) || (rc = dalloc(&w->bw_off, 1)) ||
      (rc = dalloc(&w->epoch, 2)) || (rc = dalloc(&w->clear, 1)) || (rc = dalloc(&w->abm, 3 * (int64_t)f->W)) ||
      (rc = dalloc(&w->bbm, 3 * (int64_t)f->W)) || (rc = dalloc(&w->bsum, 3 * (int64_t)f->Ws)))
    return rc;
  FST_CUDA(cudaMemset(w->alpha, 0, (size_t)2 * Q * sizeof(unsigned long long)));
  FST_CUDA(cudaMemset(w->beta, 0, (size_t)2 * Q * sizeof(unsigned long long)));
  FST_CUDA(cudaMemset(w->skey, 0, (size_t)std::max<int64_t>(1, w->max_lseg) * 8));
  FST_CUDA(cudaMemset(w->scnt, 0, (size_t)std::max<int64_t>(1, w->max_lseg) * 4));
  FST_CUDA(cudaMemset(w->bw_off, 0, sizeof(int64_t)));
  FST_CUDA(cudaMemset(w->epoch, 0, 2 * sizeof(uint32_t)));
  return FST_OK;
}

int plain_reserve(PlainWs* w, int64_t n, int64_t store, int64_t nwins, int64_t nwins_b) {
  int rc;
  if (nwins > w->cap_wlive) {
    const int64_t c = std::max<int64_t>(nwins, 2 * w->cap_wlive);
    dfree(w->wlive);
    dfree(w->fin);
    w->cap_wlive = 0;
    if ((rc = dalloc(&w->wlive, c)) || (rc = dalloc(&w->fin, c))) return rc;
    w->cap_wlive = c;
  }
  if (nwins_b > w->cap_bin) {
    const int64_t c = std::max<int64_t>(nwins_b, 2 * w->cap_bin);
    dfree(w->bin);
    dfree(w->bmk);
    w->cap_bin = 0;
    if ((rc = dalloc(&w->bin, c)) || (rc = dalloc(&w->bmk, c))) return rc;
    w->cap_bin = c;
  }
  if (n > w->cap_n) {
    const int64_t c = std::max<int64_t>(n, 2 * w->cap_n);
    dfree(w->tok_sym); dfree(w->tok_b); dfree(w->tok_t); dfree(w->cbase); dfree(w->zero64); dfree(w->wbase);
    dfree(w->bwbase);
    dfree(w->mkey); dfree(w->ekey); dfree(w->csum); dfree(w->esum); dfree(w->paths); dfree(w->olabels);
    w->cap_n = 0;
    if ((rc = dalloc(&w->tok_sym, c)) || (rc = dalloc(&w->tok_b, c)) || (rc = dalloc(&w->tok_t, c)) ||
        (rc = dalloc(&w->cbase, c)) || (rc = dalloc(&w->zero64, c)) || (rc = dalloc(&w->wbase, c)) ||
        (rc = dalloc(&w->bwbase, c)) ||
        (rc = dalloc(&w->mkey, c)) ||
        (rc = dalloc(&w->ekey, c)) || (rc = dalloc(&w->csum, c)) || (rc = dalloc(&w->esum, c)) ||
        (rc = dalloc(&w->paths, c)) || (rc = dalloc(&w->olabels, c)))
      return rc;
    FST_CUDA(cudaMemset(w->tok_b, 0, (size_t)c * sizeof(int32_t)));
    FST_CUDA(cudaMemset(w->zero64, 0, (size_t)c * sizeof(int64_t)));
    w->cap_n = c;
  }
  if (store > w->cap_store) {
    const int64_t c = std::max<int64_t>(store, 2 * w->cap_store);
    dfree(w->bp); dfree(w->rc);
    w->cap_store = 0;
    if ((rc = dalloc(&w->bp, c)) || (rc = dalloc(&w->rc, c))) return rc;
    w->cap_store = c;
  }
  return FST_OK;
}

// Upload the tokens of one string: symbol, position, compact-storage base.
int plain_tokens(fst_s* f, const int32_t* ids, int32_t n, cudaStream_t s) {
  PlainWs* w = f->plain;
  std::vector<int32_t> tt(std::max(n, 1));
  std::vector<int64_t> cb(std::max(n, 1)), wb(std::max(n, 1)), bwb(std::max(n, 1));
  int64_t acc = 0, wacc = 0, bwacc = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= f->m) {
      set_error("symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
      return FST_ERR_INVALID_ARG;
    }
    tt[i] = i + 1;
    cb[i] = acc;
    wb[i] = wacc;
    bwb[i] = bwacc;
    acc += f->fwd.h_sym_seg[ids[i] + 1] - f->fwd.h_sym_seg[ids[i]];
    wacc += f->fwd.h_sym_win[ids[i] + 1] - f->fwd.h_sym_win[ids[i]];
    bwacc += f->bwd.h_sym_win[ids[i] + 1] - f->bwd.h_sym_win[ids[i]];
  }
  int rc = plain_reserve(w, std::max(n, 1), std::max<int64_t>(acc, 1), std::max<int64_t>(wacc, 1),
                         std::max<int64_t>(bwacc, 1));
  if (rc) return rc;
  const int64_t ntsum = std::max<int64_t>((int64_t)n * f->Ws, 1);
  if (ntsum > w->cap_tsum) {
    dfree(w->tsum);
    w->cap_tsum = 0;
    if ((rc = dalloc(&w->tsum, std::max<int64_t>(ntsum, 2 * w->cap_tsum)))) return rc;
    w->cap_tsum = ntsum;
  }
  FST_CUDA(cudaMemsetAsync(w->tsum, 0, (size_t)ntsum * 4, s));
  if (n > 0) {
    FST_CUDA(cudaMemcpyAsync(w->tok_sym, ids, (size_t)n * 4, cudaMemcpyHostToDevice, s));
    FST_CUDA(cudaMemcpyAsync(w->tok_t, tt.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    FST_CUDA(cudaMemcpyAsync(w->cbase, cb.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
    FST_CUDA(cudaMemcpyAsync(w->wbase, wb.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
    FST_CUDA(cudaMemcpyAsync(w->bwbase, bwb.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
    FST_CUDA(cudaMemsetAsync(w->wlive, 0, (size_t)wacc, s));
    FST_CUDA(cudaMemsetAsync(w->fin, 0, (size_t)wacc, s));
    FST_CUDA(cudaMemsetAsync(w->bin, 0, (size_t)bwacc, s));
    FST_CUDA(cudaMemsetAsync(w->bmk, 0, (size_t)bwacc, s));
  }
  FST_CUDA(cudaMemcpyAsync(w->bw_n, &n, 4, cudaMemcpyHostToDevice, s));
  // fresh tags for this string
  k_epoch_advance<<<1, 1, 0, s>>>(w->epoch, (uint32_t)n + 1u, w->clear);
  k_clear_if<<<nblk(2 * (int64_t)f->Q), TB, 0, s>>>(w->clear, w->alpha, 2 * (int64_t)f->Q);
  k_clear_if<<<nblk(2 * (int64_t)f->Q), TB, 0, s>>>(w->clear, w->beta, 2 * (int64_t)f->Q);
  FST_CUDA(cudaMemsetAsync(w->skey, 0, (size_t)std::max<int64_t>(1, w->max_lseg) * 8, s));
  FST_CUDA(cudaMemsetAsync(w->scnt, 0, (size_t)std::max<int64_t>(1, w->max_lseg) * 4, s));
  FST_CUDA(cudaGetLastError());
  return FST_OK;
}

TokenView plain_tokview(PlainWs* w) {
  return TokenView{w->tok_sym, w->tok_b, w->tok_t, w->cbase, w->zero64, w->zero64, w->zero64, w->zero64, w->wbase,
                   w->bwbase};
}

WaveState plain_state(fst_s* f) {
  PlainWs* w = f->plain;
  WaveState S;
  memset(&S, 0, sizeof(S));
  S.Q = f->Q;
  S.epoch = w->epoch;
  S.tok0 = 0;
  S.alpha = w->alpha;
  S.beta = w->beta;
  S.bp = w->bp;
  S.rc = w->rc;
  S.mkey = w->mkey;
  S.ekey = w->ekey;
  S.csum = w->csum;
  S.esum = w->esum;
  S.skey = w->skey;
  S.scnt = w->scnt;
  S.spart = w->spart;
  S.theta_s = f->theta_s;
  S.theta_f = f->theta_f;
  S.logz = w->logz;
  S.gweight = nullptr;
  S.bw_n = w->bw_n;
  S.bw_off = w->bw_off;
  S.abm = w->abm;
  S.bbm = w->bbm;
  S.bm_start = f->bm_start;
  S.bm_final = f->bm_final;
  S.W = f->W;
  S.bm_rot = f->W;
  S.wlive = w->wlive;
  S.tsum = w->tsum;
  S.bsum = w->bsum;
  S.fin = w->fin;
  S.bin = w->bin;
  S.b_seg_state = f->bwd.seg_state;
  S.b_seg_pos = f->bwd.seg_pos;
  S.b_seg_len = f->bwd.seg_len;
  S.b_sym_seg = f->bwd.sym_seg;
  S.b_sym_win = f->bwd.sym_win;
  S.b_fwin = f->bwd.fwin;
  S.f_sym_win = f->fwd.sym_win;
  S.bmk = w->bmk;
  S.f_seg_state = f->fwd.seg_state;
  S.f_seg_pos = f->fwd.seg_pos;
  S.f_seg_len = f->fwd.seg_len;
  S.f_sym_seg = f->fwd.sym_seg;
  S.f_bwin = f->fwd.bwin;
  S.sum_start = f->sum_start;
  S.sum_final = f->sum_final;
  S.Ws = f->Ws;
  S.sum_rot = f->Ws;
  return S;
}

// Clear rotation r of a [3][W] bitmap set before the launch that fills it.
int clear_rot(uint32_t* bm, int32_t r, int64_t words, cudaStream_t s) {
  FST_CUDA(cudaMemsetAsync(bm + (int64_t)r * words, 0, (size_t)words * 4, s));
  return FST_OK;
}

WorkView single_work(int32_t p, int32_t sym, int64_t nitems) {
  WorkView W;
  memset(&W, 0, sizeof(W));
  W.single = 1;
  W.p0 = p;
  W.sym0 = sym;
  W.nitems = nitems;
  return W;
}

// the launchers size step grids from the SM count and the kernel's occupancy
int step_grid(const fst_s* f, int64_t) { return f->num_sms; }

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

// ============================================================ create/destroy
extern "C" int fst_create(int32_t num_states, int64_t num_arcs, const int32_t* src, const int32_t* dst,
                          const int32_t* ilabel, const int32_t* olabel, const float* weight, int32_t weight_kind,
                          const float* start_weight, const float* final_weight, int32_t num_isyms, int32_t flags,
                          fst_t** out) {
  if (!out) { set_error("out is NULL"); return FST_ERR_INVALID_ARG; }
  *out = nullptr;
  if (num_states < 1 || num_arcs < 0 || num_isyms < 1 || num_arcs >= ((int64_t)1 << 31) ||
      (weight_kind != FST_WEIGHT_LOG && weight_kind != FST_WEIGHT_COST)) {
    set_error("bad sizes or weight kind (Q=%d A=%lld m=%d kind=%d)", num_states, (long long)num_arcs, num_isyms,
              weight_kind);
    return FST_ERR_INVALID_ARG;
  }
  if ((num_arcs > 0 && (!src || !dst || !ilabel || !weight)) || !start_weight || !final_weight) {
    set_error("a required array is NULL");
    return FST_ERR_INVALID_ARG;
  }
  const bool dev = (flags & FST_FLAG_DEVICE_PTRS) != 0;
  fst_s* f = new fst_s();
  f->Q = num_states;
  f->A = num_arcs;
  f->m = num_isyms;
  cudaGetDevice(&f->device);
  cudaDeviceGetAttribute(&f->num_sms, cudaDevAttrMultiProcessorCount, f->device);
  if (f->num_sms <= 0) f->num_sms = 1;
  const int64_t A = num_arcs, Q = num_states;
  int32_t *d_src = nullptr, *d_dst = nullptr, *d_il = nullptr;
  float *d_w = nullptr, *d_theta = nullptr, *d_ws = nullptr, *d_wf = nullptr;
  unsigned int* d_err = nullptr;
  int rc = FST_OK;
  auto cleanup = [&]() {
    if (!dev) { dfree(d_src); dfree(d_dst); dfree(d_il); dfree(d_w); dfree(d_ws); dfree(d_wf); }
    dfree(d_theta);
    dfree(d_err);
  };
  auto copy_in = [&](const void* h, void** d, size_t bytes) -> int {
    if (dev) { *d = (void*)h; return FST_OK; }
    cudaError_t e = cudaMalloc(d, bytes ? bytes : 1);
    if (e != cudaSuccess) { (void)cudaGetLastError(); set_error("cudaMalloc failed"); return FST_ERR_OOM; }
    if (bytes) {
      e = cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "fst_create copy");
    }
    return FST_OK;
  };
  cudaStream_t s = 0;
  do {
    if ((rc = copy_in(src, (void**)&d_src, (size_t)A * 4))) break;
    if ((rc = copy_in(dst, (void**)&d_dst, (size_t)A * 4))) break;
    if ((rc = copy_in(ilabel, (void**)&d_il, (size_t)A * 4))) break;
    if ((rc = copy_in(weight, (void**)&d_w, (size_t)A * 4))) break;
    if ((rc = copy_in(start_weight, (void**)&d_ws, (size_t)Q * 4))) break;
    if ((rc = copy_in(final_weight, (void**)&d_wf, (size_t)Q * 4))) break;
    if ((rc = dalloc(&d_theta, A)) || (rc = dalloc(&d_err, 1)) || (rc = dalloc(&f->theta_s, Q)) ||
        (rc = dalloc(&f->theta_f, Q)) || (rc = dalloc(&f->olabel, A)))
      break;
    if (cudaMemset(d_err, 0, 4) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "memset"); break; }
    if (A > 0) k_convert_arcs<<<nblk(A), TB, 0, s>>>(d_src, d_dst, d_il, d_w, A, f->Q, f->m, weight_kind, d_theta, d_err);
    k_convert_states<<<nblk(Q), TB, 0, s>>>(d_ws, f->Q, weight_kind, f->theta_s, d_err);
    k_convert_states<<<nblk(Q), TB, 0, s>>>(d_wf, f->Q, weight_kind, f->theta_f, d_err);
    if (olabel) {
      cudaError_t e = cudaMemcpy(f->olabel, olabel, (size_t)A * 4, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
      if (A > 0 && e != cudaSuccess) { rc = cuda_fail(e, "olabel copy"); break; }
    } else if (A > 0) {
      k_fill_i32<<<nblk(A), TB, 0, s>>>(f->olabel, A, -1);
    }
    f->W = (int32_t)((Q + 31) / 32);
    if ((rc = dalloc(&f->bm_start, f->W)) || (rc = dalloc(&f->bm_final, f->W))) break;
    k_finite_bitmap<<<nblk(f->W), TB, 0, s>>>(f->theta_s, f->Q, f->bm_start, f->W);
    k_finite_bitmap<<<nblk(f->W), TB, 0, s>>>(f->theta_f, f->Q, f->bm_final, f->W);
    f->Ws = (f->W + 31) / 32;
    if ((rc = dalloc(&f->sum_start, f->Ws)) || (rc = dalloc(&f->sum_final, f->Ws))) break;
    k_bitmap_summary<<<nblk(f->Ws), TB, 0, s>>>(f->bm_start, f->W, f->sum_start, f->Ws);
    k_bitmap_summary<<<nblk(f->Ws), TB, 0, s>>>(f->bm_final, f->W, f->sum_final, f->Ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "fst_create kernels"); break; }
    if ((rc = read_err_flag(d_err, "fst_create"))) break;
    rc = build_store(f, d_src, d_dst, d_il, d_theta, s);
  } while (0);
  cleanup();
  if (rc) {
    fst_destroy(f);
    return rc;
  }
  *out = f;
  return FST_OK;
}

extern "C" int fst_destroy(fst_t* f) {
  if (!f) return FST_OK;
  DevGuard g(f->device);
  delete f->plain;
  f->plain = nullptr;
  free_layout(f->fwd);
  free_layout(f->bwd);
  dfree(f->theta_s);
  dfree(f->theta_f);
  dfree(f->bm_start);
  dfree(f->bm_final);
  dfree(f->sum_start);
  dfree(f->sum_final);
  dfree(f->olabel);
  dfree(f->sym_arc);
  free(f->h_sym_arc);
  delete f;
  return FST_OK;
}

extern "C" int fst_info(const fst_t* f, int32_t* num_states, int64_t* num_arcs, int32_t* num_isyms,
                        int64_t* padded_arcs, int64_t* num_windows, int64_t* dst_segments, int64_t* src_segments) {
  if (!f) { set_error("fst is NULL"); return FST_ERR_INVALID_ARG; }
  if (num_states) *num_states = f->Q;
  if (num_arcs) *num_arcs = f->A;
  if (num_isyms) *num_isyms = f->m;
  if (padded_arcs) *padded_arcs = f->fwd.P;
  if (num_windows) *num_windows = f->fwd.nwin;
  if (dst_segments) *dst_segments = f->fwd.nseg;
  if (src_segments) *src_segments = f->bwd.nseg;
  return FST_OK;
}

extern "C" int fst_symbol_stats(const fst_t* f, int64_t* arcs, int64_t* dsts, int64_t* srcs) {
  if (!f) { set_error("fst is NULL"); return FST_ERR_INVALID_ARG; }
  for (int32_t a = 0; a < f->m; ++a) {
    if (arcs) arcs[a] = f->h_sym_arc[a + 1] - f->h_sym_arc[a];
    if (dsts) dsts[a] = f->fwd.h_sym_seg[a + 1] - f->fwd.h_sym_seg[a];
    if (srcs) srcs[a] = f->bwd.h_sym_seg[a + 1] - f->bwd.h_sym_seg[a];
  }
  return FST_OK;
}

extern "C" int fst_set_weights(fst_t* f, const float* weight, int32_t weight_kind, int32_t flags) {
  if (!f || (!weight && f->A > 0) || (weight_kind != FST_WEIGHT_LOG && weight_kind != FST_WEIGHT_COST)) {
    set_error("fst_set_weights: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  DevGuard g(f->device);
  const int64_t A = f->A;
  if (A == 0) return FST_OK;
  const bool dev = (flags & FST_FLAG_DEVICE_PTRS) != 0;
  float *d_w = nullptr, *d_theta = nullptr;
  unsigned int* d_err = nullptr;
  int rc = FST_OK;
  do {
    if (!dev) {
      if ((rc = to_device(weight, &d_w, A))) break;
    }
    if ((rc = dalloc(&d_theta, A)) || (rc = dalloc(&d_err, 1))) break;
    if (cudaMemset(d_err, 0, 4) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "memset"); break; }
    k_convert_arcs<<<nblk(A), TB>>>(nullptr, nullptr, nullptr, dev ? weight : d_w, A, f->Q, f->m, weight_kind,
                                    d_theta, d_err);
    if ((rc = read_err_flag(d_err, "fst_set_weights"))) break;
    if ((rc = set_layout_weights(f, d_theta, 0))) break;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = cuda_fail(e, "fst_set_weights");
  } while (0);
  dfree(d_w);
  dfree(d_theta);
  dfree(d_err);
  return rc;
}

// ============================================================ plain method
extern "C" int fst_viterbi(fst_t* f, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path,
                           int32_t* olabels) {
  if (!f || n < 0 || (n > 0 && (!ids || !arc_path)) || !best_score) {
    set_error("fst_viterbi: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  DevGuard g(f->device);
  int rc;
  if ((rc = plain_init(f))) return rc;
  cudaStream_t s = 0;
  if ((rc = plain_tokens(f, ids, n, s))) return rc;
  PlainWs* w = f->plain;
  const LayoutView Lf = view_of(f->fwd);
  const TokenView T = plain_tokview(w);
  const WaveState S = plain_state(f);
  // one launch per input position over the arcs of delta[w_t] (Sec. 5)
  for (int32_t t = 1; t <= n; ++t) {
    const int32_t a = ids[t - 1];
    const int64_t nitems = f->fwd.h_sym_win[a + 1] - f->fwd.h_sym_win[a];
    if ((rc = clear_rot(w->abm, t % 3, f->W, s))) return rc;
    if ((rc = launch_vit_step(Lf, T, single_work(t - 1, a, nitems), S, step_grid(f, nitems), s))) return rc;
  }
  if ((rc = launch_vit_final(S, 1, w->score, w->qfinal, w->status, s))) return rc;
  if ((rc = launch_backtrace(Lf, w->tok_sym, w->cbase, S, f->olabel, f->fwd.arc_id, 1, w->qfinal, w->paths,
                             w->olabels, s)))
    return rc;
  int32_t st = 0;
  FST_CUDA(cudaMemcpy(best_score, w->score, 4, cudaMemcpyDeviceToHost));
  FST_CUDA(cudaMemcpy(&st, w->status, 4, cudaMemcpyDeviceToHost));
  if (n > 0) {
    FST_CUDA(cudaMemcpy(arc_path, w->paths, (size_t)n * 4, cudaMemcpyDeviceToHost));
    if (olabels) FST_CUDA(cudaMemcpy(olabels, w->olabels, (size_t)n * 4, cudaMemcpyDeviceToHost));
  }
  if (st != FST_OK) {
    set_error("no accepting path");
    return FST_ERR_NO_PATH;
  }
  return FST_OK;
}

extern "C" int fst_forward_backward(fst_t* f, const int32_t* ids, int32_t n, double* log_z, float* arc_posteriors) {
  if (!f || n < 0 || (n > 0 && !ids) || !log_z) {
    set_error("fst_forward_backward: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  DevGuard g(f->device);
  int rc;
  if ((rc = plain_init(f))) return rc;
  cudaStream_t s = 0;
  if ((rc = plain_tokens(f, ids, n, s))) return rc;
  PlainWs* w = f->plain;
  if (arc_posteriors && !w->cnt) {
    if ((rc = dalloc(&w->cnt, f->bwd.P)) || (rc = dalloc(&w->comp, f->bwd.P)) || (rc = dalloc(&w->counts_out, f->A)))
      return rc;
  }
  const LayoutView Lf = view_of(f->fwd), Lb = view_of(f->bwd);
  const TokenView T = plain_tokview(w);
  WaveState S = plain_state(f);
  if (n > 0) {
    FST_CUDA(cudaMemsetAsync(w->mkey, 0, (size_t)n * 4, s));
    FST_CUDA(cudaMemsetAsync(w->ekey, 0, (size_t)n * 4, s));
  }
  for (int32_t t = 1; t <= n; ++t) {
    const int32_t a = ids[t - 1];
    const int64_t nitems = f->fwd.h_sym_win[a + 1] - f->fwd.h_sym_win[a];
    if ((rc = clear_rot(w->abm, t % 3, f->W, s))) return rc;
    if ((rc = launch_fwd_step(Lf, T, single_work(t - 1, a, nitems), S, step_grid(f, nitems), s))) return rc;
  }
  if ((rc = launch_fb_final(S, 1, w->logz, w->status, s))) return rc;
  if (arc_posteriors) {
    CountView C{0, w->cnt, w->comp, nullptr};
    FST_CUDA(cudaMemsetAsync(w->cnt, 0, (size_t)f->bwd.P * 4, s));
    FST_CUDA(cudaMemsetAsync(w->comp, 0, (size_t)f->bwd.P * 4, s));
    for (int32_t t = n; t >= 1; --t) {
      // step t also restores alpha_{t-2} when the string is longer than t - 1
      ScatterJob J{Lf, WorkView{}, t - 1};
      if (t >= 3 && t - 1 < n) {
        const int32_t a = ids[t - 3];
        J.W = single_work(t - 3, a, f->fwd.h_sym_win[a + 1] - f->fwd.h_sym_win[a]);
      }
      const int32_t a = ids[t - 1];
      const int64_t nitems = f->bwd.h_sym_win[a + 1] - f->bwd.h_sym_win[a];
      if (t >= 2 && ((rc = clear_rot(w->bbm, (t - 1) % 3, f->W, s)) || (rc = clear_rot(w->bsum, (t - 1) % 3, f->Ws, s))))
        return rc;
      if ((rc = launch_bwd_step(Lb, T, single_work(t - 1, a, nitems), S, C, J,
                                step_grid(f, std::max(nitems, J.W.nitems)), s)))
        return rc;
    }
    if ((rc = launch_counts_out(f->bwd.arc_id, f->bwd.P, C, w->counts_out, s))) return rc;
    if (f->A > 0)
      FST_CUDA(cudaMemcpy(arc_posteriors, w->counts_out, (size_t)f->A * 4, cudaMemcpyDeviceToHost));
  }
  int32_t st = 0;
  FST_CUDA(cudaMemcpy(log_z, w->logz, 8, cudaMemcpyDeviceToHost));
  FST_CUDA(cudaMemcpy(&st, w->status, 4, cudaMemcpyDeviceToHost));
  if (st != FST_OK) {
    set_error("no accepting path");
    return FST_ERR_NO_PATH;
  }
  return FST_OK;
}
