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
#include <array>
#include <chrono>
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
int LaunchProfile::read(double* ms_by_kind, int64_t* launches_by_kind) {
  double ms[FST_PROF_KINDS] = {0};
  int64_t cnt[FST_PROF_KINDS] = {0};
  if (used > 0) FST_CUDA(cudaEventSynchronize(ev[2 * (used - 1) + 1]));
  for (size_t i = 0; i < used; ++i) {
    float t = 0.f;
    FST_CUDA(cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]));
    const int k = kind[i];
    if (k >= 0 && k < FST_PROF_KINDS) {
      ms[k] += t;
      cnt[k] += 1;
    }
  }
  used = 0;
  for (int k = 0; k < FST_PROF_KINDS; ++k) {
    if (ms_by_kind) ms_by_kind[k] = ms[k];
    if (launches_by_kind) launches_by_kind[k] = cnt[k];
  }
  return FST_OK;
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

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
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

// Launch bracketed by the handle's profile events (fst_profile).
#define PLAIN_PROF(kind, call)                        \
  do {                                                \
    const long pi__ = f->prof.begin((kind), s);       \
    const int rc__ = (call);                          \
    f->prof.end(pi__, s);                             \
    if (rc__) return rc__;                            \
  } while (0)

// ======================================================== plain workspace
// Working memory of the plain method (one string, one launch per position),
// kept by the FST handle and grown on demand.
struct PlainWs {
  unsigned long long* acc = nullptr;    // [2][Q] x 2 words (sum, maximum), zero between runs
  double* beta = nullptr;               // [2][Q] backward values
  int32_t* vmap = nullptr;              // [2][Q]
  int32_t *tok_sym = nullptr, *tok_b = nullptr;
  int32_t* iota = nullptr;              // step list: token t-1 is the only slot of position t
  int32_t* step0 = nullptr;             // [cap_n + 2] step offsets of the persistent passes: step0[t] = t - 1
  uint32_t* gbar = nullptr;             // [2] grid barrier of the persistent passes
  int64_t* zero64 = nullptr;            // staging offsets: one token per step
  int64_t *slot_base = nullptr, *step_rng = nullptr;
  uint32_t* scnt = nullptr;
  int64_t* pool_base = nullptr;
  int32_t* pool_cnt = nullptr;
  uint32_t *mkey = nullptr, *ekey = nullptr;
  double *csum = nullptr, *esum = nullptr;
  int32_t *paths = nullptr, *olabels = nullptr;
  int64_t cap_n = 0;
  int32_t *stage = nullptr, *stage_b = nullptr;
  int64_t cap_stage = 0;
  int32_t *pool_q = nullptr, *pool_x = nullptr, *pool_n = nullptr;
  double* pool_v = nullptr;             // Viterbi scores (float32) or forward values (float64)
  int64_t cap_pool = 0;
  float *cnt = nullptr, *comp = nullptr, *counts_out = nullptr;
  int32_t *jfinal = nullptr, *status = nullptr, *bw_n = nullptr;
  float* score = nullptr;
  double* logz = nullptr;
  int64_t* bw_off = nullptr;
  int64_t* pool_top = nullptr;
  uint32_t* flags = nullptr;
  bool last_fb = false;                 // the last call was forward-backward (pool_n holds arc counts)
  ~PlainWs() {
    dfree(acc); dfree(beta); dfree(vmap); dfree(tok_sym); dfree(tok_b); dfree(iota); dfree(zero64);
    dfree(step0); dfree(gbar); dfree(slot_base); dfree(step_rng); dfree(scnt); dfree(pool_base); dfree(pool_cnt); dfree(mkey); dfree(ekey);
    dfree(csum); dfree(esum); dfree(paths); dfree(olabels); dfree(stage); dfree(stage_b); dfree(pool_q);
    dfree(pool_x); dfree(pool_n); dfree(pool_v); dfree(cnt); dfree(comp); dfree(counts_out); dfree(jfinal); dfree(status);
    dfree(bw_n); dfree(score); dfree(logz); dfree(bw_off); dfree(pool_top); dfree(flags);
  }
};

namespace {

int plain_init(fst_s* f) {
  if (f->plain) return FST_OK;
  PlainWs* w = new PlainWs();
  f->plain = w;
  const int64_t Q = f->Q;
  int rc;
  if ((rc = dalloc(&w->acc, 4 * Q)) || (rc = dalloc(&w->beta, 2 * Q)) || (rc = dalloc(&w->vmap, 2 * Q)) ||
      (rc = dalloc(&w->jfinal, 1)) || (rc = dalloc(&w->status, 1)) || (rc = dalloc(&w->score, 1)) ||
      (rc = dalloc(&w->logz, 1)) || (rc = dalloc(&w->bw_n, 1)) || (rc = dalloc(&w->bw_off, 1)) ||
      (rc = dalloc(&w->pool_top, 1)) || (rc = dalloc(&w->flags, 2)) || (rc = dalloc(&w->gbar, 2)))
    return rc;
  FST_CUDA(cudaMemset(w->acc, 0, (size_t)4 * Q * sizeof(unsigned long long)));
  FST_CUDA(cudaMemset(w->beta, 0, (size_t)2 * Q * sizeof(double)));
  FST_CUDA(cudaMemset(w->bw_off, 0, sizeof(int64_t)));
  FST_CUDA(cudaMemset(w->flags, 0, 2 * sizeof(uint32_t)));
  return FST_OK;
}

// Grow the per-string buffers: n tokens, a staging buffer for the largest
// slice, and a pool for every destination of the string's symbols (its
// exact bound, so the plain method never runs out of pool).
int plain_reserve(PlainWs* w, int64_t n, int64_t stage, int64_t pool) {
  int rc;
  if (n > w->cap_n) {
    const int64_t c = std::max<int64_t>(n, 2 * w->cap_n);
    dfree(w->tok_sym); dfree(w->tok_b); dfree(w->iota); dfree(w->step0); dfree(w->zero64); dfree(w->slot_base);
    dfree(w->step_rng); dfree(w->scnt); dfree(w->pool_base); dfree(w->pool_cnt); dfree(w->mkey); dfree(w->ekey);
    dfree(w->csum); dfree(w->esum); dfree(w->paths); dfree(w->olabels);
    w->cap_n = 0;
    if ((rc = dalloc(&w->iota, c)) || (rc = dalloc(&w->slot_base, c)) || (rc = dalloc(&w->step_rng, 2 * (c + 2))) ||
        (rc = dalloc(&w->step0, c + 2)))
      return rc;
    {
      std::vector<int32_t> io(c), s0(c + 2);
      for (int64_t i = 0; i < c; ++i) io[i] = (int32_t)i;
      for (int64_t t = 0; t < c + 2; ++t) s0[t] = (int32_t)std::max<int64_t>(t - 1, 0);
      FST_CUDA(cudaMemcpy(w->iota, io.data(), (size_t)c * 4, cudaMemcpyHostToDevice));
      FST_CUDA(cudaMemcpy(w->step0, s0.data(), (size_t)(c + 2) * 4, cudaMemcpyHostToDevice));
    }
    if ((rc = dalloc(&w->tok_sym, c)) || (rc = dalloc(&w->tok_b, c)) || (rc = dalloc(&w->zero64, c)) ||
        (rc = dalloc(&w->scnt, c)) || (rc = dalloc(&w->pool_base, c)) || (rc = dalloc(&w->pool_cnt, c)) ||
        (rc = dalloc(&w->mkey, c)) || (rc = dalloc(&w->ekey, c)) || (rc = dalloc(&w->csum, c)) ||
        (rc = dalloc(&w->esum, c)) || (rc = dalloc(&w->paths, c)) || (rc = dalloc(&w->olabels, c)))
      return rc;
    FST_CUDA(cudaMemset(w->tok_b, 0, (size_t)c * sizeof(int32_t)));
    FST_CUDA(cudaMemset(w->zero64, 0, (size_t)c * sizeof(int64_t)));
    w->cap_n = c;
  }
  if (stage > w->cap_stage) {
    const int64_t c = std::max<int64_t>(stage, 2 * w->cap_stage);
    dfree(w->stage);
    dfree(w->stage_b);
    w->cap_stage = 0;
    if ((rc = dalloc(&w->stage, c)) || (rc = dalloc(&w->stage_b, c))) return rc;
    w->cap_stage = c;
  }
  if (pool > w->cap_pool) {
    const int64_t c = std::max<int64_t>(pool, 2 * w->cap_pool);
    dfree(w->pool_q); dfree(w->pool_x); dfree(w->pool_n); dfree(w->pool_v);
    w->cap_pool = 0;
    if ((rc = dalloc(&w->pool_q, c)) || (rc = dalloc(&w->pool_x, c)) || (rc = dalloc(&w->pool_n, c)) ||
        (rc = dalloc(&w->pool_v, c)))
      return rc;
    w->cap_pool = c;
  }
  return FST_OK;
}

// Upload the tokens of one string and start a run.
int plain_tokens(fst_s* f, const int32_t* ids, int32_t n, cudaStream_t s) {
  PlainWs* w = f->plain;
  int64_t stage = 1, pool = 1;
  for (int32_t i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= f->m) {
      set_error("symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
      return FST_ERR_INVALID_ARG;
    }
    const int64_t D = f->fwd.h_sym_seg[ids[i] + 1] - f->fwd.h_sym_seg[ids[i]];
    stage = std::max(stage, D);
    pool += D;
  }
  int rc = plain_reserve(w, std::max(n, 1), stage, pool);
  if (rc) return rc;
  const size_t n4 = (size_t)std::max(n, 1) * 4;
  if (n > 0) FST_CUDA(cudaMemcpyAsync(w->tok_sym, ids, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  FST_CUDA(cudaMemcpyAsync(w->bw_n, &n, 4, cudaMemcpyHostToDevice, s));
  FST_CUDA(cudaMemsetAsync(w->scnt, 0, n4, s));
  FST_CUDA(cudaMemsetAsync(w->mkey, 0, n4, s));
  FST_CUDA(cudaMemsetAsync(w->ekey, 0, n4, s));
  FST_CUDA(cudaMemsetAsync(w->pool_top, 0, 8, s));
  FST_CUDA(cudaMemsetAsync(w->flags, 0, 8, s));
  return FST_OK;
}

TokenView plain_tokview(PlainWs* w) { return TokenView{w->iota, w->tok_sym, w->tok_b, w->zero64}; }

FrontierState plain_state(fst_s* f) {
  PlainWs* w = f->plain;
  FrontierState S;
  memset(&S, 0, sizeof(S));
  S.Q = f->Q;
  S.acc = w->acc;
  S.acc_stride = 2;
  S.beta = w->beta;
  S.vmap = w->vmap;
  S.src_by_id = f->src_by_id;
  S.stage = w->stage;
  S.stage_b = w->stage_b;
  S.stage_cap = w->cap_stage;
  S.Bw = 1;
  S.chain = 1;
  S.scnt = w->scnt;
  S.pool_q = w->pool_q;
  S.pool_x = w->pool_x;
  S.pool_n = w->pool_n;
  S.pool_v = (float*)w->pool_v;
  S.pool_d = w->pool_v;
  S.pool_base = w->pool_base;
  S.pool_cnt = w->pool_cnt;
  S.slot_base = w->slot_base;
  S.step_rng = w->step_rng;
  S.pool_top = w->pool_top;
  S.pool_cap = w->cap_pool;
  S.flags = w->flags;
  S.theta_s = f->theta_s;
  S.theta_f = f->theta_f;
  S.start_q = f->start_q;
  S.nstart = f->nstart;
  S.mkey = w->mkey;
  S.ekey = w->ekey;
  S.csum = w->csum;
  S.esum = w->esum;
  S.logz = w->logz;
  S.gweight = nullptr;
  S.bw_n = w->bw_n;
  S.bw_off = w->bw_off;
  return S;
}

// The single token of position t (slot t-1); x_t names the other position
// a kernel works on (the next one for the forward steps, the previous one
// for the kernels that walk the live states of t-1).
StepView plain_step(const fst_s* f, int32_t n, int32_t t, int32_t x_t) {
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
}

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
  f->batch_mu = new std::mutex();
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
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "fst_create kernels"); break; }
    if ((rc = read_err_flag(d_err, "fst_create"))) break;
    // the states with a finite start weight: the live states before the
    // first position
    {
      std::vector<float> hs(Q);
      FST_CUDA(cudaMemcpy(hs.data(), f->theta_s, (size_t)Q * 4, cudaMemcpyDeviceToHost));
      std::vector<int32_t> sq;
      for (int64_t q = 0; q < Q; ++q)
        if (hs[q] != -INFINITY) sq.push_back((int32_t)q);
      f->nstart = (int32_t)sq.size();
      if ((rc = to_device(sq.data(), &f->start_q, (int64_t)sq.size()))) break;
    }
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
  for (int k = 0; k < 2; ++k) {
    fst_plan_destroy(f->batch_plan[k]);
    f->batch_plan[k] = nullptr;
  }
  delete f->batch_mu;
  f->batch_mu = nullptr;
  delete f->pair_keys;
  f->pair_keys = nullptr;
  dfree(f->slice_arcs);
  dfree(f->slice_arcs_src);
  dfree(f->slice_keys);
  dfree(f->slice_fb);
  dfree(f->slice_out);
  dfree(f->block_ids);
  dfree(f->block_ws);
  delete f->plain;
  f->plain = nullptr;
  free_layout(f->fwd);
  free_layout(f->bwd);
  dfree(f->theta_s);
  dfree(f->theta_f);
  dfree(f->start_q);
  dfree(f->olabel);
  dfree(f->src_by_id);
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

extern "C" int fst_set_state_weights(fst_t* f, const float* start_weight, const float* final_weight,
                                     int32_t weight_kind, int32_t flags) {
  if (!f || (weight_kind != FST_WEIGHT_LOG && weight_kind != FST_WEIGHT_COST)) {
    set_error("fst_set_state_weights: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  DevGuard g(f->device);
  const int64_t Q = f->Q;
  const bool dev = (flags & FST_FLAG_DEVICE_PTRS) != 0;
  float *d_in = nullptr, *d_s = nullptr, *d_f = nullptr;
  unsigned int* d_err = nullptr;
  int rc = FST_OK;
  do {
    if ((rc = dalloc(&d_err, 1)) || (rc = dalloc(&d_s, Q)) || (rc = dalloc(&d_f, Q))) break;
    if (cudaMemset(d_err, 0, 4) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "memset"); break; }
    const float* src[2] = {start_weight, final_weight};
    float* out[2] = {d_s, d_f};
    for (int i = 0; i < 2 && !rc; ++i) {
      if (!src[i]) continue;
      const float* in = src[i];
      if (!dev) {
        dfree(d_in);
        if ((rc = to_device(src[i], &d_in, Q))) break;
        in = d_in;
      }
      k_convert_states<<<nblk(Q), TB>>>(in, f->Q, weight_kind, out[i], d_err);
    }
    if (rc) break;
    if ((rc = read_err_flag(d_err, "fst_set_state_weights"))) break;
    // validated: install the new weights and list the start states again
    if (start_weight) {
      std::vector<float> hs(Q);
      if (cudaMemcpy(hs.data(), d_s, (size_t)Q * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "start weights");
        break;
      }
      std::vector<int32_t> sq;
      for (int64_t q = 0; q < Q; ++q)
        if (hs[q] != -INFINITY) sq.push_back((int32_t)q);
      int32_t* d_sq = nullptr;
      if ((rc = to_device(sq.data(), &d_sq, (int64_t)sq.size()))) break;
      dfree(f->start_q);
      f->start_q = d_sq;
      f->nstart = (int32_t)sq.size();
      std::swap(f->theta_s, d_s);
    }
    if (final_weight) std::swap(f->theta_f, d_f);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = cuda_fail(e, "fst_set_state_weights");
  } while (0);
  dfree(d_in);
  dfree(d_s);
  dfree(d_f);
  dfree(d_err);
  return rc;
}

// ============================================================ plain method
static int fst_viterbi_frontier(fst_t* f, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path,
                                int32_t* olabels);
static bool plain_uses_slice(const fst_s* f, const int32_t* ids, int32_t n);
static bool plain_uses_block(const fst_s* f);

extern "C" int fst_viterbi(fst_t* f, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path,
                           int32_t* olabels) {
  if (!f || n < 0 || (n > 0 && (!ids || !arc_path)) || !best_score) {
    set_error("fst_viterbi: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  DevGuard g(f->device);
  if (plain_uses_block(f)) {
    for (int32_t i = 0; i < n; ++i)
      if (ids[i] < 0 || ids[i] >= f->m) {
        set_error("symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
        return FST_ERR_INVALID_ARG;
      }
    int32_t st = FST_OK;
    const int rc = viterbi_block_run(f, ids, n, best_score, arc_path, olabels, &st);
    if (rc) return rc;
    if (st != FST_OK) set_error("no accepting path");
    return st;
  }
  if (plain_uses_slice(f, ids, n)) return viterbi_slice_run(f, ids, n, best_score, arc_path, olabels);
  return fst_viterbi_frontier(f, ids, n, best_score, arc_path, olabels);
}
// Whether the single-string calls take the one-block kernels: by the
// handle's setting, or (FST_PLAIN_AUTO) once calibration chose them.
static bool plain_uses_block(const fst_s* f) {
  return f->plain_method == FST_PLAIN_BLOCK || (f->plain_method == FST_PLAIN_AUTO && f->plain_tuned && f->plain_block);
}
// Whether fst_viterbi takes the slice-wide kernel for this string: by the
// handle's setting, or (FST_PLAIN_AUTO, once calibrated) by the predicted
// times of the two kernels.
static bool plain_uses_slice(const fst_s* f, const int32_t* ids, int32_t n) {
  if (f->plain_method == FST_PLAIN_SLICE) return true;
  if (f->plain_method != FST_PLAIN_AUTO || !f->plain_tuned) return false;
  double arcs = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= f->m) return false;  // the frontier path reports the error
    arcs += (double)(f->h_sym_arc[ids[i] + 1] - f->h_sym_arc[ids[i]]);
  }
  const double* c = f->plain_coef;
  return c[2] + c[3] * n + c[4] * arcs < c[0] + c[1] * n;
}

// The frontier kernels' single-string Viterbi.
static int fst_viterbi_frontier(fst_t* f, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path,
                                int32_t* olabels) {
  int rc;
  if ((rc = plain_init(f))) return rc;
  cudaStream_t s = 0;
  if ((rc = plain_tokens(f, ids, n, s))) return rc;
  PlainWs* w = f->plain;
  const LayoutView L = view_of(f->bwd);
  const TokenView T = plain_tokview(w);
  const FrontierState S = plain_state(f);
  if (f->plain_fb_driver == FST_DRIVER_PERSISTENT && n >= 1) {
    // one cooperative launch for all positions
    const int32_t pgrid = std::max(1, std::min(f->plain_fb_grid > 0 ? f->plain_fb_grid : f->num_sms,
                                               persist_grid_limit(0)));
    FST_CUDA(cudaMemsetAsync(w->gbar, 0, 8, s));
    PLAIN_PROF(FST_PROF_VIT_STEP, launch_vit_persist(L, T, WaveSteps{w->step0, n}, S, pgrid,
                                                     GridSync{w->gbar, 0u, 2000000000ull}, s));
  } else {
    // one launch per input position (Sec. 5), after the first position's push
    if (n >= 1) PLAIN_PROF(FST_PROF_VIT_FIRST, launch_vit_first(L, T, plain_step(f, n, 1, 0), S, s));
    for (int32_t t = 1; t <= n; ++t)
      PLAIN_PROF(FST_PROF_VIT_STEP, launch_vit_step(L, T, plain_step(f, n, t, t + 1), S, s));
  }
  PLAIN_PROF(FST_PROF_VIT_FINAL, launch_vit_final(S, 1, w->score, w->jfinal, w->status, s));
  PLAIN_PROF(FST_PROF_BACKTRACE, launch_backtrace(S, f->olabel, 1, w->jfinal, w->paths, w->olabels, s));
  w->last_fb = false;
  int32_t st = 0;
  FST_CUDA(cudaMemcpy(best_score, w->score, 4, cudaMemcpyDeviceToHost));
  FST_CUDA(cudaMemcpy(&st, w->status, 4, cudaMemcpyDeviceToHost));
  if (n > 0) {
    FST_CUDA(cudaMemcpy(arc_path, w->paths, (size_t)n * 4, cudaMemcpyDeviceToHost));
    if (olabels) FST_CUDA(cudaMemcpy(olabels, w->olabels, (size_t)n * 4, cudaMemcpyDeviceToHost));
  }
  if (st == FST_ERR_TIMEOUT) {
    set_error("a grid barrier of the persistent pass timed out");
    return FST_ERR_TIMEOUT;
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
  if (plain_uses_block(f)) {
    for (int32_t i = 0; i < n; ++i)
      if (ids[i] < 0 || ids[i] >= f->m) {
        set_error("symbol %d at position %d is outside [0, %d)", ids[i], i, f->m);
        return FST_ERR_INVALID_ARG;
      }
    int32_t st = FST_OK;
    if ((rc = fb_block_run(f, ids, n, arc_posteriors, log_z, &st))) return rc;
    if (st != FST_OK) set_error("no accepting path");
    return st;
  }
  if ((rc = plain_init(f))) return rc;
  cudaStream_t s = 0;
  if ((rc = plain_tokens(f, ids, n, s))) return rc;
  PlainWs* w = f->plain;
  if (arc_posteriors && !w->cnt) {
    if ((rc = dalloc(&w->cnt, f->A)) || (rc = dalloc(&w->comp, f->A)) || (rc = dalloc(&w->counts_out, f->A)))
      return rc;
  }
  const LayoutView L = view_of(f->bwd);
  const TokenView T = plain_tokview(w);
  const FrontierState S = plain_state(f);
  // persistent driver: one cooperative launch per pass, positions separated
  // by grid barriers (the barrier words are cleared before each pass)
  const bool persist = f->plain_fb_driver == FST_DRIVER_PERSISTENT && n >= 1;
  const int32_t pgrid = std::max(1, std::min(f->plain_fb_grid > 0 ? f->plain_fb_grid : f->num_sms,
                                             std::min(persist_grid_limit(1), persist_grid_limit(2))));
  const WaveSteps D{w->step0, n};
  const GridSync G{w->gbar, 0u, 2000000000ull};
  if (persist) {
    FST_CUDA(cudaMemsetAsync(w->gbar, 0, 8, s));
    PLAIN_PROF(FST_PROF_FWD_STEP, launch_fwd_persist(L, T, D, S, pgrid, G, s));
  } else {
    if (n >= 1) PLAIN_PROF(FST_PROF_FWD_FIRST, launch_fwd_first(L, T, plain_step(f, n, 1, 0), S, s));
    for (int32_t t = 1; t <= n; ++t) {
      PLAIN_PROF(FST_PROF_FWD_SUM, launch_fwd_sum(L, T, plain_step(f, n, t, t - 1), S, PullView{}, s));
      PLAIN_PROF(FST_PROF_FWD_STEP, launch_fwd_step(L, T, plain_step(f, n, t, t + 1), S, s));
    }
  }
  PLAIN_PROF(FST_PROF_FB_FINAL, launch_fb_final(S, 1, w->logz, w->status, s));
  w->last_fb = true;
  if (arc_posteriors) {
    const CountView C{0, w->cnt, w->comp, nullptr};
    FST_CUDA(cudaMemsetAsync(w->cnt, 0, (size_t)std::max<int64_t>(f->A, 1) * 4, s));
    FST_CUDA(cudaMemsetAsync(w->comp, 0, (size_t)std::max<int64_t>(f->A, 1) * 4, s));
    if (persist) {
      FST_CUDA(cudaMemsetAsync(w->gbar, 0, 8, s));
      PLAIN_PROF(FST_PROF_BWD_STEP, launch_bwd_persist(L, T, D, S, C, pgrid, G, s));
    } else {
      for (int32_t t = n; t >= 1; --t)
        PLAIN_PROF(FST_PROF_BWD_STEP, launch_bwd_step(L, T, plain_step(f, n, t, t - 1), S, C, s));
    }
    PLAIN_PROF(FST_PROF_COUNTS, launch_counts_out(f->A, C, w->counts_out, s));
    if (f->A > 0)
      FST_CUDA(cudaMemcpy(arc_posteriors, w->counts_out, (size_t)f->A * 4, cudaMemcpyDeviceToHost));
  }
  int32_t st = 0;
  FST_CUDA(cudaMemcpy(log_z, w->logz, 8, cudaMemcpyDeviceToHost));
  FST_CUDA(cudaMemcpy(&st, w->status, 4, cudaMemcpyDeviceToHost));
  if (st == FST_ERR_TIMEOUT) {
    set_error("a grid barrier of the persistent pass timed out");
    return FST_ERR_TIMEOUT;
  }
  if (st != FST_OK) {
    set_error("no accepting path");
    return FST_ERR_NO_PATH;
  }
  return FST_OK;
}

// ============================================================ measurement
extern "C" int fst_debug_checks(int64_t* violations, int32_t* code, int64_t* index, int64_t* bound) {
  return debug_read(violations, code, index, bound);
}

extern "C" int fst_profile(fst_t* f, int32_t enable) {
  if (!f) { set_error("fst is NULL"); return FST_ERR_INVALID_ARG; }
  f->prof.on = enable != 0;
  f->prof.used = 0;
  return FST_OK;
}

extern "C" int fst_profile_read(fst_t* f, double* ms_by_kind, int64_t* launches_by_kind) {
  if (!f) { set_error("fst is NULL"); return FST_ERR_INVALID_ARG; }
  DevGuard g(f->device);
  return f->prof.read(ms_by_kind, launches_by_kind);
}

namespace {
// *sum += the non-negative values of v[0..n).
__global__ void k_sum_nonneg(const int32_t* __restrict__ v, int64_t n, unsigned long long* __restrict__ sum) {
  unsigned long long acc = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (unsigned long long)(uint32_t)max(v[i], 0);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sum, acc);
}
}  // namespace

extern "C" int fst_live_work(fst_t* f, int64_t* entries, int64_t* arcs) {
  if (!f) { set_error("fst is NULL"); return FST_ERR_INVALID_ARG; }
  DevGuard g(f->device);
  PlainWs* w = f->plain;
  if (entries) *entries = 0;
  if (arcs) *arcs = w && w->last_fb ? 0 : -1;
  if (!w) return FST_OK;
  int64_t top = 0;
  FST_CUDA(cudaMemcpy(&top, w->pool_top, 8, cudaMemcpyDeviceToHost));
  top = std::min(top, w->cap_pool);
  if (entries) *entries = top;
  if (arcs && w->last_fb && top > 0) {
    DevBuf sum;
    FST_CUDA(cudaMalloc(&sum.p, 8));
    FST_CUDA(cudaMemset(sum.p, 0, 8));
    k_sum_nonneg<<<(unsigned)std::min<int64_t>(1024, (top + TB - 1) / TB), TB>>>(w->pool_n, top,
                                                                              (unsigned long long*)sum.p);
    FST_CUDA(cudaGetLastError());
    unsigned long long h = 0;
    FST_CUDA(cudaMemcpy(&h, sum.p, 8, cudaMemcpyDeviceToHost));
    *arcs = (int64_t)h;
  }
  return FST_OK;
}

// ------------------------------------------------- plain-method calibration
extern "C" int fst_set_plain_method(fst_t* f, int32_t method) {
  if (!f || method < FST_PLAIN_FRONTIER || method > FST_PLAIN_BLOCK) {
    set_error("fst_set_plain_method: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  if (method == FST_PLAIN_BLOCK && !block_fits(f)) {
    set_error("the one-block kernels hold at most %d states (this FST has %d)", BLOCK_QMAX, f->Q);
    return FST_ERR_UNSUPPORTED;
  }
  f->plain_method = method;
  return FST_OK;
}

// Least squares y ~ X b with X of k <= 3 columns (normal equations,
// Gaussian elimination with partial pivoting); false if singular.
static bool least_squares(const std::vector<std::array<double, 3>>& X, const std::vector<double>& y, int k,
                          double* b) {
  double M[3][4] = {{0}};
  for (size_t r = 0; r < X.size(); ++r)
    for (int i = 0; i < k; ++i) {
      for (int j = 0; j < k; ++j) M[i][j] += X[r][i] * X[r][j];
      M[i][3] += X[r][i] * y[r];
    }
  for (int c = 0; c < k; ++c) {
    int piv = c;
    for (int r = c + 1; r < k; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (fabs(M[piv][c]) < 1e-30) return false;
    for (int j = 0; j < 4; ++j) std::swap(M[c][j], M[piv][j]);
    for (int r = 0; r < k; ++r) {
      if (r == c) continue;
      const double m = M[r][c] / M[c][c];
      for (int j = c; j < 4; ++j) M[r][j] -= m * M[c][j];
    }
  }
  for (int i = 0; i < k; ++i) b[i] = M[i][3] / M[i][i];
  return true;
}

extern "C" int fst_autotune_plain(fst_t* f, const int32_t* ids, const int64_t* offsets, int32_t B, double* coef) {
  if (!f || B < 1 || !offsets || (offsets[B] > 0 && !ids)) {
    set_error("fst_autotune_plain: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  for (int32_t b = 0; b < B; ++b)
    if (offsets[b + 1] < offsets[b] || offsets[b + 1] - offsets[b] >= INT32_MAX) {
      set_error("fst_autotune_plain: offsets must be non-decreasing");
      return FST_ERR_INVALID_ARG;
    }
  for (int64_t i = 0; i < offsets[B]; ++i)
    if (ids[i] < 0 || ids[i] >= f->m) { set_error("fst_autotune_plain: symbol outside [0, %d)", f->m); return FST_ERR_INVALID_ARG; }
  DevGuard g(f->device);
  std::vector<int32_t> path, olab;
  auto now = [] { return std::chrono::steady_clock::now(); };
  auto us = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
  };
  // 1. the driver of the frontier kernels (both passes): per-position
  //    launches, or persistent passes of 1, 8, 32 or one-per-SM blocks,
  //    whichever decodes the sample (Viterbi + forward-backward) fastest
  std::vector<std::pair<int32_t, int32_t>> cands = {{FST_DRIVER_LAUNCH, 0}};
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, f->device) != cudaSuccess) {
    (void)cudaGetLastError();
    coop = 0;
  }
  const int cap = std::min(persist_grid_limit(0), std::min(persist_grid_limit(1), persist_grid_limit(2)));
  if (coop && cap > 0)
    for (int32_t gsz : {1, 8, 32, f->num_sms})
      if (gsz <= cap) cands.push_back({FST_DRIVER_PERSISTENT, gsz});
  // the one-block kernels, where the FST fits, compete as one more candidate
  const bool try_block = block_fits(f);
  if (try_block) cands.push_back({-1, 0});
  f->plain_method = FST_PLAIN_FRONTIER;
  f->plain_block = false;
  double best_t = 1e300;
  std::pair<int32_t, int32_t> best = cands[0];
  for (const auto& c : cands) {
    const bool blk = c.first < 0;
    if (!blk) {
      f->plain_fb_driver = c.first;
      f->plain_fb_grid = c.second;
    }
    f->plain_method = blk ? FST_PLAIN_BLOCK : FST_PLAIN_FRONTIER;
    double tot = 0.0;
    for (int32_t b = -1; b < B; ++b) {  // b = -1: the first string again, untimed (first-use costs)
      const int32_t bb = b < 0 ? 0 : b;
      const int32_t* x = ids + offsets[bb];
      const int32_t n = (int32_t)(offsets[bb + 1] - offsets[bb]);
      path.resize(std::max(n, 1));
      olab.resize(std::max(n, 1));
      float score = 0.f;
      double lz = 0.0;
      const auto t0 = now();
      int rc = fst_viterbi(f, x, n, &score, path.data(), olab.data());
      if (rc == FST_OK || rc == FST_ERR_NO_PATH) rc = fst_forward_backward(f, x, n, &lz, nullptr);
      if (rc != FST_OK && rc != FST_ERR_NO_PATH) {
        f->plain_method = FST_PLAIN_FRONTIER;
        return rc;
      }
      if (b >= 0) tot += us(t0, now());
    }
    if (tot < best_t) {
      best_t = tot;
      best = c;
    }
  }
  f->plain_method = FST_PLAIN_FRONTIER;
  if (best.first < 0) {
    // the one-block kernels beat every frontier driver
    f->plain_block = true;
    for (int i = 0; i < 5; ++i) {
      f->plain_coef[i] = 0.0;
      if (coef) coef[i] = 0.0;
    }
    f->plain_tuned = true;
    f->plain_method = FST_PLAIN_AUTO;
    return FST_OK;
  }
  f->plain_fb_driver = best.first;
  f->plain_fb_grid = best.second;
  // 2. Viterbi: frontier (with that driver) or slice-wide, by a cost model
  std::vector<std::array<double, 3>> Xf, Xs;
  std::vector<double> yf, ys;
  for (int32_t b = -1; b < B; ++b) {
    const int32_t bb = b < 0 ? 0 : b;
    const int32_t* x = ids + offsets[bb];
    const int32_t n = (int32_t)(offsets[bb + 1] - offsets[bb]);
    path.resize(std::max(n, 1));
    olab.resize(std::max(n, 1));
    double arcs = 0.0;
    for (int32_t i = 0; i < n; ++i) arcs += (double)(f->h_sym_arc[x[i] + 1] - f->h_sym_arc[x[i]]);
    float score = 0.f;
    double t[2];
    for (int k = 0; k < 2; ++k) {
      const auto t0 = now();
      const int rc = k == 0 ? fst_viterbi_frontier(f, x, n, &score, path.data(), olab.data())
                            : viterbi_slice_run(f, x, n, &score, path.data(), olab.data());
      if (rc != FST_OK && rc != FST_ERR_NO_PATH) return rc;
      t[k] = us(t0, now());
    }
    if (b < 0) continue;
    Xf.push_back({1.0, (double)n, 0.0});
    yf.push_back(t[0]);
    Xs.push_back({1.0, (double)n, arcs});
    ys.push_back(t[1]);
  }
  double cf[2] = {0, 0}, cs[3] = {0, 0, 0};
  // a fit needs strings of several lengths and slice sizes; with fewer the
  // mean times alone decide
  std::vector<double> ns, ss;
  for (size_t i = 0; i < Xs.size(); ++i) { ns.push_back(Xs[i][1]); ss.push_back(Xs[i][2]); }
  std::sort(ns.begin(), ns.end());
  std::sort(ss.begin(), ss.end());
  const bool spread = Xs.size() >= 4 && ns.front() < ns.back() && ss.front() < ss.back();
  if (!spread || !least_squares(Xf, yf, 2, cf) || !least_squares(Xs, ys, 3, cs)) {
    double mf = 0, ms = 0;
    for (size_t i = 0; i < yf.size(); ++i) { mf += yf[i]; ms += ys[i]; }
    cf[0] = mf / yf.size(); cf[1] = 0;
    cs[0] = ms / ys.size(); cs[1] = cs[2] = 0;
  }
  const double c[5] = {cf[0], cf[1], cs[0], cs[1], cs[2]};
  for (int i = 0; i < 5; ++i) {
    f->plain_coef[i] = c[i];
    if (coef) coef[i] = c[i];
  }
  f->plain_tuned = true;
  f->plain_method = FST_PLAIN_AUTO;
  return FST_OK;
}

extern "C" int fst_get_plain_method(const fst_t* f, int32_t* method, int32_t* driver, int32_t* grid_blocks) {
  if (!f) {
    set_error("fst_get_plain_method: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  int32_t m = f->plain_method;
  if (plain_uses_block(f)) m = FST_PLAIN_BLOCK;
  else if (m == FST_PLAIN_AUTO && !f->plain_tuned) m = FST_PLAIN_FRONTIER;
  if (method) *method = m;
  if (driver) *driver = f->plain_fb_driver;
  if (grid_blocks) *grid_blocks = f->plain_fb_grid;
  return FST_OK;
}

extern "C" int fst_set_plain_driver(fst_t* f, int32_t driver, int32_t grid_blocks) {
  if (!f || (driver != FST_DRIVER_LAUNCH && driver != FST_DRIVER_PERSISTENT) || grid_blocks < 0) {
    set_error("fst_set_plain_driver: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  DevGuard g(f->device);
  if (driver == FST_DRIVER_PERSISTENT) {
    int coop = 0;
    FST_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, f->device));
    const int cap = std::min(persist_grid_limit(1), persist_grid_limit(2));
    if (!coop || cap <= 0 || grid_blocks > cap) {
      set_error("no co-resident grid of %d blocks for the persistent passes (at most %d)", grid_blocks, cap);
      return FST_ERR_UNSUPPORTED;
    }
  }
  f->plain_fb_driver = driver;
  f->plain_fb_grid = grid_blocks;
  return FST_OK;
}
