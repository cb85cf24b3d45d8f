// plan.cu -- batch plans: many strings of uneven length advanced together.
//
// The paper decodes one string at a time and launches one kernel per input
// position (Sec. 5; Sec. 7 times 100 sentences one after another).  A plan
// instead advances every string of a wave by one position per launch.  The
// work list of position t is built on the device once per plan: the tokens
// of position t are sorted by symbol and cut into groups of up to GMAX
// tokens with the same symbol, and every (group, window of the symbol's
// slice) pair is one warp-sized work item; a warp loads the window's arcs
// once and relaxes them for every token of its group.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fst_internal.cuh"
#include "kernels.cuh"

using namespace fstgpu;

namespace {

constexpr int TB = 256;
inline unsigned nblk(int64_t n, int tb = TB) { return (unsigned)std::max<int64_t>(1, (n + tb - 1) / tb); }

inline int bits_for(int64_t maxval) {
  int b = 0;
  while (b < 63 && ((int64_t)1 << b) <= maxval) ++b;
  return b;
}

__global__ void k_check_ids(const int32_t* __restrict__ ids, int64_t n, int32_t m, unsigned int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (ids[i] < 0 || ids[i] >= m)) atomicOr(err, 1u);
}

__global__ void k_tok_nseg(const int32_t* __restrict__ ids, int64_t n, const int64_t* __restrict__ sym_seg,
                           int64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sym_seg[ids[i] + 1] - sym_seg[ids[i]];
}

// one warp per string of the wave
__global__ void k_tok_info(const int32_t* __restrict__ ids, const int64_t* __restrict__ bw_off,
                           const int32_t* __restrict__ bw_n, int32_t Bw, int32_t* __restrict__ tok_sym,
                           int32_t* __restrict__ tok_b, int32_t* __restrict__ tok_t) {
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= Bw) return;
  const int64_t off = bw_off[b];
  for (int32_t i = lane; i < bw_n[b]; i += 32) {
    tok_sym[off + i] = ids[off + i];
    tok_b[off + i] = (int32_t)b;
    tok_t[off + i] = i + 1;
  }
}

__global__ void k_tok_counts(const int32_t* __restrict__ sym, int64_t n, const int64_t* __restrict__ f_seg,
                             const int64_t* __restrict__ f_lseg, const int64_t* __restrict__ f_lwin,
                             const int64_t* __restrict__ b_lseg, const int64_t* __restrict__ b_lwin,
                             const int64_t* __restrict__ f_win, int64_t* __restrict__ c0,
                             int64_t* __restrict__ c1, int64_t* __restrict__ c2, int64_t* __restrict__ c3,
                             int64_t* __restrict__ c4, int64_t* __restrict__ c5,
                             const int64_t* __restrict__ b_win, int64_t* __restrict__ c6) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t a = sym[i];
  c0[i] = f_seg[a + 1] - f_seg[a];
  c1[i] = f_lseg[a + 1] - f_lseg[a];
  c2[i] = f_lwin[a + 1] - f_lwin[a];
  c3[i] = b_lseg[a + 1] - b_lseg[a];
  c4[i] = b_lwin[a + 1] - b_lwin[a];
  c5[i] = f_win[a + 1] - f_win[a];
  c6[i] = b_win[a + 1] - b_win[a];
}

__global__ void k_tok_keys(const int32_t* __restrict__ sym, const int32_t* __restrict__ t, int64_t n, int sbits,
                           uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = ((uint64_t)(uint32_t)t[i] << sbits) | (uint64_t)(uint32_t)sym[i];
  vals[i] = (uint32_t)i;
}

__global__ void k_run_heads(const uint64_t* __restrict__ keys, int64_t n, int64_t* __restrict__ rh) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rh[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_run_first(const int64_t* __restrict__ rh, const int64_t* __restrict__ rx, int64_t n,
                            int64_t* __restrict__ run_first) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && rh[i]) run_first[rx[i]] = i;
}

// group heads: run starts and every GMAX-th token inside a run
__global__ void k_grp_heads(const int64_t* __restrict__ rh, const int64_t* __restrict__ rx,
                            const int64_t* __restrict__ run_first, int64_t n, int gmax, int64_t* __restrict__ gh) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t r = rx[i] + rh[i] - 1;
  gh[i] = ((i - run_first[r]) % gmax == 0) ? 1 : 0;
}

__global__ void k_grp_fill(const uint64_t* __restrict__ keys, const int64_t* __restrict__ gh,
                           const int64_t* __restrict__ gx, int64_t n, int sbits, int32_t* __restrict__ grp_first,
                           int32_t* __restrict__ grp_sym, int32_t* __restrict__ grp_t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !gh[i]) return;
  const int64_t g = gx[i];
  grp_first[g] = (int32_t)i;
  grp_sym[g] = (int32_t)(keys[i] & (((uint64_t)1 << sbits) - 1));
  grp_t[g] = (int32_t)(keys[i] >> sbits);
}

__global__ void k_grp_cnt_win(const int32_t* __restrict__ grp_first, const int32_t* __restrict__ grp_sym, int64_t G,
                              int64_t n, const int64_t* __restrict__ fwin, const int64_t* __restrict__ bwin,
                              int32_t* __restrict__ grp_cnt, int64_t* __restrict__ wf, int64_t* __restrict__ wb) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int64_t end = (g + 1 < G) ? grp_first[g + 1] : n;
  grp_cnt[g] = (int32_t)(end - grp_first[g]);
  const int32_t a = grp_sym[g];
  wf[g] = fwin[a + 1] - fwin[a];
  wb[g] = bwin[a + 1] - bwin[a];
}

// step_g0[t] = first group with position >= t, for t in [0, tmax+1]
__global__ void k_step_g0(const int32_t* __restrict__ grp_t, int64_t G, int32_t tmax, int32_t* __restrict__ step_g0) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t > tmax + 1) return;
  int64_t lo = 0, hi = G;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (grp_t[mid] < t) lo = mid + 1; else hi = mid;
  }
  step_g0[t] = (int32_t)lo;
}

__global__ void k_grp_item_local(const int32_t* __restrict__ grp_t, const int32_t* __restrict__ step_g0,
                                 const int64_t* __restrict__ gif, const int64_t* __restrict__ gib, int64_t G,
                                 int64_t* __restrict__ lf, int64_t* __restrict__ lb) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int32_t g0 = step_g0[grp_t[g]];
  lf[g] = gif[g] - gif[g0];
  lb[g] = gib[g] - gib[g0];
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

struct Wave {
  int32_t b0 = 0, b1 = 0, Bw = 0, tmax = 0;
  int64_t tok0 = 0, ntok = 0, store = 0, G = 0, nwins = 0, nwins_b = 0;
  int64_t nlseg = 0, nlwin = 0;  // scratch slots needed (max of both layouts)
  int32_t *tok_sym = nullptr, *tok_b = nullptr, *tok_t = nullptr;
  int64_t *cbase = nullptr, *lbase_f = nullptr, *lwbase_f = nullptr, *lbase_b = nullptr, *lwbase_b = nullptr;
  int64_t* wbase = nullptr;
  int64_t* bwbase = nullptr;
  int32_t *sorted_tok = nullptr, *grp_first = nullptr, *grp_cnt = nullptr, *grp_sym = nullptr;
  int64_t *grp_item_f = nullptr, *grp_item_b = nullptr;
  int32_t* bw_n = nullptr;
  int64_t* bw_off = nullptr;
  std::vector<int32_t> step_g0;        // [tmax + 2]
  std::vector<int64_t> items_f, items_b;  // [tmax + 1]
  void release() {
    dfree(tok_sym); dfree(tok_b); dfree(tok_t); dfree(cbase); dfree(lbase_f); dfree(lwbase_f); dfree(lbase_b);
    dfree(wbase); dfree(bwbase);
    dfree(lwbase_b); dfree(sorted_tok); dfree(grp_first); dfree(grp_cnt); dfree(grp_sym); dfree(grp_item_f);
    dfree(grp_item_b); dfree(bw_n); dfree(bw_off);
  }
};

}  // namespace

struct fst_plan_s {
  fst_t* fst = nullptr;
  int32_t B = 0, flags = 0, max_len = 0;
  int64_t N = 0, relax = 0, bytes = 0;
  std::vector<Wave> waves;
  int32_t* ids = nullptr;
  // shared per-wave buffers (sized for the largest wave)
  unsigned long long *alpha = nullptr, *beta = nullptr;
  int32_t* bp = nullptr;
  float* rc = nullptr;
  uint32_t *mkey = nullptr, *ekey = nullptr;
  double *csum = nullptr, *esum = nullptr;
  unsigned long long* skey = nullptr;
  uint32_t* scnt = nullptr;
  float2* spart = nullptr;
  int32_t* qfinal = nullptr;
  double* cnt64 = nullptr;
  double* logz = nullptr;
  uint32_t *epoch = nullptr, *clear = nullptr;
  uint32_t *abm = nullptr, *bbm = nullptr;  // [3][max_bw][W] live-state bitmaps
  uint32_t *tsum = nullptr, *bsum = nullptr;  // forward summaries per token [max_ntok][Ws]; backward [3][max_bw][Ws]
  uint8_t* wlive = nullptr;                 // per (token, forward window) liveness of the largest wave
  uint8_t *fin = nullptr, *bin = nullptr;   // window marks (forward / backward windows)
  uint8_t* bmk = nullptr;                   // backward marks (backward windows)
  int64_t max_nwins = 0, max_nwins_b = 0;
  int64_t max_bw = 0, max_ntok = 0, max_store = 0, max_lseg = 0, max_lwin = 0;
  bool forward_done = false;
  // optional per-launch CUDA events (fst_plan_profile)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_kind;
  size_t prof_used = 0;
  ~fst_plan_s() {
    for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    for (Wave& w : waves) w.release();
    dfree(ids); dfree(alpha); dfree(beta); dfree(bp); dfree(rc); dfree(mkey); dfree(ekey); dfree(csum);
    dfree(esum); dfree(skey); dfree(scnt); dfree(spart); dfree(qfinal); dfree(cnt64); dfree(logz);
    dfree(epoch); dfree(clear); dfree(abm); dfree(bbm); dfree(tsum); dfree(bsum); dfree(wlive); dfree(fin); dfree(bin); dfree(bmk);
  }
};

// Per-launch timing: an event before and after every kernel of a run.
static long prof_begin(fst_plan_s* P, int kind, cudaStream_t s) {
  if (!P->prof_on) return -1;
  const size_t i = P->prof_used;
  while (P->prof_ev.size() < 2 * (i + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    P->prof_ev.push_back(e);
  }
  if (P->prof_kind.size() < i + 1) P->prof_kind.resize(i + 1);
  P->prof_kind[i] = kind;
  cudaEventRecord(P->prof_ev[2 * i], s);
  P->prof_used = i + 1;
  return (long)i;
}
static void prof_end(fst_plan_s* P, long i, cudaStream_t s) {
  if (i >= 0) cudaEventRecord(P->prof_ev[2 * i + 1], s);
}
#define PROF(kind, call)                              \
  do {                                                \
    const long pi__ = prof_begin(P, (kind), s);       \
    const int rc__ = (call);                          \
    prof_end(P, pi__, s);                             \
    if (rc__) return rc__;                            \
  } while (0)

namespace {

template <class T>
int alloc_track(fst_plan_s* P, T** p, int64_t n) {
  int rc = dalloc(p, n);
  if (!rc) P->bytes += std::max<int64_t>(n, 1) * (int64_t)sizeof(T);
  return rc;
}

int build_wave(fst_plan_s* P, Wave& W, const std::vector<int64_t>& h_off, cudaStream_t s) {
  fst_s* f = P->fst;
  int rc;
  W.Bw = W.b1 - W.b0;
  W.tok0 = h_off[W.b0];
  W.ntok = h_off[W.b1] - W.tok0;
  std::vector<int64_t> boff(std::max(W.Bw, 1));
  std::vector<int32_t> bn(std::max(W.Bw, 1));
  W.tmax = 0;
  for (int32_t b = 0; b < W.Bw; ++b) {
    boff[b] = h_off[W.b0 + b] - W.tok0;
    bn[b] = (int32_t)(h_off[W.b0 + b + 1] - h_off[W.b0 + b]);
    W.tmax = std::max(W.tmax, bn[b]);
  }
  const int64_t n = std::max<int64_t>(W.ntok, 1);
  if ((rc = alloc_track(P, &W.bw_off, W.Bw)) || (rc = alloc_track(P, &W.bw_n, W.Bw)) ||
      (rc = alloc_track(P, &W.tok_sym, n)) || (rc = alloc_track(P, &W.tok_b, n)) ||
      (rc = alloc_track(P, &W.tok_t, n)) || (rc = alloc_track(P, &W.cbase, n + 1)) ||
      (rc = alloc_track(P, &W.lbase_f, n + 1)) || (rc = alloc_track(P, &W.lwbase_f, n + 1)) ||
      (rc = alloc_track(P, &W.lbase_b, n + 1)) || (rc = alloc_track(P, &W.lwbase_b, n + 1)) ||
      (rc = alloc_track(P, &W.wbase, n + 1)) || (rc = alloc_track(P, &W.bwbase, n + 1)) ||
      (rc = alloc_track(P, &W.sorted_tok, n)))
    return rc;
  FST_CUDA(cudaMemcpy(W.bw_off, boff.data(), (size_t)W.Bw * 8, cudaMemcpyHostToDevice));
  FST_CUDA(cudaMemcpy(W.bw_n, bn.data(), (size_t)W.Bw * 4, cudaMemcpyHostToDevice));
  if (W.Bw > 0)
    k_tok_info<<<nblk((int64_t)W.Bw * 32), TB, 0, s>>>(P->ids + W.tok0, W.bw_off, W.bw_n, W.Bw, W.tok_sym, W.tok_b,
                                                       W.tok_t);
  // per-token storage and scratch bases
  int64_t *c[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (auto& p : c)
    if ((rc = dalloc(&p, n))) { for (auto& q : c) dfree(q); return rc; }
  if (W.ntok > 0)
    k_tok_counts<<<nblk(W.ntok), TB, 0, s>>>(W.tok_sym, W.ntok, f->fwd.sym_seg, f->fwd.sym_lseg, f->fwd.sym_lwin,
                                             f->bwd.sym_lseg, f->bwd.sym_lwin, f->fwd.sym_win, c[0], c[1], c[2], c[3],
                                             c[4], c[5], f->bwd.sym_win, c[6]);
  int64_t tot[7] = {0, 0, 0, 0, 0, 0, 0};
  int64_t* outs[7] = {W.cbase, W.lbase_f, W.lwbase_f, W.lbase_b, W.lwbase_b, W.wbase, W.bwbase};
  for (int i = 0; i < 7 && !rc; ++i) rc = exclusive_scan_i64(c[i], outs[i], W.ntok, &tot[i], s);
  for (auto& q : c) dfree(q);
  if (rc) return rc;
  W.store = tot[0];
  W.nwins = tot[5];
  W.nwins_b = tot[6];
  W.nlseg = std::max(tot[1], tot[3]);
  W.nlwin = std::max(tot[2], tot[4]);
  // sort tokens by (position, symbol) and cut groups
  uint64_t* keys = nullptr;
  int64_t *rh = nullptr, *rx = nullptr, *rfirst = nullptr, *gh = nullptr, *gx = nullptr;
  int32_t* grp_t = nullptr;
  int64_t *wf = nullptr, *wb = nullptr, *gif = nullptr, *gib = nullptr;
  int32_t* d_step_g0 = nullptr;
  auto cleanup = [&]() {
    dfree(keys); dfree(rh); dfree(rx); dfree(rfirst); dfree(gh); dfree(gx); dfree(grp_t); dfree(wf); dfree(wb);
    dfree(gif); dfree(gib); dfree(d_step_g0);
  };
  do {
    const int sbits = bits_for(f->m > 1 ? f->m - 1 : 1);
    const int tbits = bits_for(W.tmax + 1);
    if ((rc = dalloc(&keys, n)) || (rc = dalloc(&rh, n)) || (rc = dalloc(&rx, n + 1)) ||
        (rc = dalloc(&rfirst, n + 1)) || (rc = dalloc(&gh, n)) || (rc = dalloc(&gx, n + 1)))
      break;
    if (W.ntok > 0) {
      k_tok_keys<<<nblk(W.ntok), TB, 0, s>>>(W.tok_sym, W.tok_t, W.ntok, sbits, keys, (uint32_t*)W.sorted_tok);
      if ((rc = radix_sort_pairs(keys, (uint32_t*)W.sorted_tok, W.ntok, sbits + tbits, s))) break;
      k_run_heads<<<nblk(W.ntok), TB, 0, s>>>(keys, W.ntok, rh);
    }
    int64_t nruns = 0;
    if ((rc = exclusive_scan_i64(rh, rx, W.ntok, &nruns, s))) break;
    if (W.ntok > 0) {
      k_run_first<<<nblk(W.ntok), TB, 0, s>>>(rh, rx, W.ntok, rfirst);
      k_grp_heads<<<nblk(W.ntok), TB, 0, s>>>(rh, rx, rfirst, W.ntok, GMAX, gh);
    }
    int64_t G = 0;
    if ((rc = exclusive_scan_i64(gh, gx, W.ntok, &G, s))) break;
    W.G = G;
    if ((rc = alloc_track(P, &W.grp_first, G)) || (rc = alloc_track(P, &W.grp_cnt, G)) ||
        (rc = alloc_track(P, &W.grp_sym, G)) || (rc = alloc_track(P, &W.grp_item_f, G)) ||
        (rc = alloc_track(P, &W.grp_item_b, G)) || (rc = dalloc(&grp_t, G)) || (rc = dalloc(&wf, G)) ||
        (rc = dalloc(&wb, G)) || (rc = dalloc(&gif, G + 1)) || (rc = dalloc(&gib, G + 1)) ||
        (rc = dalloc(&d_step_g0, (int64_t)W.tmax + 2)))
      break;
    if (W.ntok > 0) {
      k_grp_fill<<<nblk(W.ntok), TB, 0, s>>>(keys, gh, gx, W.ntok, sbits, W.grp_first, W.grp_sym, grp_t);
      k_grp_cnt_win<<<nblk(G), TB, 0, s>>>(W.grp_first, W.grp_sym, G, W.ntok, f->fwd.sym_win, f->bwd.sym_win,
                                           W.grp_cnt, wf, wb);
    }
    int64_t totf = 0, totb = 0;
    if ((rc = exclusive_scan_i64(wf, gif, G, &totf, s))) break;
    if ((rc = exclusive_scan_i64(wb, gib, G, &totb, s))) break;
    FST_CUDA(cudaMemcpy(gif + G, &totf, 8, cudaMemcpyHostToDevice));
    FST_CUDA(cudaMemcpy(gib + G, &totb, 8, cudaMemcpyHostToDevice));
    k_step_g0<<<nblk((int64_t)W.tmax + 2), TB, 0, s>>>(grp_t, G, W.tmax, d_step_g0);
    if (G > 0) k_grp_item_local<<<nblk(G), TB, 0, s>>>(grp_t, d_step_g0, gif, gib, G, W.grp_item_f, W.grp_item_b);
    FST_CUDA(cudaGetLastError());
    W.step_g0.assign(W.tmax + 2, 0);
    FST_CUDA(cudaMemcpy(W.step_g0.data(), d_step_g0, (size_t)(W.tmax + 2) * 4, cudaMemcpyDeviceToHost));
    std::vector<int64_t> hf(G + 1), hb(G + 1);
    FST_CUDA(cudaMemcpy(hf.data(), gif, (size_t)(G + 1) * 8, cudaMemcpyDeviceToHost));
    FST_CUDA(cudaMemcpy(hb.data(), gib, (size_t)(G + 1) * 8, cudaMemcpyDeviceToHost));
    W.items_f.assign(W.tmax + 1, 0);
    W.items_b.assign(W.tmax + 1, 0);
    for (int32_t t = 1; t <= W.tmax; ++t) {
      W.items_f[t] = hf[W.step_g0[t + 1]] - hf[W.step_g0[t]];
      W.items_b[t] = hb[W.step_g0[t + 1]] - hb[W.step_g0[t]];
    }
  } while (0);
  cleanup();
  return rc;
}

WaveState wave_state(fst_plan_s* P, const Wave& W, const float* gweight) {
  fst_s* f = P->fst;
  WaveState S;
  memset(&S, 0, sizeof(S));
  S.Q = f->Q;
  S.epoch = P->epoch;
  S.tok0 = (uint32_t)W.tok0;
  S.alpha = P->alpha;
  S.beta = P->beta;
  S.bp = P->bp;
  S.rc = P->rc;
  S.mkey = P->mkey;
  S.ekey = P->ekey;
  S.csum = P->csum;
  S.esum = P->esum;
  S.skey = P->skey;
  S.scnt = P->scnt;
  S.spart = P->spart;
  S.theta_s = f->theta_s;
  S.theta_f = f->theta_f;
  S.logz = P->logz + W.b0;
  S.gweight = gweight ? gweight + W.b0 : nullptr;
  S.bw_n = W.bw_n;
  S.bw_off = W.bw_off;
  S.abm = P->abm;
  S.bbm = P->bbm;
  S.bm_start = f->bm_start;
  S.bm_final = f->bm_final;
  S.W = f->W;
  S.bm_rot = P->max_bw * (int64_t)f->W;
  S.wlive = P->wlive;
  S.tsum = P->tsum;
  S.bsum = P->bsum;
  S.fin = P->fin;
  S.bin = P->bin;
  S.b_seg_state = f->bwd.seg_state;
  S.b_seg_pos = f->bwd.seg_pos;
  S.b_seg_len = f->bwd.seg_len;
  S.b_sym_seg = f->bwd.sym_seg;
  S.b_sym_win = f->bwd.sym_win;
  S.b_fwin = f->bwd.fwin;
  S.f_sym_win = f->fwd.sym_win;
  S.bmk = P->bmk;
  S.f_seg_state = f->fwd.seg_state;
  S.f_seg_pos = f->fwd.seg_pos;
  S.f_seg_len = f->fwd.seg_len;
  S.f_sym_seg = f->fwd.sym_seg;
  S.f_bwin = f->fwd.bwin;
  S.sum_start = f->sum_start;
  S.sum_final = f->sum_final;
  S.Ws = f->Ws;
  S.sum_rot = P->max_bw * (int64_t)f->Ws;
  return S;
}

// Clear rotation r of a [3][max_bw][words] bitmap (or summary) set before the
// launch that fills it.
int clear_rot(fst_plan_s* P, uint32_t* bm, int32_t r, int32_t words_per_string, cudaStream_t s) {
  const int64_t words = P->max_bw * (int64_t)words_per_string;
  FST_CUDA(cudaMemsetAsync(bm + (int64_t)r * words, 0, (size_t)std::max<int64_t>(words, 1) * 4, s));
  return FST_OK;
}

TokenView wave_tokens(const Wave& W) {
  return TokenView{W.tok_sym, W.tok_b, W.tok_t, W.cbase, W.lbase_f, W.lbase_b, W.lwbase_f, W.lwbase_b, W.wbase,
                   W.bwbase};
}

WorkView wave_work(const Wave& W, int32_t t, bool fwd) {
  WorkView V;
  memset(&V, 0, sizeof(V));
  V.single = 0;
  V.g0 = W.step_g0[t];
  V.g1 = W.step_g0[t + 1];
  V.nitems = fwd ? W.items_f[t] : W.items_b[t];
  V.grp_first = W.grp_first;
  V.grp_cnt = W.grp_cnt;
  V.grp_sym = W.grp_sym;
  V.grp_item = fwd ? W.grp_item_f : W.grp_item_b;
  V.sorted_tok = W.sorted_tok;
  return V;
}

// the launchers size step grids from the SM count and the kernel's occupancy
int step_grid(const fst_s* f, int64_t) { return f->num_sms; }

int run_begin(fst_plan_s* P, cudaStream_t s, bool fb) {
  const uint32_t span = (uint32_t)std::min<int64_t>(P->N + 1, 0x7fffffff);
  k_epoch_advance<<<1, 1, 0, s>>>(P->epoch, span, P->clear);
  const int64_t na = P->max_bw * 2 * (int64_t)P->fst->Q;
  if (P->alpha) k_clear_if<<<nblk(na), TB, 0, s>>>(P->clear, P->alpha, na);
  if (fb && P->beta) k_clear_if<<<nblk(na), TB, 0, s>>>(P->clear, P->beta, na);
  FST_CUDA(cudaMemsetAsync(P->skey, 0, (size_t)std::max<int64_t>(1, P->max_lseg) * 8, s));
  FST_CUDA(cudaMemsetAsync(P->scnt, 0, (size_t)std::max<int64_t>(1, P->max_lseg) * 4, s));
  FST_CUDA(cudaGetLastError());
  return FST_OK;
}

int run_forward_wave(fst_plan_s* P, const Wave& W, cudaStream_t s, int32_t* d_status) {
  fst_s* f = P->fst;
  int rc;
  const LayoutView Lf = view_of(f->fwd);
  const TokenView T = wave_tokens(W);
  const WaveState S = wave_state(P, W, nullptr);
  FST_CUDA(cudaMemsetAsync(P->mkey, 0, (size_t)std::max<int64_t>(1, W.ntok) * 4, s));
  FST_CUDA(cudaMemsetAsync(P->ekey, 0, (size_t)std::max<int64_t>(1, W.ntok) * 4, s));
  FST_CUDA(cudaMemsetAsync(P->wlive, 0, (size_t)std::max<int64_t>(1, W.nwins), s));
  FST_CUDA(cudaMemsetAsync(P->tsum, 0, (size_t)std::max<int64_t>(1, W.ntok * (int64_t)f->Ws) * 4, s));
  FST_CUDA(cudaMemsetAsync(P->fin, 0, (size_t)std::max<int64_t>(1, W.nwins), s));
  FST_CUDA(cudaMemsetAsync(P->bin, 0, (size_t)std::max<int64_t>(1, W.nwins_b), s));
  FST_CUDA(cudaMemsetAsync(P->bmk, 0, (size_t)std::max<int64_t>(1, W.nwins_b), s));
  for (int32_t t = 1; t <= W.tmax; ++t) {
    const WorkView V = wave_work(W, t, true);
    if ((rc = clear_rot(P, P->abm, t % 3, f->W, s))) return rc;
    PROF(FST_PROF_FWD_STEP, launch_fwd_step(Lf, T, V, S, step_grid(f, V.nitems), s));
  }
  PROF(FST_PROF_FB_FINAL, launch_fb_final(S, W.Bw, P->logz + W.b0,
                                           d_status ? d_status + W.b0 : nullptr, s));
  return FST_OK;
}

int run_backward_wave(fst_plan_s* P, const Wave& W, const float* d_weights, cudaStream_t s) {
  fst_s* f = P->fst;
  int rc;
  const LayoutView Lf = view_of(f->fwd), Lb = view_of(f->bwd);
  const TokenView T = wave_tokens(W);
  const WaveState S = wave_state(P, W, d_weights);
  const CountView C{1, nullptr, nullptr, P->cnt64};
  for (int32_t t = W.tmax; t >= 1; --t) {
    // step t also restores alpha_{t-2} of the strings longer than t - 1
    // (their buffer of that parity now holds alpha_t)
    ScatterJob J{Lf, WorkView{}, t - 1};
    if (t >= 3) J.W = wave_work(W, t - 2, true);
    const WorkView V = wave_work(W, t, false);
    if (t >= 2 && ((rc = clear_rot(P, P->bbm, (t - 1) % 3, f->W, s)) ||
                   (rc = clear_rot(P, P->bsum, (t - 1) % 3, f->Ws, s))))
      return rc;
    PROF(FST_PROF_BWD_STEP, launch_bwd_step(Lb, T, V, S, C, J, step_grid(f, std::max(V.nitems, J.W.nitems)), s));
  }
  return FST_OK;
}

inline cudaStream_t as_stream(void* p) { return (cudaStream_t)p; }

}  // namespace



extern "C" int fst_plan_create(fst_t* f, const int32_t* d_ids, const int64_t* d_offsets, int32_t B,
                               int64_t mem_budget_bytes, int32_t flags, void* stream, fst_plan_t** out) {
  if (!out) { set_error("out is NULL"); return FST_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!f || B < 0 || !d_offsets) { set_error("fst_plan_create: bad arguments"); return FST_ERR_INVALID_ARG; }
  cudaStream_t s = as_stream(stream);
  std::vector<int64_t> h_off(B + 1);
  FST_CUDA(cudaMemcpyAsync(h_off.data(), d_offsets, (size_t)(B + 1) * 8, cudaMemcpyDeviceToHost, s));
  FST_CUDA(cudaStreamSynchronize(s));
  if (h_off[0] != 0) { set_error("offsets[0] must be 0"); return FST_ERR_INVALID_ARG; }
  for (int32_t b = 0; b < B; ++b)
    if (h_off[b + 1] < h_off[b]) { set_error("offsets must be non-decreasing"); return FST_ERR_INVALID_ARG; }
  const int64_t N = h_off[B];
  if (N >= ((int64_t)1 << 31)) { set_error("too many tokens"); return FST_ERR_UNSUPPORTED; }
  if (N > 0 && !d_ids) { set_error("ids is NULL"); return FST_ERR_INVALID_ARG; }
  fst_plan_s* P = new fst_plan_s();
  P->fst = f;
  P->B = B;
  P->N = N;
  P->flags = flags;
  int rc = FST_OK;
  int64_t* tok_nseg = nullptr;
  int64_t* tok_cum = nullptr;
  unsigned int* d_err = nullptr;
  do {
    if ((rc = alloc_track(P, &P->ids, N))) break;
    if (N > 0) FST_CUDA(cudaMemcpyAsync(P->ids, d_ids, (size_t)N * 4, cudaMemcpyDeviceToDevice, s));
    if ((rc = dalloc(&d_err, 1))) break;
    if (cudaMemsetAsync(d_err, 0, 4, s) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "memset"); break; }
    if (N > 0) k_check_ids<<<nblk(N), TB, 0, s>>>(P->ids, N, f->m, d_err);
    unsigned int e = 0;
    if (cudaMemcpyAsync(&e, d_err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "id check");
      break;
    }
    if (e) { set_error("a symbol id is outside [0, %d)", f->m); rc = FST_ERR_INVALID_ARG; break; }
    // per-string storage (forward segments per token), for the wave split
    if ((rc = dalloc(&tok_nseg, std::max<int64_t>(N, 1))) || (rc = dalloc(&tok_cum, N + 1))) break;
    if (N > 0) k_tok_nseg<<<nblk(N), TB, 0, s>>>(P->ids, N, f->fwd.sym_seg, tok_nseg);
    int64_t tot = 0;
    if ((rc = exclusive_scan_i64(tok_nseg, tok_cum, N, &tot, s))) break;
    std::vector<int64_t> cum(N + 1);
    if (N > 0) FST_CUDA(cudaMemcpy(cum.data(), tok_cum, (size_t)N * 8, cudaMemcpyDeviceToHost));
    cum[N] = tot;
    // relaxations of one pass
    P->relax = 0;
    {
      std::vector<int32_t> hid(std::max<int64_t>(N, 1));
      if (N > 0) FST_CUDA(cudaMemcpy(hid.data(), P->ids, (size_t)N * 4, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < N; ++i) P->relax += f->h_sym_arc[hid[i] + 1] - f->h_sym_arc[hid[i]];
    }
    // waves: consecutive strings whose storage fits the budget
    const bool want_vit = !(flags & FST_PLAN_NO_VITERBI);
    const bool want_fb = !(flags & FST_PLAN_NO_FB);
    const int64_t budget = mem_budget_bytes > 0 ? mem_budget_bytes : ((int64_t)16 << 30);
    const int64_t per_seg = (want_vit ? 4 : 0) + (want_fb ? 4 : 0);
    const int64_t per_string = (int64_t)f->Q * 16 * (want_fb ? 2 : 1);
    int32_t b0 = 0;
    int64_t acc = 0;
    for (int32_t b = 0; b <= B; ++b) {
      const int64_t need = (b < B) ? (cum[h_off[b + 1]] - cum[h_off[b]]) * per_seg + per_string +
                                         (h_off[b + 1] - h_off[b]) * 64
                                   : 0;
      if (b == B || (b > b0 && acc + need > budget)) {
        if (b > b0 || (b == B && B == 0)) {
          Wave w;
          w.b0 = b0;
          w.b1 = b;
          P->waves.push_back(w);
        }
        b0 = b;
        acc = 0;
      }
      acc += need;
    }
    if ((flags & FST_PLAN_SINGLE_WAVE) && P->waves.size() > 1) {
      set_error("the batch needs %d waves under a budget of %lld bytes", (int)P->waves.size(),
                (long long)budget);
      rc = FST_ERR_OOM;
      break;
    }
    for (Wave& w : P->waves) {
      if ((rc = build_wave(P, w, h_off, s))) break;
      P->max_bw = std::max<int64_t>(P->max_bw, w.Bw);
      P->max_ntok = std::max<int64_t>(P->max_ntok, w.ntok);
      P->max_store = std::max<int64_t>(P->max_store, w.store);
      P->max_lseg = std::max<int64_t>(P->max_lseg, w.nlseg);
      P->max_lwin = std::max<int64_t>(P->max_lwin, w.nlwin);
      P->max_len = std::max(P->max_len, w.tmax);
      P->max_nwins = std::max(P->max_nwins, w.nwins);
      P->max_nwins_b = std::max(P->max_nwins_b, w.nwins_b);
    }
    if (rc) break;
    const int64_t na = P->max_bw * 2 * (int64_t)f->Q;
    if ((rc = alloc_track(P, &P->alpha, na))) break;
    if (want_fb && (rc = alloc_track(P, &P->beta, na))) break;
    if (want_vit && (rc = alloc_track(P, &P->bp, P->max_store))) break;
    if (want_fb && (rc = alloc_track(P, &P->rc, P->max_store))) break;
    if ((rc = alloc_track(P, &P->mkey, P->max_ntok)) || (rc = alloc_track(P, &P->ekey, P->max_ntok)) ||
        (rc = alloc_track(P, &P->csum, P->max_ntok)) || (rc = alloc_track(P, &P->esum, P->max_ntok)) ||
        (rc = alloc_track(P, &P->skey, P->max_lseg)) || (rc = alloc_track(P, &P->scnt, P->max_lseg)) ||
        (rc = alloc_track(P, &P->spart, P->max_lwin)) || (rc = alloc_track(P, &P->qfinal, P->max_bw)) ||
        (rc = alloc_track(P, &P->logz, B)) || (rc = alloc_track(P, &P->epoch, 2)) ||
        (rc = alloc_track(P, &P->clear, 1)))
      break;
    if (want_fb && (rc = alloc_track(P, &P->cnt64, f->bwd.P))) break;
    if ((rc = alloc_track(P, &P->abm, 3 * P->max_bw * (int64_t)f->W))) break;
    if ((rc = alloc_track(P, &P->tsum, P->max_ntok * (int64_t)f->Ws))) break;
    if (want_fb && (rc = alloc_track(P, &P->bbm, 3 * P->max_bw * (int64_t)f->W))) break;
    if (want_fb && (rc = alloc_track(P, &P->bsum, 3 * P->max_bw * (int64_t)f->Ws))) break;
    if (want_fb && (rc = alloc_track(P, &P->wlive, P->max_nwins))) break;
    if ((rc = alloc_track(P, &P->fin, P->max_nwins))) break;
    if (want_fb && (rc = alloc_track(P, &P->bin, P->max_nwins_b))) break;
    if (want_fb && (rc = alloc_track(P, &P->bmk, P->max_nwins_b))) break;
    FST_CUDA(cudaMemsetAsync(P->alpha, 0, (size_t)std::max<int64_t>(na, 1) * 8, s));
    if (P->beta) FST_CUDA(cudaMemsetAsync(P->beta, 0, (size_t)std::max<int64_t>(na, 1) * 8, s));
    FST_CUDA(cudaMemsetAsync(P->epoch, 0, 8, s));
    FST_CUDA(cudaMemsetAsync(P->skey, 0, (size_t)std::max<int64_t>(1, P->max_lseg) * 8, s));
    FST_CUDA(cudaMemsetAsync(P->scnt, 0, (size_t)std::max<int64_t>(1, P->max_lseg) * 4, s));
    FST_CUDA(cudaStreamSynchronize(s));
  } while (0);
  dfree(tok_nseg);
  dfree(tok_cum);
  dfree(d_err);
  if (rc) {
    delete P;
    return rc;
  }
  *out = P;
  return FST_OK;
}

extern "C" int fst_plan_destroy(fst_plan_t* P) {
  delete P;
  return FST_OK;
}

extern "C" int fst_plan_info(const fst_plan_t* P, int32_t* num_strings, int64_t* num_tokens, int32_t* num_waves,
                             int32_t* max_len, int64_t* relaxations, int64_t* viterbi_launches,
                             int64_t* fb_launches, int64_t* device_bytes) {
  if (!P) { set_error("plan is NULL"); return FST_ERR_INVALID_ARG; }
  int64_t vl = 1, fl = 1;  // epoch kernel
  for (const Wave& w : P->waves) {
    for (int32_t t = 1; t <= w.tmax; ++t) {
      vl += w.items_f[t] > 0;
      fl += (w.items_f[t] > 0) + (w.items_b[t] > 0);
      if (t < w.tmax && t >= 2) fl += w.items_f[t - 1] > 0;
    }
    vl += 2;  // final + backtrace
    fl += 1;  // final
  }
  fl += 1;  // counts out
  if (num_strings) *num_strings = P->B;
  if (num_tokens) *num_tokens = P->N;
  if (num_waves) *num_waves = (int32_t)P->waves.size();
  if (max_len) *max_len = P->max_len;
  if (relaxations) *relaxations = P->relax;
  if (viterbi_launches) *viterbi_launches = vl;
  if (fb_launches) *fb_launches = fl;
  if (device_bytes) *device_bytes = P->bytes;
  return FST_OK;
}

extern "C" int fst_plan_viterbi(fst_plan_t* P, float* d_scores, int32_t* d_paths, int32_t* d_olabels,
                                int32_t* d_status, void* stream) {
  if (!P || !d_scores || (P->N > 0 && !d_paths)) { set_error("fst_plan_viterbi: bad arguments"); return FST_ERR_INVALID_ARG; }
  if (!P->bp) { set_error("plan was created without Viterbi storage"); return FST_ERR_STATE; }
  fst_s* f = P->fst;
  cudaStream_t s = as_stream(stream);
  int rc;
  if ((rc = run_begin(P, s, false))) return rc;
  const LayoutView Lf = view_of(f->fwd);
  for (const Wave& W : P->waves) {
    const TokenView T = wave_tokens(W);
    const WaveState S = wave_state(P, W, nullptr);
    FST_CUDA(cudaMemsetAsync(P->tsum, 0, (size_t)std::max<int64_t>(1, W.ntok * (int64_t)f->Ws) * 4, s));
    FST_CUDA(cudaMemsetAsync(P->fin, 0, (size_t)std::max<int64_t>(1, W.nwins), s));
    for (int32_t t = 1; t <= W.tmax; ++t) {
      const WorkView V = wave_work(W, t, true);
      if ((rc = clear_rot(P, P->abm, t % 3, f->W, s))) return rc;
      PROF(FST_PROF_VIT_STEP, launch_vit_step(Lf, T, V, S, step_grid(f, V.nitems), s));
    }
    PROF(FST_PROF_VIT_FINAL, launch_vit_final(S, W.Bw, d_scores + W.b0, P->qfinal,
                                              d_status ? d_status + W.b0 : nullptr, s));
    PROF(FST_PROF_BACKTRACE, launch_backtrace(Lf, W.tok_sym, W.cbase, S, f->olabel, f->fwd.arc_id, W.Bw,
                                              P->qfinal, d_paths + W.tok0, d_olabels ? d_olabels + W.tok0 : nullptr,
                                              s));
  }
  return FST_OK;
}

extern "C" int fst_plan_forward(fst_plan_t* P, double* d_logz, int32_t* d_status, void* stream) {
  if (!P || !d_logz) { set_error("fst_plan_forward: bad arguments"); return FST_ERR_INVALID_ARG; }
  if (!P->rc) { set_error("plan was created without forward-backward storage"); return FST_ERR_STATE; }
  if (P->waves.size() > 1) { set_error("fst_plan_forward needs a single-wave plan"); return FST_ERR_STATE; }
  cudaStream_t s = as_stream(stream);
  int rc;
  if ((rc = run_begin(P, s, true))) return rc;
  for (const Wave& W : P->waves)
    if ((rc = run_forward_wave(P, W, s, d_status))) return rc;
  if (P->B > 0) FST_CUDA(cudaMemcpyAsync(d_logz, P->logz, (size_t)P->B * 8, cudaMemcpyDeviceToDevice, s));
  P->forward_done = true;
  return FST_OK;
}

extern "C" int fst_plan_backward(fst_plan_t* P, const float* d_weights, float* d_counts, void* stream) {
  if (!P || !d_counts) { set_error("fst_plan_backward: bad arguments"); return FST_ERR_INVALID_ARG; }
  if (!P->forward_done) { set_error("fst_plan_backward before fst_plan_forward"); return FST_ERR_STATE; }
  fst_s* f = P->fst;
  cudaStream_t s = as_stream(stream);
  int rc;
  FST_CUDA(cudaMemsetAsync(P->cnt64, 0, (size_t)std::max<int64_t>(1, f->bwd.P) * 8, s));
  for (const Wave& W : P->waves)
    if ((rc = run_backward_wave(P, W, d_weights, s))) return rc;
  const CountView C{1, nullptr, nullptr, P->cnt64};
  PROF(FST_PROF_COUNTS, launch_counts_out(f->bwd.arc_id, f->bwd.P, C, d_counts, s));
  return FST_OK;
}

extern "C" int fst_plan_forward_backward(fst_plan_t* P, const float* d_weights, double* d_logz, float* d_counts,
                                         int32_t* d_status, void* stream) {
  if (!P || !d_logz) { set_error("fst_plan_forward_backward: bad arguments"); return FST_ERR_INVALID_ARG; }
  if (!P->rc) { set_error("plan was created without forward-backward storage"); return FST_ERR_STATE; }
  fst_s* f = P->fst;
  cudaStream_t s = as_stream(stream);
  int rc;
  if ((rc = run_begin(P, s, true))) return rc;
  if (d_counts) FST_CUDA(cudaMemsetAsync(P->cnt64, 0, (size_t)std::max<int64_t>(1, f->bwd.P) * 8, s));
  for (const Wave& W : P->waves) {
    if ((rc = run_forward_wave(P, W, s, d_status))) return rc;
    if (d_counts && (rc = run_backward_wave(P, W, d_weights, s))) return rc;
  }
  if (P->B > 0) FST_CUDA(cudaMemcpyAsync(d_logz, P->logz, (size_t)P->B * 8, cudaMemcpyDeviceToDevice, s));
  if (d_counts) {
    const CountView C{1, nullptr, nullptr, P->cnt64};
    PROF(FST_PROF_COUNTS, launch_counts_out(f->bwd.arc_id, f->bwd.P, C, d_counts, s));
  }
  P->forward_done = P->waves.size() <= 1;
  return FST_OK;
}

extern "C" int fst_viterbi_batch(fst_t* f, const int32_t* d_ids, const int64_t* d_offsets, int32_t B,
                                 float* d_scores, int32_t* d_paths, int32_t* d_olabels, int32_t* d_status,
                                 void* stream) {
  fst_plan_t* P = nullptr;
  int rc = fst_plan_create(f, d_ids, d_offsets, B, 0, FST_PLAN_NO_FB, stream, &P);
  if (rc) return rc;
  rc = fst_plan_viterbi(P, d_scores, d_paths, d_olabels, d_status, stream);
  cudaError_t e = cudaStreamSynchronize(as_stream(stream));
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "fst_viterbi_batch");
  fst_plan_destroy(P);
  return rc;
}

extern "C" int fst_forward_backward_batch(fst_t* f, const int32_t* d_ids, const int64_t* d_offsets, int32_t B,
                                          const float* d_weights, double* d_logz, float* d_counts,
                                          int32_t* d_status, void* stream) {
  fst_plan_t* P = nullptr;
  int rc = fst_plan_create(f, d_ids, d_offsets, B, 0, FST_PLAN_NO_VITERBI, stream, &P);
  if (rc) return rc;
  rc = fst_plan_forward_backward(P, d_weights, d_logz, d_counts, d_status, stream);
  cudaError_t e = cudaStreamSynchronize(as_stream(stream));
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "fst_forward_backward_batch");
  fst_plan_destroy(P);
  return rc;
}

extern "C" int fst_plan_profile(fst_plan_t* P, int32_t enable) {
  if (!P) { set_error("plan is NULL"); return FST_ERR_INVALID_ARG; }
  P->prof_on = enable != 0;
  P->prof_used = 0;
  return FST_OK;
}

extern "C" int fst_plan_profile_read(fst_plan_t* P, double* ms_by_kind, int64_t* launches_by_kind) {
  if (!P) { set_error("plan is NULL"); return FST_ERR_INVALID_ARG; }
  double ms[FST_PROF_KINDS] = {0};
  int64_t cnt[FST_PROF_KINDS] = {0};
  if (P->prof_used > 0) FST_CUDA(cudaEventSynchronize(P->prof_ev[2 * (P->prof_used - 1) + 1]));
  for (size_t i = 0; i < P->prof_used; ++i) {
    float t = 0.f;
    FST_CUDA(cudaEventElapsedTime(&t, P->prof_ev[2 * i], P->prof_ev[2 * i + 1]));
    const int k = P->prof_kind[i];
    if (k >= 0 && k < FST_PROF_KINDS) {
      ms[k] += t;
      cnt[k] += 1;
    }
  }
  P->prof_used = 0;
  for (int k = 0; k < FST_PROF_KINDS; ++k) {
    if (ms_by_kind) ms_by_kind[k] = ms[k];
    if (launches_by_kind) launches_by_kind[k] = cnt[k];
  }
  return FST_OK;
}
