// plan.cu -- batch plans: many strings of uneven length advanced together.
//
// The paper decodes one string at a time and launches one kernel per input
// position (Sec. 5; Sec. 7 times 100 sentences one after another).  A plan
// instead advances every string of a wave by one position per launch
// (kernels.cu): the tokens of position t are all the strings' t-th symbols,
// listed once per plan.  The plan also fixes, per token, where its staged
// destinations go inside the step's staging buffer, and holds the dense
// accumulators, the live pool and the per-token scalars.  Strings are split
// into waves whose memory fits a budget.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "fst_internal.cuh"
#include "kernels.cuh"

using namespace fstgpu;

namespace {

constexpr int TB = 256;

// live-pool entries reserved per token (the pool never exceeds the sum of
// the tokens' destination-segment counts, its exact bound)
constexpr int64_t POOL_PER_TOKEN = 256;
// approximate device bytes per token of a wave (token tables, staging
// counts, pool ranges, step maxima and running sums)
constexpr int64_t TOKEN_BYTES = 80;
// compact accumulators: the live states of one position that the tables
// are sized for, 128 per token of the busiest position and at least 2^18
// (one string's frontier can span most of a 200,000-state FST), never more
// than the position's destination bound
constexpr int64_t LIVE_PER_TOKEN = 128;
constexpr int64_t LIVE_FLOOR = (int64_t)1 << 18;
// internal plan flag: a part of a plan of several parts (the parent owns
// the count accumulators)
constexpr int32_t PLAN_PART = 1 << 16;

// *sum += the non-negative values of v[0..n).
__global__ void k_sum_i32(const int32_t* __restrict__ v, int64_t n, unsigned long long* __restrict__ sum) {
  unsigned long long acc = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (unsigned long long)(uint32_t)max(v[i], 0);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sum, acc);
}

struct Wave {
  int32_t b0 = 0, b1 = 0, Bw = 0, tmax = 0;
  int64_t tok0 = 0, ntok = 0;
  int64_t stage = 0;       // staging entries the largest step needs
  int64_t pool_bound = 0;  // sum of the tokens' destination counts
  int32_t *tok_sym = nullptr, *tok_b = nullptr, *step_tok = nullptr;
  int64_t* stf = nullptr;
  int32_t* bw_n = nullptr;
  int64_t* bw_off = nullptr;
  std::vector<int32_t> step0;  // [tmax + 2]: tokens of position t are step_tok[step0[t] .. step0[t+1])
  int32_t* d_step0 = nullptr;  // the same on the device (persistent passes)
  int32_t grid_est = 1;        // blocks of the busiest position (about 64 live states per token)
  // the device arrays above point into the plan's token arena
  void release() {}
};

// Host copies of a wave's token tables, uploaded into the token arena.
struct HostWave {
  std::vector<int32_t> sym, tb, step_tok, bn;
  std::vector<int64_t> stf, boff;
};

}  // namespace

// The storage budget of a plan created with none: a quarter of the device
// memory free now, at most 32 GiB and at least 256 MiB.
int64_t default_budget() {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    (void)cudaGetLastError();
    free_b = 0;
  }
  return std::max<int64_t>((int64_t)256 << 20, std::min<int64_t>((int64_t)32 << 30, (int64_t)(free_b / 4)));
}

// Dense accumulator bytes per string of a plan (forward-backward and/or
// Viterbi), and the other per-string and per-token storage.
int64_t dense_bytes_per_string(const fst_s* f, bool fb, bool vit) {
  return (int64_t)f->Q * ((fb ? 48 : 16) + (vit ? 8 : 0));
}

// The device storage of a plan (everything but the per-wave token tables).
#define PLAN_STORAGE(X)                                                                                          \
  X(acc) X(beta) X(vmap) X(stage) X(stage_b) X(scnt) X(pool_q) X(pool_x) X(pool_n) X(pool_v) X(pool_base)          \
  X(pool_cnt) X(slot_base) X(step_rng) X(pool_top) X(flags_d) X(mkey) X(ekey) X(csum) X(esum) X(jfinal) X(logz) \
  X(cnt64) X(start64) X(final64) X(gbar) X(htab) X(bslot) X(tok_arena) X(dvec) X(dslot) X(dlist) X(dcnt)

struct fst_plan_s {
  fst_t* fst = nullptr;
  int32_t B = 0, flags = 0, max_len = 0;
  int64_t N = 0, relax = 0, bytes = 0;
  std::vector<Wave> waves;
  bool want_vit = true, want_fb = true;
  // shared per-wave buffers (sized for the largest wave)
  unsigned long long* acc = nullptr;  // [max_bw][2][Q] x acc_stride words
  int32_t acc_stride = 1;
  double* beta = nullptr;
  int32_t* vmap = nullptr;
  // compact accumulators (the default; FST_PLAN_DENSE_ACC: the dense arrays
  // above): the two parity tables, then (forward-backward) the three
  // backward-value tables, cap_hslots slots each, in one allocation
  bool compact = true;
  bool chain = true;  // launch the step kernels chained (set per part by its parent)
  int64_t hslots = 0;                  // slots this plan's busiest position needs
  int64_t table_limit = 0;             // fst_plan_limit_table: slots a run may use (0 = cap_hslots)
  unsigned long long* htab = nullptr;
  int32_t* bslot = nullptr;            // [pool_cap]
  // every wave's token tables, one allocation (cap_tok bytes)
  unsigned char* tok_arena = nullptr;
  int64_t cap_tok = 0;
  // direction switch of the forward pass (dense accumulators, launch
  // driver): dense value vectors and the dense tokens of each position
  double* dvec = nullptr;      // [DENSE_SLOTS][2][Q], -inf between uses
  int32_t* dslot = nullptr;    // [cap_nt]
  int32_t* dlist = nullptr;    // [cap_len + 2][DENSE_SLOTS]
  int32_t* dcnt = nullptr;     // [cap_len + 2]
  int64_t pull_min = 0;        // fst_plan_set_pull: 0 off (the default), -1 pull_default, else the threshold
  int32_t *stage = nullptr, *stage_b = nullptr;
  uint32_t* scnt = nullptr;
  int32_t *pool_q = nullptr, *pool_x = nullptr, *pool_n = nullptr;
  double* pool_v = nullptr;  // Viterbi scores (float32) or forward values (float64)
  int64_t* pool_base = nullptr;
  int32_t* pool_cnt = nullptr;
  int64_t *slot_base = nullptr, *step_rng = nullptr;
  int64_t* pool_top = nullptr;
  int64_t pool_cap = 0;
  int64_t pool_limit = 0;  // fst_plan_limit_pool: entries a run may use (0 = pool_cap)
  uint32_t* flags_d = nullptr;
  uint32_t *mkey = nullptr, *ekey = nullptr;
  double *csum = nullptr, *esum = nullptr;
  int32_t* jfinal = nullptr;
  double* cnt64 = nullptr;
  double *start64 = nullptr, *final64 = nullptr;  // [Q] expected start and final states
  double* logz = nullptr;
  int64_t max_bw = 0, max_ntok = 0, max_stage = 0;
  // capacities of the device storage below: this plan's needs, or more when
  // the storage was taken over from an earlier plan of the same handle
  int64_t cap_bw = 0, cap_nt = 0, cap_stage = 0, cap_len = 0, cap_B = 0, store_bytes = 0, cap_hslots = 0;
  bool forward_done = false;
  // optional per-launch CUDA events (fst_plan_profile)
  LaunchProfile prof;
  // driver: one launch per position, or one persistent launch per pass
  int32_t driver = FST_DRIVER_LAUNCH;
  int32_t persist_grid = 0;          // 0: the plan's estimate, capped at what is co-resident
  int32_t density = 64;              // launch driver: live states per token assumed when sizing a grid
  // launch driver, single-wave plans: the live states of every position
  // read back after a completed run (pool ranges), which size the grids of
  // the later runs' launches instead of the density estimate
  std::vector<int64_t> live;
  bool learned = false, ran = false;
  cudaEvent_t run_event = nullptr;   // recorded at the end of each run outside a graph capture
  uint64_t barrier_limit_ns = 2000000000ull;
  uint32_t barrier_extra = 0;        // fault injection: blocks a barrier waits for beyond the grid
  uint32_t* gbar = nullptr;          // [2] grid barrier (arrivals, generation)
  // stream-parallel parts (FST_PLAN_PARTS): sub-plans over contiguous string
  // ranges, each run on its own stream; the plan itself then holds only the
  // count accumulators that the parts share
  std::vector<fst_plan_s*> parts;
  std::vector<int32_t> part_b0;
  std::vector<int64_t> part_tok0;
  std::vector<cudaStream_t> part_stream;
  std::vector<cudaEvent_t> part_event;  // [0] fork, [1 + i] the end of part i
  bool borrowed_counts = false;         // a part: cnt64 / start64 / final64 belong to the parent
  ~fst_plan_s() {
    for (fst_plan_s* q : parts) delete q;
    for (cudaStream_t st : part_stream) cudaStreamDestroy(st);
    for (cudaEvent_t e : part_event) cudaEventDestroy(e);
    if (run_event) cudaEventDestroy(run_event);
    if (borrowed_counts) cnt64 = start64 = final64 = nullptr;
    for (Wave& w : waves) w.release();
#define PLAN_FREE(x) dfree(x);
    PLAN_STORAGE(PLAN_FREE)
#undef PLAN_FREE
  }
};

#define PROF(kind, call)                              \
  do {                                                \
    const long pi__ = P->prof.begin((kind), s);       \
    const int rc__ = (call);                          \
    P->prof.end(pi__, s);                             \
    if (rc__) return rc__;                            \
  } while (0)

namespace {

template <class T>
int alloc_track(fst_plan_s* P, T** p, int64_t n) {
  int rc = dalloc(p, n);
  if (!rc) P->bytes += std::max<int64_t>(n, 1) * (int64_t)sizeof(T);
  return rc;
}

template <class T>
int alloc_store(fst_plan_s* P, T** p, int64_t n) {
  int rc = dalloc(p, n);
  if (!rc) {
    const int64_t by = std::max<int64_t>(n, 1) * (int64_t)sizeof(T);
    P->bytes += by;
    P->store_bytes += by;
  }
  return rc;
}

// Token tables of one wave, built on the host from the offsets and symbols.
// Tokens of a string are consecutive (token p = position t of string b is
// p = off_b + t - 1); the tokens of position t are listed string by string.
int build_wave(fst_plan_s* P, Wave& W, const int64_t* h_off, const int32_t* hid, HostWave& H) {
  fst_s* f = P->fst;
  W.Bw = W.b1 - W.b0;
  W.tok0 = h_off[W.b0];
  W.ntok = h_off[W.b1] - W.tok0;
  std::vector<int64_t> boff(W.Bw);
  std::vector<int32_t> bn(W.Bw);
  W.tmax = 0;
  for (int32_t b = 0; b < W.Bw; ++b) {
    boff[b] = h_off[W.b0 + b] - W.tok0;
    bn[b] = (int32_t)(h_off[W.b0 + b + 1] - h_off[W.b0 + b]);
    W.tmax = std::max(W.tmax, bn[b]);
  }
  std::vector<int32_t> sym(W.ntok), tb(W.ntok), step_tok;
  std::vector<int64_t> stf(W.ntok);
  step_tok.reserve(W.ntok);
  for (int32_t b = 0; b < W.Bw; ++b)
    for (int32_t i = 0; i < bn[b]; ++i) {
      sym[boff[b] + i] = hid[W.tok0 + boff[b] + i];
      tb[boff[b] + i] = b;
    }
  // strings sorted by length (descending) so that the tokens of position t
  // are a prefix of that order: string b has a token at t iff n_b >= t
  std::vector<int32_t> order(W.Bw);
  for (int32_t b = 0; b < W.Bw; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return bn[x] > bn[y]; });
  W.step0.assign(W.tmax + 2, 0);
  W.stage = 0;
  W.pool_bound = 0;
  int32_t live = W.Bw;
  for (int32_t t = 1; t <= W.tmax; ++t) {
    while (live > 0 && bn[order[live - 1]] < t) --live;
    W.step0[t] = (int32_t)step_tok.size();
    int64_t accf = 0;
    for (int32_t j = 0; j < live; ++j) {
      const int64_t p = boff[order[j]] + t - 1;
      const int32_t a = sym[p];
      step_tok.push_back((int32_t)p);
      stf[p] = accf;
      // distinct destinations of the symbol's arcs: the most a token can stage
      const int64_t D = f->fwd.h_sym_seg[a + 1] - f->fwd.h_sym_seg[a];
      accf += D;
      W.pool_bound += D;
    }
    W.stage = std::max(W.stage, accf);
  }
  W.step0[W.tmax + 1] = (int32_t)step_tok.size();
  int64_t busiest = 1;
  for (int32_t t = 1; t <= W.tmax; ++t) busiest = std::max<int64_t>(busiest, W.step0[t + 1] - W.step0[t]);
  W.grid_est = (int32_t)std::min<int64_t>((int64_t)f->num_sms * 8, (busiest * 64 + 255) / 256);
  H.sym = std::move(sym);
  H.tb = std::move(tb);
  H.step_tok = std::move(step_tok);
  H.bn = std::move(bn);
  H.stf = std::move(stf);
  H.boff = std::move(boff);
  return FST_OK;
}

// The suggested threshold of the direction switch (fst_plan_set_pull(-1)):
// half the states, at least 2,048.  A pull reads the whole slice; below
// about half the states live the pushes touch so much less of it that they
// win.
int32_t pull_default(const fst_s* f) { return std::max<int32_t>(2048, f->Q / 2); }

// The waves' token tables in the plan's token arena (grown when the one
// taken over from a donor is too small), uploaded with one copy.
int upload_tokens(fst_plan_s* P, std::vector<HostWave>& hw, cudaStream_t s) {
  auto up16 = [](int64_t b) { return (b + 15) & ~(int64_t)15; };
  int64_t total = 0;
  for (size_t i = 0; i < P->waves.size(); ++i) {
    const Wave& W = P->waves[i];
    total += up16(8 * (int64_t)W.Bw) + up16(4 * (int64_t)W.Bw) + up16(4 * W.ntok) * 3 + up16(8 * W.ntok) +
             up16(4 * ((int64_t)W.tmax + 2));
  }
  total = std::max<int64_t>(total, 16);
  if (total > P->cap_tok) {
    dfree(P->tok_arena);
    P->cap_tok = 0;
    int rc = dalloc(&P->tok_arena, total);
    if (rc) return rc;
    P->cap_tok = total;
    P->store_bytes += total;
    P->bytes += total;
  }
  std::vector<unsigned char> h((size_t)total);
  int64_t at = 0;
  auto put = [&](auto** dptr, const void* src, int64_t bytes) {
    *dptr = (std::remove_pointer_t<decltype(dptr)>)(P->tok_arena + at);
    if (bytes > 0) memcpy(h.data() + at, src, (size_t)bytes);
    at += up16(bytes);
  };
  for (size_t i = 0; i < P->waves.size(); ++i) {
    Wave& W = P->waves[i];
    HostWave& H = hw[i];
    put(&W.bw_off, H.boff.data(), 8 * (int64_t)W.Bw);
    put(&W.bw_n, H.bn.data(), 4 * (int64_t)W.Bw);
    put(&W.tok_sym, H.sym.data(), 4 * W.ntok);
    put(&W.tok_b, H.tb.data(), 4 * W.ntok);
    put(&W.step_tok, H.step_tok.data(), 4 * W.ntok);
    put(&W.stf, H.stf.data(), 8 * W.ntok);
    put(&W.d_step0, W.step0.data(), 4 * ((int64_t)W.tmax + 2));
  }
  FST_CUDA(cudaMemcpyAsync(P->tok_arena, h.data(), (size_t)at, cudaMemcpyHostToDevice, s));
  FST_CUDA(cudaStreamSynchronize(s));
  return FST_OK;
}

FrontierState wave_state(fst_plan_s* P, const Wave& W, const float* gweight) {
  fst_s* f = P->fst;
  FrontierState S;
  memset(&S, 0, sizeof(S));
  S.Q = f->Q;
  S.acc = P->acc;
  S.acc_stride = P->acc_stride;
  S.beta = P->beta;
  S.vmap = P->vmap;
  if (P->dvec && P->driver == FST_DRIVER_LAUNCH && P->pull_min != 0) {
    S.dvec = P->dvec;
    S.dslot = P->dslot;
    S.dlist = P->dlist;
    S.dcnt = P->dcnt;
    S.pull_lseg = P->fst->fwd.sym_lseg;
    S.dense_min = (int32_t)(P->pull_min > 0 ? std::min<int64_t>(P->pull_min, INT32_MAX) : pull_default(P->fst));
  }
  if (P->compact) {
    const int64_t n = P->cap_hslots, hw = 2 * (int64_t)P->acc_stride;
    S.htab0 = P->htab;
    S.htab1 = P->htab + n * hw;
    if (P->want_fb) {
      S.btab0 = P->htab + 2 * n * hw;
      S.btab1 = S.btab0 + 2 * n;
      S.btab2 = S.btab0 + 4 * n;
    }
    S.bslot = P->bslot;
    // a limit uses the first slots of each table (a power of two)
    int64_t use = n;
    if (P->table_limit > 0)
      while (use > 2 && use / 2 >= P->table_limit) use /= 2;  // at least 2: a mask of 0 means dense
    S.hmask = (uint64_t)(use - 1);
  }
  S.src_by_id = f->src_by_id;
  S.stage = P->stage;
  S.stage_b = P->stage_b;
  S.stage_cap = P->cap_stage;
  S.Bw = (int32_t)P->cap_bw;
  S.chain = P->chain;
  S.scnt = P->scnt;
  S.pool_q = P->pool_q;
  S.pool_x = P->pool_x;
  S.pool_n = P->pool_n;
  S.pool_v = (float*)P->pool_v;
  S.pool_d = P->pool_v;
  S.pool_base = P->pool_base;
  S.pool_cnt = P->pool_cnt;
  S.slot_base = P->slot_base;
  S.step_rng = P->step_rng;
  S.pool_top = P->pool_top;
  S.pool_cap = P->pool_limit > 0 ? std::min(P->pool_limit, P->pool_cap) : P->pool_cap;
  S.flags = P->flags_d;
  S.theta_s = f->theta_s;
  S.theta_f = f->theta_f;
  S.start_q = f->start_q;
  S.nstart = f->nstart;
  S.mkey = P->mkey;
  S.ekey = P->ekey;
  S.csum = P->csum;
  S.esum = P->esum;
  S.logz = P->logz + W.b0;
  S.gweight = gweight ? gweight + W.b0 : nullptr;
  S.bw_n = W.bw_n;
  S.bw_off = W.bw_off;
  return S;
}

TokenView wave_tokens(const Wave& W) { return TokenView{W.step_tok, W.tok_sym, W.tok_b, W.stf}; }

// Position t of a wave; x names position x_t (the next position for the
// forward steps, the previous one for the kernels that walk the live states
// of t-1).  The grid assumes about 64 live states per token and is capped at
// what is resident at once.
StepView wave_step(const fst_plan_s* P, const Wave& W, int32_t t, int32_t x_t) {
  StepView V;
  V.t = t;
  V.slot0 = W.step0[t];
  V.n = W.step0[t + 1] - W.step0[t];
  const bool hasx = x_t >= 1 && x_t <= W.tmax;
  V.x_t = hasx ? x_t : 0;
  V.x_slot0 = hasx ? W.step0[x_t] : 0;
  V.x_n = hasx ? W.step0[x_t + 1] - W.step0[x_t] : 0;
  int64_t est = (int64_t)std::max(V.n, V.x_n) * P->density;
  if (P->learned) {
    // the live states the launch walks: those of t-1 for the sums and the
    // backward steps, those of t for the forward steps
    const int32_t u = (x_t == t - 1) ? t - 1 : t;
    est = (u >= 1 && u < (int32_t)P->live.size()) ? P->live[u] : est;
  }
  V.blocks = (int32_t)std::min<int64_t>((int64_t)P->fst->num_sms * 8, std::max<int64_t>(1, (est + 255) / 256));
  V.y_t = 0;
  return V;
}

// Learn the live states of every position from the last completed run (a
// single-wave plan, outside a graph capture); no waiting: a run still in
// flight leaves the estimate in place until a later call.
void plan_learn(fst_plan_s* P, cudaStream_t s) {
  if (P->learned || !P->ran || P->waves.size() != 1 || !P->run_event) return;
  // nothing that would break a graph capture of this run
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    (void)cudaGetLastError();
    return;
  }
  if (cudaEventQuery(P->run_event) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  const Wave& W = P->waves[0];
  std::vector<int64_t> rng(2 * ((size_t)W.tmax + 2));
  if (cudaMemcpyAsync(rng.data(), P->step_rng, rng.size() * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  P->live.assign((size_t)W.tmax + 2, 0);
  for (int32_t t = 1; t <= W.tmax; ++t) P->live[t] = std::max<int64_t>(0, rng[2 * t + 1] - rng[2 * t]);
  P->learned = true;
}

// A run ended: mark it, outside a graph capture, for plan_learn.
void plan_ran(fst_plan_s* P, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    (void)cudaGetLastError();
    return;
  }
  if (!P->run_event && cudaEventCreateWithFlags(&P->run_event, cudaEventDisableTiming) != cudaSuccess) {
    (void)cudaGetLastError();
    P->run_event = nullptr;
    return;
  }
  if (cudaEventRecord(P->run_event, s) == cudaSuccess) P->ran = true;
  else (void)cudaGetLastError();
}

// State that starts every pass of a wave at zero.  A pass whose pool
// overflowed left staged accumulators behind: they are cleared first.
int64_t htab_words(const fst_plan_s* P, int64_t slots) {
  return slots * (2 * 2 * (int64_t)P->acc_stride + (P->want_fb ? 3 * 2 : 0));
}

int wave_begin(fst_plan_s* P, const Wave& W, cudaStream_t s, bool fb) {
  int rc;
  if (P->compact) {
    rc = launch_clear_if_overflow(P->flags_d + 1, P->htab, htab_words(P, P->cap_hslots), P->fst->num_sms, s);
  } else {
    const int64_t na = P->cap_bw * 2 * (int64_t)P->fst->Q * P->acc_stride;
    rc = launch_clear_if_overflow(P->flags_d + 1, P->acc, na, P->fst->num_sms, s);
  }
  if (rc) return rc;
  const size_t n4 = (size_t)std::max<int64_t>(1, W.ntok) * 4;
  FST_CUDA(cudaMemsetAsync(P->scnt, 0, n4, s));
  FST_CUDA(cudaMemsetAsync(P->pool_top, 0, 8, s));
  FST_CUDA(cudaMemsetAsync(P->flags_d, 0, 8, s));
  if (P->driver == FST_DRIVER_PERSISTENT) FST_CUDA(cudaMemsetAsync(P->gbar, 0, 8, s));
  if (fb) {
    FST_CUDA(cudaMemsetAsync(P->mkey, 0, n4, s));
    FST_CUDA(cudaMemsetAsync(P->ekey, 0, n4, s));
  }
  return FST_OK;
}

// The persistent grid of a pass: the plan's setting or its estimate, capped
// at what can be co-resident.
int32_t persist_grid(const fst_plan_s* P, const Wave& W, int which) {
  const int cap = persist_grid_limit(which);
  const int32_t want = P->persist_grid > 0 ? P->persist_grid : W.grid_est;
  return std::max(1, std::min(want, cap));
}
GridSync grid_sync_of(const fst_plan_s* P) { return GridSync{P->gbar, P->barrier_extra, P->barrier_limit_ns}; }
WaveSteps wave_steps(const Wave& W) { return WaveSteps{W.d_step0, W.tmax}; }

int run_viterbi_wave(fst_plan_s* P, const Wave& W, float* d_scores, int32_t* d_paths, int32_t* d_olabels,
                     int32_t* d_status, cudaStream_t s) {
  fst_s* f = P->fst;
  int rc;
  plan_learn(P, s);
  const LayoutView L = view_of(f->bwd);
  const TokenView T = wave_tokens(W);
  const FrontierState S = wave_state(P, W, nullptr);
  if ((rc = wave_begin(P, W, s, false))) return rc;
  if (P->driver == FST_DRIVER_PERSISTENT) {
    PROF(FST_PROF_VIT_STEP, launch_vit_persist(L, T, wave_steps(W), S, persist_grid(P, W, 0), grid_sync_of(P), s));
  } else {
    if (W.tmax >= 1) PROF(FST_PROF_VIT_FIRST, launch_vit_first(L, T, wave_step(P, W, 1, 0), S, s));
    for (int32_t t = 1; t <= W.tmax; ++t)
      PROF(FST_PROF_VIT_STEP, launch_vit_step(L, T, wave_step(P, W, t, t + 1), S, s));
  }
  PROF(FST_PROF_VIT_FINAL,
       launch_vit_final(S, W.Bw, d_scores + W.b0, P->jfinal, d_status ? d_status + W.b0 : nullptr, s));
  PROF(FST_PROF_BACKTRACE, launch_backtrace(S, f->olabel, W.Bw, P->jfinal, d_paths + W.tok0,
                                            d_olabels ? d_olabels + W.tok0 : nullptr, s));
  plan_ran(P, s);
  return FST_OK;
}

// The destination-ordered slices of the direction switch.
PullView pull_view(const fst_plan_s* P) {
  const fst_s* f = P->fst;
  return PullView{f->slice_arcs, f->fwd.theta, f->fwd.sym_win};
}

int run_forward_wave(fst_plan_s* P, const Wave& W, cudaStream_t s, int32_t* d_status) {
  fst_s* f = P->fst;
  int rc;
  plan_learn(P, s);
  const LayoutView L = view_of(f->bwd);
  const TokenView T = wave_tokens(W);
  const FrontierState S = wave_state(P, W, nullptr);
  if ((rc = wave_begin(P, W, s, true))) return rc;
  if (P->driver == FST_DRIVER_PERSISTENT) {
    PROF(FST_PROF_FWD_STEP, launch_fwd_persist(L, T, wave_steps(W), S, persist_grid(P, W, 1), grid_sync_of(P), s));
  } else {
    const PullView R = pull_view(P);
    if (W.tmax >= 1) PROF(FST_PROF_FWD_FIRST, launch_fwd_first(L, T, wave_step(P, W, 1, 0), S, s));
    for (int32_t t = 1; t <= W.tmax; ++t) {
      PROF(FST_PROF_FWD_SUM, launch_fwd_sum(L, T, wave_step(P, W, t, t - 1), S, R, s));
      PROF(FST_PROF_FWD_STEP, launch_fwd_step(L, T, wave_step(P, W, t, t + 1), S, s));

    }
  }
  PROF(FST_PROF_FB_FINAL, launch_fb_final(S, W.Bw, P->logz + W.b0, d_status ? d_status + W.b0 : nullptr, s));
  plan_ran(P, s);
  return FST_OK;
}

// The backward pass of a wave; with `states`, also the expected start and
// final states.
int run_backward_wave(fst_plan_s* P, const Wave& W, const float* d_weights, bool states, cudaStream_t s) {
  fst_s* f = P->fst;
  const LayoutView L = view_of(f->bwd);
  const TokenView T = wave_tokens(W);
  const FrontierState S = wave_state(P, W, d_weights);
  const CountView C{1, nullptr, nullptr, P->cnt64, states ? P->start64 : nullptr, states ? P->final64 : nullptr};
  if (P->driver == FST_DRIVER_PERSISTENT) {
    if (P->gbar) FST_CUDA(cudaMemsetAsync(P->gbar, 0, 4, s));  // arrivals; a timed-out forward pass leaves them
    if (W.tmax >= 1)
      PROF(FST_PROF_BWD_STEP,
           launch_bwd_persist(L, T, wave_steps(W), S, C, persist_grid(P, W, 2), grid_sync_of(P), s));
  } else {
    for (int32_t t = W.tmax; t >= 1; --t) {
      StepView V = wave_step(P, W, t, t - 1);
      // compact accumulators: the step empties the backward values of t+1
      // (none are stored for the last position) and one more launch those
      // of position 1
      V.y_t = t + 1 < W.tmax ? t + 1 : 0;
      PROF(FST_PROF_BWD_STEP, launch_bwd_step(L, T, V, S, C, s));
    }
    if (W.tmax >= 2 && P->compact) PROF(FST_PROF_BWD_STEP, launch_bwd_clear(S, 1, f->num_sms, s));
  }
  if (states) PROF(FST_PROF_COUNTS, launch_final_posteriors(S, W.Bw, C, s));
  return FST_OK;
}

// Zero the count accumulators of a backward run.
int counts_begin(fst_plan_s* P, bool states, cudaStream_t s) {
  fst_s* f = P->fst;
  FST_CUDA(cudaMemsetAsync(P->cnt64, 0, (size_t)std::max<int64_t>(1, f->A) * 8, s));
  if (states) {
    FST_CUDA(cudaMemsetAsync(P->start64, 0, (size_t)f->Q * 8, s));
    FST_CUDA(cudaMemsetAsync(P->final64, 0, (size_t)f->Q * 8, s));
  }
  return FST_OK;
}

// Counts (and state posteriors) from their float64 accumulators to the
// caller's float arrays.
int counts_end(fst_plan_s* P, float* d_counts, float* d_start, float* d_final, cudaStream_t s) {
  fst_s* f = P->fst;
  int rc;
  if (d_counts) {
    const CountView C{1, nullptr, nullptr, P->cnt64};
    PROF(FST_PROF_COUNTS, launch_counts_out(f->A, C, d_counts, s));
  }
  if (d_start && (rc = launch_to_float(P->start64, f->Q, d_start, s))) return rc;
  if (d_final && (rc = launch_to_float(P->final64, f->Q, d_final, s))) return rc;
  return FST_OK;
}

inline cudaStream_t as_stream(void* p) { return (cudaStream_t)p; }

}  // namespace

static int plan_build(fst_t* f, const int32_t* hid, const int64_t* h_off, int32_t B, int64_t mem_budget_bytes,
                      int32_t flags, cudaStream_t s, fst_plan_s* donor, fst_plan_t** out);

static bool part_threads_on();

// The most parts a plan may have for its parts' step kernels to run chained
// (FSTGPU_CHAIN_PARTS, default 1: parts run unchained, where one part's
// early-scheduled blocks would hold SM slots that the other parts' running
// positions need).
static int32_t chain_parts_max() {
  static const int32_t v = [] {
    const char* e = std::getenv("FSTGPU_CHAIN_PARTS");
    return e && *e ? std::max(1, atoi(e)) : 1;
  }();
  return v;
}

// A plan of nparts stream-parallel parts: contiguous string ranges of about
// equal token counts, each an ordinary plan with its own stream; the count
// accumulators (and the expected start and final states) are the parent's,
// shared by the parts (their float64 atomics add up across parts).
static int plan_create_parts(fst_t* f, const int32_t* hid, const int64_t* h_off, int32_t B, int64_t budget,
                             int32_t flags, cudaStream_t s, int32_t nparts, fst_plan_s* donor, fst_plan_t** out) {
  // an earlier plan of as many parts lends each part's storage to the new
  // part of the same index, and its shared count accumulators
  std::unique_ptr<fst_plan_s> donor_owner(donor);
  if (donor && (int32_t)donor->parts.size() != nparts) donor_owner.reset();
  donor = donor_owner.get();
  std::unique_ptr<fst_plan_s> P(new fst_plan_s());
  P->fst = f;
  P->B = B;
  P->N = h_off[B];
  P->flags = flags;
  P->want_vit = !(flags & FST_PLAN_NO_VITERBI);
  P->want_fb = !(flags & FST_PLAN_NO_FB);
  int rc;
  // the parts' string ranges: each ends where the token count reaches its
  // share
  std::vector<int32_t> bs((size_t)nparts + 1, 0);
  for (int32_t i = 0; i < nparts; ++i) {
    int32_t b1 = B;
    if (i < nparts - 1) {
      const int64_t goal = (P->N * (i + 1)) / nparts;
      b1 = bs[i] + 1;
      while (b1 < B - (nparts - 1 - i) && h_off[b1] < goal) ++b1;
    }
    bs[i + 1] = b1;
  }
  // each part's donor: the earlier plan's part of the same index
  std::vector<fst_plan_s*> pd((size_t)nparts, nullptr);
  for (int32_t i = 0; i < nparts; ++i) {
    if (donor) std::swap(pd[i], donor->parts[i]);
    if (pd[i] && pd[i]->borrowed_counts) {
      // the count accumulators belong to the donor's parent (taken below)
      pd[i]->cnt64 = pd[i]->start64 = pd[i]->final64 = nullptr;
      pd[i]->borrowed_counts = false;
    }
  }
  // what the parts would otherwise each set up on the handle or read from
  // the device: the destination-ordered slice records (dense accumulators
  // with forward-backward) and the budget, taken once before they are built
  if (P->want_fb && (flags & FST_PLAN_DENSE_ACC) && (rc = slice_records_dst(f, s))) {
    for (fst_plan_s* q : pd) delete q;
    return rc;
  }
  const int64_t part_budget = budget > 0 ? std::max<int64_t>(budget / nparts, 1) : default_budget();
  // the parts are built in parallel, one host thread each (the caller's
  // building part 0; one after the other when FSTGPU_PART_THREADS=0):
  // their host tables and uploads are independent
  std::vector<fst_plan_t*> sub((size_t)nparts, nullptr);
  std::vector<int> prc((size_t)nparts, FST_OK);
  std::vector<std::string> perr((size_t)nparts);
  const int dev = f->device;
  auto build_part = [&](int32_t i) {
    if (i > 0 && cudaSetDevice(dev) != cudaSuccess) {
      prc[i] = cuda_fail(cudaGetLastError(), "part thread");
      perr[i] = fst_last_error();
      delete pd[i];
      return;
    }
    std::vector<int64_t> off((size_t)(bs[i + 1] - bs[i]) + 1);
    for (int32_t b = bs[i]; b <= bs[i + 1]; ++b) off[b - bs[i]] = h_off[b] - h_off[bs[i]];
    prc[i] = plan_build(f, hid + h_off[bs[i]], off.data(), bs[i + 1] - bs[i], part_budget,
                        (flags & 0xff) | PLAN_PART, s, pd[i], &sub[i]);
    if (prc[i]) perr[i] = fst_last_error();
  };
  {
    std::vector<std::thread> th;
    const bool threads = part_threads_on();
    for (int32_t i = 1; i < nparts && threads; ++i) th.emplace_back(build_part, i);
    build_part(0);
    for (int32_t i = 1; i < nparts && !threads; ++i) build_part(i);
    for (std::thread& t : th) t.join();
  }
  rc = FST_OK;
  for (int32_t i = 0; i < nparts; ++i) {
    if (prc[i] && !rc) {
      rc = prc[i];
      set_error("%s", perr[i].c_str());
    }
  }
  if (rc) {
    for (fst_plan_t* q : sub) delete q;
    return rc;
  }
  for (int32_t i = 0; i < nparts; ++i) {
    sub[i]->chain = nparts <= chain_parts_max();
    P->parts.push_back(sub[i]);
    P->part_b0.push_back(bs[i]);
    P->part_tok0.push_back(h_off[bs[i]]);
    P->relax += sub[i]->relax;
    P->bytes += sub[i]->bytes;
    P->max_len = std::max(P->max_len, sub[i]->max_len);
  }
  if (P->want_fb && donor && donor->want_fb && donor->cnt64 && donor->fst == f) {
    P->cnt64 = donor->cnt64;
    P->start64 = donor->start64;
    P->final64 = donor->final64;
    donor->cnt64 = donor->start64 = donor->final64 = nullptr;
    P->bytes += (int64_t)(f->A + 2 * (int64_t)f->Q) * 8;
    for (fst_plan_s* q : P->parts) {
      dfree(q->cnt64);
      dfree(q->start64);
      dfree(q->final64);
      q->cnt64 = P->cnt64;
      q->start64 = P->start64;
      q->final64 = P->final64;
      q->borrowed_counts = true;
    }
  } else if (P->want_fb) {
    if ((rc = alloc_track(P.get(), &P->cnt64, f->A)) || (rc = alloc_track(P.get(), &P->start64, f->Q)) ||
        (rc = alloc_track(P.get(), &P->final64, f->Q)))
      return rc;
    for (fst_plan_s* q : P->parts) {
      dfree(q->cnt64);
      dfree(q->start64);
      dfree(q->final64);
      q->cnt64 = P->cnt64;
      q->start64 = P->start64;
      q->final64 = P->final64;
      q->borrowed_counts = true;
    }
  }
  P->part_event.resize(nparts + 1, nullptr);
  for (cudaEvent_t& e : P->part_event) FST_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  P->part_stream.resize(nparts, nullptr);
  for (cudaStream_t& st : P->part_stream) FST_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  *out = P.release();
  return FST_OK;
}

// fn(i) for every part i: from one host thread per part (the caller's
// taking part 0), so that the parts' launches are issued in parallel, or
// one after the other while the stream is being recorded into a graph, or
// when FSTGPU_PART_THREADS=0 (a profiler that selects launches by a range
// of the calling thread then sees them all).
static bool part_threads_on() {
  static const bool on = [] {
    const char* e = std::getenv("FSTGPU_PART_THREADS");
    return !(e && e[0] == '0');
  }();
  return on;
}
template <class Fn>
static int parts_each(fst_plan_s* P, cudaStream_t s, Fn fn) {
  const size_t n = P->parts.size();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  bool threads = n > 1 && part_threads_on();
  if (threads && (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)) {
    (void)cudaGetLastError();
    threads = false;
  }
  if (!threads) {
    for (size_t i = 0; i < n; ++i) {
      const int rc = fn(i);
      if (rc) return rc;
    }
    return FST_OK;
  }
  std::vector<int> rcs(n, FST_OK);
  const int dev = P->fst->device;
  std::vector<std::thread> th;
  th.reserve(n - 1);
  for (size_t i = 1; i < n; ++i)
    th.emplace_back([&rcs, &fn, dev, i] {
      rcs[i] = cudaSetDevice(dev) == cudaSuccess ? fn(i) : cuda_fail(cudaGetLastError(), "part thread");
    });
  rcs[0] = fn(0);
  for (std::thread& t : th) t.join();
  for (int rc : rcs)
    if (rc) return rc;
  return FST_OK;
}

// The parts start after the work queued on s and s waits for all of them.
static int parts_fork(fst_plan_s* P, cudaStream_t s) {
  FST_CUDA(cudaEventRecord(P->part_event[0], s));
  for (cudaStream_t st : P->part_stream) FST_CUDA(cudaStreamWaitEvent(st, P->part_event[0], 0));
  return FST_OK;
}
static int parts_join(fst_plan_s* P, cudaStream_t s) {
  for (size_t i = 0; i < P->parts.size(); ++i) {
    FST_CUDA(cudaEventRecord(P->part_event[1 + i], P->part_stream[i]));
    FST_CUDA(cudaStreamWaitEvent(s, P->part_event[1 + i], 0));
  }
  return FST_OK;
}

// Plan creation from device inputs: the offsets and symbols are read back
// once and checked on the host, then the plan is built from those host
// arrays (plan_build).  Synchronises the stream.
static int plan_create(fst_t* f, const int32_t* d_ids, const int64_t* d_offsets, int32_t B, int64_t mem_budget_bytes,
                       int32_t flags, void* stream, fst_plan_s* donor, fst_plan_t** out) {
  std::unique_ptr<fst_plan_s> donor_owner(donor);
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
  std::vector<int32_t> hid((size_t)std::max<int64_t>(N, 1));
  if (N > 0) {
    FST_CUDA(cudaMemcpyAsync(hid.data(), d_ids, (size_t)N * 4, cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
  }
  for (int64_t i = 0; i < N; ++i)
    if (hid[i] < 0 || hid[i] >= f->m) {
      set_error("a symbol id is outside [0, %d)", f->m);
      return FST_ERR_INVALID_ARG;
    }
  return plan_build(f, hid.data(), h_off.data(), B, mem_budget_bytes, flags, s, donor_owner.release(), out);
}

// Plan building from host arrays (symbols checked; h_off[0] = 0).
// `donor` (owned: always released here) is an earlier plan of the same
// handle whose device storage is taken over when it is large enough, so
// that repeated batch calls neither allocate nor clear it again.
static int plan_build(fst_t* f, const int32_t* hid, const int64_t* h_off, int32_t B, int64_t mem_budget_bytes,
                      int32_t flags, cudaStream_t s, fst_plan_s* donor, fst_plan_t** out) {
  std::unique_ptr<fst_plan_s> donor_owner(donor);
  *out = nullptr;
  const int64_t N = h_off[B];
  const int32_t nparts = std::min<int32_t>((flags >> 8) & 0xff, std::max(B, 1));
  if (nparts > 1) return plan_create_parts(f, hid, h_off, B, mem_budget_bytes, flags, s, nparts, donor_owner.release(), out);
  if (donor && !donor->parts.empty()) donor_owner.reset();  // a parts plan lends nothing to a single plan
  fst_plan_s* P = new fst_plan_s();
  P->fst = f;
  P->B = B;
  P->N = N;
  P->flags = flags;
  P->want_vit = !(flags & FST_PLAN_NO_VITERBI);
  P->want_fb = !(flags & FST_PLAN_NO_FB);
  int rc = FST_OK;
  std::vector<HostWave> hw;
  do {
    // relaxations of one pass (the paper's definition: every arc of every slice)
    P->relax = 0;
    for (int64_t i = 0; i < N; ++i) P->relax += f->h_sym_arc[hid[i] + 1] - f->h_sym_arc[hid[i]];
    // waves: consecutive strings whose memory fits the budget.  Default: a
    // quarter of the device memory free now, at most 32 GiB and at least
    // 256 MiB (the GPU may be shared; fst_set_batch_budget raises it)
    const int64_t budget = mem_budget_bytes > 0 ? mem_budget_bytes : default_budget();
    // dense accumulators: 2 x 8 bytes per state (Viterbi), or 2 x 16 for
    // the forward sums and maxima plus 2 x 8 for the backward values;
    // Viterbi also maps states to pool entries, 2 x 4 bytes.  Compact ones
    // do not grow with the strings.
    P->compact = !(flags & FST_PLAN_DENSE_ACC);
    const int64_t per_string = (P->compact ? 0 : dense_bytes_per_string(f, P->want_fb, P->want_vit)) + 64;
    const int64_t per_token = TOKEN_BYTES + POOL_PER_TOKEN * 20;
    int32_t b0 = 0;
    int64_t acc = 0;
    for (int32_t b = 0; b <= B; ++b) {
      const int64_t need = (b < B) ? per_string + (h_off[b + 1] - h_off[b]) * per_token : 0;
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
      set_error("the batch needs %d waves under a budget of %lld bytes", (int)P->waves.size(), (long long)budget);
      rc = FST_ERR_OOM;
      break;
    }
    for (Wave& w : P->waves) {
      hw.emplace_back();
      if ((rc = build_wave(P, w, h_off, hid, hw.back()))) break;
      P->max_bw = std::max<int64_t>(P->max_bw, w.Bw);
      P->max_ntok = std::max<int64_t>(P->max_ntok, w.ntok);
      P->max_stage = std::max(P->max_stage, w.stage);
      P->max_len = std::max(P->max_len, w.tmax);
      // live pool: its exact bound when that is small, else the larger of
      // POOL_PER_TOKEN entries per token and a quarter of the budget (at
      // least 256 MiB, at most 4 GiB)
      const int64_t ebytes = 20;
      const int64_t want = std::max(w.ntok * POOL_PER_TOKEN,
                                    std::min(std::max(budget / 4, (int64_t)256 << 20), (int64_t)4 << 30) / ebytes);
      // pool entries are named by int32 indices
      P->pool_cap = std::max(P->pool_cap, std::min(std::min(w.pool_bound, want), (int64_t)INT32_MAX));
      // compact accumulators at half load (a power of two; slots are named
      // by int32 indices)
      int64_t busiest = 0;
      for (int32_t t = 1; t <= w.tmax; ++t) busiest = std::max<int64_t>(busiest, w.step0[t + 1] - w.step0[t]);
      const int64_t live = std::min(w.stage, std::max(busiest * LIVE_PER_TOKEN, LIVE_FLOOR));
      int64_t slots = 1024;
      while (slots < 2 * live && slots < ((int64_t)1 << 30)) slots <<= 1;
      P->hslots = std::max(P->hslots, slots);
    }
    if (rc) break;
    P->acc_stride = P->want_fb ? 2 : 1;
    fst_plan_s* d = donor_owner.get();
    if (d && d->fst == f && d->want_fb == P->want_fb && d->want_vit == P->want_vit && d->compact == P->compact &&
        (!P->compact || d->cap_hslots >= P->hslots) && (P->compact || d->cap_bw >= P->max_bw) &&
        d->cap_nt >= P->max_ntok && d->cap_stage >= P->max_stage && d->pool_cap >= P->pool_cap &&
        d->cap_len >= P->max_len && d->cap_B >= B) {
      // take the donor's storage: its accumulators are zero (or, after an
      // overflow, cleared by the next pass through the moved error flag)
#define PLAN_MOVE(x) P->x = d->x; d->x = nullptr;
      PLAN_STORAGE(PLAN_MOVE)
#undef PLAN_MOVE
      P->cap_bw = d->cap_bw;
      P->cap_nt = d->cap_nt;
      P->cap_stage = d->cap_stage;
      P->cap_len = d->cap_len;
      P->cap_B = d->cap_B;
      P->cap_hslots = d->cap_hslots;
      P->cap_tok = d->cap_tok;
      P->pool_cap = d->pool_cap;
      P->store_bytes = d->store_bytes;
      P->bytes += d->store_bytes;
      break;
    }
    donor_owner.reset();  // too small (or none): release its memory first
    P->cap_bw = P->max_bw;
    P->cap_nt = P->max_ntok;
    P->cap_stage = P->max_stage;
    P->cap_len = P->max_len;
    P->cap_B = B;
    P->cap_hslots = P->compact ? P->hslots : 0;
    const int64_t na = P->compact ? 0 : P->max_bw * 2 * (int64_t)f->Q;
    const int64_t nt = P->max_ntok;
    const int64_t nh = P->compact ? htab_words(P, P->cap_hslots) : 0;
    if (P->compact) {
      if ((rc = alloc_store(P, &P->htab, nh))) break;
      if (P->want_fb && (rc = alloc_store(P, &P->bslot, P->pool_cap))) break;
    } else {
      if ((rc = alloc_store(P, &P->acc, na * P->acc_stride))) break;
      if (P->want_fb && (rc = alloc_store(P, &P->beta, na))) break;
      if (P->want_vit && (rc = alloc_store(P, &P->vmap, na))) break;
      if (P->want_fb) {
        // the direction switch's dense vectors, and the destination-ordered
        // slice records it reads
        if ((rc = alloc_store(P, &P->dvec, (int64_t)DENSE_SLOTS * 2 * f->Q)) ||
            (rc = alloc_store(P, &P->dslot, nt)) ||
            (rc = alloc_store(P, &P->dlist, ((int64_t)P->max_len + 2) * DENSE_SLOTS)) ||
            (rc = alloc_store(P, &P->dcnt, (int64_t)P->max_len + 2)))
          break;
        if ((rc = launch_fill_neg_inf(P->dvec, (int64_t)DENSE_SLOTS * 2 * f->Q, s))) break;
        // (a part's parent has set them up before building its parts)
        if (!(flags & PLAN_PART) && (rc = slice_records_dst(f, s))) break;
      }
    }
    // forward: arcs on the next symbol; Viterbi with dense accumulators:
    // the predecessor entry
    if ((P->want_fb || !P->compact) && (rc = alloc_store(P, &P->pool_n, P->pool_cap))) break;
    if ((rc = alloc_store(P, &P->stage, P->max_stage)) || (rc = alloc_store(P, &P->stage_b, P->max_stage)) ||
        (rc = alloc_store(P, &P->scnt, nt)) || (rc = alloc_store(P, &P->pool_q, P->pool_cap)) ||
        (rc = alloc_store(P, &P->pool_x, P->pool_cap)) || (rc = alloc_store(P, &P->pool_v, P->pool_cap)) ||
        (rc = alloc_store(P, &P->pool_base, nt)) || (rc = alloc_store(P, &P->pool_cnt, nt)) ||
        (rc = alloc_store(P, &P->pool_top, 1)) || (rc = alloc_store(P, &P->slot_base, nt)) ||
        (rc = alloc_store(P, &P->step_rng, 2 * ((int64_t)P->max_len + 2))) ||
        (rc = alloc_store(P, &P->flags_d, 2)) || (rc = alloc_store(P, &P->mkey, nt)) ||
        (rc = alloc_store(P, &P->ekey, nt)) || (rc = alloc_store(P, &P->csum, nt)) ||
        (rc = alloc_store(P, &P->esum, nt)) || (rc = alloc_store(P, &P->jfinal, P->max_bw)) ||
        (rc = alloc_store(P, &P->logz, B)) || (rc = alloc_store(P, &P->gbar, 2)))
      break;
    if (P->want_fb && !(flags & PLAN_PART) &&
        ((rc = alloc_store(P, &P->cnt64, f->A)) || (rc = alloc_store(P, &P->start64, f->Q)) ||
         (rc = alloc_store(P, &P->final64, f->Q))))
      break;
    // the accumulators start at zero and every run leaves them so
    cudaError_t ce = cudaSuccess;
    if (P->acc) ce = cudaMemsetAsync(P->acc, 0, (size_t)std::max<int64_t>(na * P->acc_stride, 1) * 8, s);
    if (ce == cudaSuccess && P->beta) ce = cudaMemsetAsync(P->beta, 0, (size_t)std::max<int64_t>(na, 1) * 8, s);
    if (ce == cudaSuccess && P->htab) ce = cudaMemsetAsync(P->htab, 0, (size_t)std::max<int64_t>(nh, 1) * 8, s);
    if (ce == cudaSuccess && P->dcnt)
      ce = cudaMemsetAsync(P->dcnt, 0, (size_t)((int64_t)P->max_len + 2) * 4, s);
    // position ranges start empty (a backward step reads those of a later
    // position to empty its tables)
    if (ce == cudaSuccess)
      ce = cudaMemsetAsync(P->step_rng, 0, (size_t)(2 * ((int64_t)P->max_len + 2)) * 8, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(P->flags_d, 0, 8, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(P->gbar, 0, 8, s);
    // per-token pool ranges start empty: a run that stops early leaves the
    // later positions' ranges as the previous run (or this clear) left them
    if (ce == cudaSuccess) ce = cudaMemsetAsync(P->pool_base, 0, (size_t)std::max<int64_t>(nt, 1) * 8, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(P->pool_cnt, 0, (size_t)std::max<int64_t>(nt, 1) * 4, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "plan storage");
  } while (0);
  if (!rc) rc = upload_tokens(P, hw, s);
  if (rc) {
    delete P;
    return rc;
  }
  *out = P;
  return FST_OK;
}

extern "C" int fst_plan_create(fst_t* f, const int32_t* d_ids, const int64_t* d_offsets, int32_t B,
                               int64_t mem_budget_bytes, int32_t flags, void* stream, fst_plan_t** out) {
  return plan_create(f, d_ids, d_offsets, B, mem_budget_bytes, flags & ~PLAN_PART, stream, nullptr, out);
}

extern "C" int fst_plan_destroy(fst_plan_t* P) {
  delete P;
  return FST_OK;
}

extern "C" int fst_plan_info(const fst_plan_t* P, int32_t* num_strings, int64_t* num_tokens, int32_t* num_waves,
                             int32_t* max_len, int64_t* relaxations, int64_t* viterbi_launches,
                             int64_t* fb_launches, int64_t* device_bytes) {
  if (!P) { set_error("plan is NULL"); return FST_ERR_INVALID_ARG; }
  int64_t vl = 0, fl = 0;
  if (!P->parts.empty()) {
    int32_t nw = 0;
    for (fst_plan_s* q : P->parts) {
      int32_t w = 0;
      int64_t v = 0, fb = 0;
      fst_plan_info(q, nullptr, nullptr, &w, nullptr, nullptr, &v, &fb, nullptr);
      nw = std::max(nw, w);
      vl += v;
      fl += fb - 1;  // the parts share one counts-out launch
    }
    if (num_strings) *num_strings = P->B;
    if (num_tokens) *num_tokens = P->N;
    if (num_waves) *num_waves = nw;
    if (max_len) *max_len = P->max_len;
    if (relaxations) *relaxations = P->relax;
    if (viterbi_launches) *viterbi_launches = vl;
    if (fb_launches) *fb_launches = fl + 1;
    if (device_bytes) *device_bytes = P->bytes;
    return FST_OK;
  }
  for (const Wave& w : P->waves) {
    if (P->driver == FST_DRIVER_PERSISTENT) {
      // overflow clear, the persistent pass, final, backtrace
      vl += 4;
      // overflow clear, forward pass, final, backward pass
      fl += w.tmax >= 1 ? 4 : 3;
      continue;
    }
    // overflow clear, first push, one step per position, final, backtrace
    vl += (int64_t)w.tmax + 4;
    // overflow clear, first push, sum and step per position, final; one
    // backward step per position (and, compact, the clear of position 1)
    fl += 3 * (int64_t)w.tmax + 3 + ((P->compact && w.tmax >= 2) ? 1 : 0);

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
  if (!P || !d_scores || (P->N > 0 && !d_paths)) {
    set_error("fst_plan_viterbi: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  if (!P->want_vit) { set_error("plan was created without Viterbi storage"); return FST_ERR_STATE; }
  cudaStream_t s = as_stream(stream);
  int rc;
  // the Viterbi run reuses the accumulators and pool a pending backward pass needs
  P->forward_done = false;
  if (!P->parts.empty()) {
    if ((rc = parts_fork(P, s))) return rc;
    rc = parts_each(P, s, [&](size_t i) {
      const int32_t b0 = P->part_b0[i];
      const int64_t k0 = P->part_tok0[i];
      return fst_plan_viterbi(P->parts[i], d_scores + b0, d_paths + k0, d_olabels ? d_olabels + k0 : nullptr,
                              d_status ? d_status + b0 : nullptr, P->part_stream[i]);
    });
    if (rc) return rc;
    return parts_join(P, s);
  }
  for (const Wave& W : P->waves)
    if ((rc = run_viterbi_wave(P, W, d_scores, d_paths, d_olabels, d_status, s))) return rc;
  return FST_OK;
}

extern "C" int fst_plan_forward(fst_plan_t* P, double* d_logz, int32_t* d_status, void* stream) {
  if (!P || !d_logz) { set_error("fst_plan_forward: bad arguments"); return FST_ERR_INVALID_ARG; }
  if (!P->want_fb) { set_error("plan was created without forward-backward storage"); return FST_ERR_STATE; }
  cudaStream_t s = as_stream(stream);
  int rc;
  if (!P->parts.empty()) {
    if ((rc = parts_fork(P, s))) return rc;
    rc = parts_each(P, s, [&](size_t i) {
      const int32_t b0 = P->part_b0[i];
      return fst_plan_forward(P->parts[i], d_logz + b0, d_status ? d_status + b0 : nullptr, P->part_stream[i]);
    });
    if (rc) return rc;
    if ((rc = parts_join(P, s))) return rc;
    P->forward_done = true;
    return FST_OK;
  }
  if (P->waves.size() > 1) { set_error("fst_plan_forward needs a single-wave plan"); return FST_ERR_STATE; }
  for (const Wave& W : P->waves)
    if ((rc = run_forward_wave(P, W, s, d_status))) return rc;
  if (P->B > 0) FST_CUDA(cudaMemcpyAsync(d_logz, P->logz, (size_t)P->B * 8, cudaMemcpyDeviceToDevice, s));
  P->forward_done = true;
  return FST_OK;
}

extern "C" int fst_plan_backward_ex(fst_plan_t* P, const float* d_weights, float* d_counts, float* d_start,
                                    float* d_final, void* stream) {
  if (!P || (!d_counts && !d_start && !d_final)) {
    set_error("fst_plan_backward: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  if (!P->forward_done) { set_error("fst_plan_backward needs a preceding fst_plan_forward"); return FST_ERR_STATE; }
  cudaStream_t s = as_stream(stream);
  const bool states = d_start || d_final;
  int rc;
  if ((rc = counts_begin(P, states, s))) return rc;
  if (!P->parts.empty()) {
    if ((rc = parts_fork(P, s))) return rc;
    rc = parts_each(P, s, [&](size_t i) {
      fst_plan_s* q = P->parts[i];
      const float* w = d_weights ? d_weights + P->part_b0[i] : nullptr;
      for (const Wave& W : q->waves) {
        const int r = run_backward_wave(q, W, w, states, P->part_stream[i]);
        if (r) return r;
      }
      return (int)FST_OK;
    });
    if (rc) return rc;
    if ((rc = parts_join(P, s))) return rc;
    return counts_end(P, d_counts, d_start, d_final, s);
  }
  for (const Wave& W : P->waves)
    if ((rc = run_backward_wave(P, W, d_weights, states, s))) return rc;
  return counts_end(P, d_counts, d_start, d_final, s);
}

extern "C" int fst_plan_backward(fst_plan_t* P, const float* d_weights, float* d_counts, void* stream) {
  if (!d_counts) { set_error("fst_plan_backward: bad arguments"); return FST_ERR_INVALID_ARG; }
  return fst_plan_backward_ex(P, d_weights, d_counts, nullptr, nullptr, stream);
}

extern "C" int fst_plan_forward_backward_ex(fst_plan_t* P, const float* d_weights, double* d_logz,
                                            float* d_counts, float* d_start, float* d_final, int32_t* d_status,
                                            void* stream) {
  if (!P || !d_logz) { set_error("fst_plan_forward_backward: bad arguments"); return FST_ERR_INVALID_ARG; }
  if (!P->want_fb) { set_error("plan was created without forward-backward storage"); return FST_ERR_STATE; }
  cudaStream_t s = as_stream(stream);
  const bool states = d_start || d_final;
  const bool bwd = d_counts || states;
  int rc;
  if (bwd && (rc = counts_begin(P, states, s))) return rc;
  if (!P->parts.empty()) {
    if ((rc = parts_fork(P, s))) return rc;
    rc = parts_each(P, s, [&](size_t i) {
      fst_plan_s* q = P->parts[i];
      cudaStream_t st = P->part_stream[i];
      const int32_t b0 = P->part_b0[i];
      const float* w = d_weights ? d_weights + b0 : nullptr;
      for (const Wave& W : q->waves) {
        int r = run_forward_wave(q, W, st, d_status ? d_status + b0 : nullptr);
        if (!r && bwd) r = run_backward_wave(q, W, w, states, st);
        if (r) return r;
      }
      if (q->B > 0) FST_CUDA(cudaMemcpyAsync(d_logz + b0, q->logz, (size_t)q->B * 8, cudaMemcpyDeviceToDevice, st));
      q->forward_done = q->waves.size() <= 1;
      return (int)FST_OK;
    });
    if (rc) return rc;
    if ((rc = parts_join(P, s))) return rc;
    if (bwd && (rc = counts_end(P, d_counts, d_start, d_final, s))) return rc;
    P->forward_done = true;
    for (fst_plan_s* q : P->parts) P->forward_done = P->forward_done && q->forward_done;
    return FST_OK;
  }
  for (const Wave& W : P->waves) {
    if ((rc = run_forward_wave(P, W, s, d_status))) return rc;
    if (bwd && (rc = run_backward_wave(P, W, d_weights, states, s))) return rc;
  }
  if (P->B > 0) FST_CUDA(cudaMemcpyAsync(d_logz, P->logz, (size_t)P->B * 8, cudaMemcpyDeviceToDevice, s));
  if (bwd && (rc = counts_end(P, d_counts, d_start, d_final, s))) return rc;
  P->forward_done = P->waves.size() <= 1;
  return FST_OK;
}

extern "C" int fst_plan_forward_backward(fst_plan_t* P, const float* d_weights, double* d_logz, float* d_counts,
                                         int32_t* d_status, void* stream) {
  return fst_plan_forward_backward_ex(P, d_weights, d_logz, d_counts, nullptr, nullptr, d_status, stream);
}

// The batch calls keep the storage of their last plan in the handle (one
// slot per kind, taken out under a lock while a call runs), so that a
// stream of batches of similar size allocates and clears it once.
static fst_plan_s* take_cached(fst_t* f, int kind) {
  std::lock_guard<std::mutex> lock(*f->batch_mu);
  fst_plan_s* p = f->batch_plan[kind];
  f->batch_plan[kind] = nullptr;
  return p;
}
static void put_cached(fst_t* f, int kind, fst_plan_s* p) {
  fst_plan_s* old = nullptr;
  {
    std::lock_guard<std::mutex> lock(*f->batch_mu);
    old = f->batch_plan[kind];
    f->batch_plan[kind] = p;
  }
  delete old;
}

// Plan flags of a batch call (kind 0: Viterbi, 1: forward-backward): the
// handle's setting (fst_set_batch_plan) or, by default, stream-parallel
// parts by batch size (one Viterbi part per 32 strings, at most 2 and at
// most 400 / the longest string; one forward-backward part per 8 strings,
// at most 4 and at most 1,600 / the longest string) and dense accumulators
// when they fit the budget in one wave.
static int batch_flags(fst_t* f, int kind, const int64_t* d_offsets, int32_t B, cudaStream_t s, int32_t* flags) {
  int32_t fl = kind == 0 ? FST_PLAN_NO_FB : FST_PLAN_NO_VITERBI;
  std::vector<int64_t> h_off((size_t)B + 1, 0);
  if (B > 0) {
    FST_CUDA(cudaMemcpyAsync(h_off.data(), d_offsets, (size_t)(B + 1) * 8, cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
  }
  int64_t tmax = 1;
  for (int32_t b = 0; b < B; ++b) tmax = std::max(tmax, h_off[b + 1] - h_off[b]);
  const int64_t N = h_off[B];
  int32_t parts = f->batch_parts[kind];
  if (parts <= 0) {
    // by batch size, and few enough that a run stays near 400 (Viterbi) or
    // 1,600 (forward-backward) position launches: the parts of a long
    // string's batch multiply launches that the host issues one by one
    const int64_t by_len = (kind == 0 ? 400 : 1600) / tmax;
    parts = (int32_t)std::max<int64_t>(
        1, std::min<int64_t>(kind == 0 ? std::min(2, B / 32) : std::min(4, B / 8), by_len));
  }
  if (parts > 1) fl |= FST_PLAN_PARTS(parts);
  int32_t layout = f->batch_layout;
  if (layout < 0) {
    const int64_t budget = f->batch_budget > 0 ? f->batch_budget : default_budget();
    const int64_t need = (dense_bytes_per_string(f, kind == 1, kind == 0) + 64) * (int64_t)B +
                         (TOKEN_BYTES + POOL_PER_TOKEN * 20) * N;
    layout = need <= budget ? 1 : 0;
  }
  if (layout == 1) fl |= FST_PLAN_DENSE_ACC;
  *flags = fl;
  return FST_OK;
}

extern "C" int fst_set_batch_plan(fst_t* f, int32_t parts_viterbi, int32_t parts_fb, int32_t layout, int32_t graph) {
  if (!f || parts_viterbi < 0 || parts_viterbi > 255 || parts_fb < 0 || parts_fb > 255 || layout < -1 || layout > 1 ||
      graph < -1 || graph > 1) {
    set_error("fst_set_batch_plan: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  f->batch_parts[0] = parts_viterbi;
  f->batch_parts[1] = parts_fb;
  f->batch_layout = layout;
  f->batch_graph = graph;
  return FST_OK;
}

// Run a batch call's plan: its launches recorded into a CUDA graph and the
// graph launched (fst_set_batch_plan), or launched one by one (the
// default: recording a plan of several thousand launches and instantiating
// the graph measured slower than launching it once).  The legacy default
// stream cannot be recorded: launches one by one there, as inside a capture
// the caller has begun.
template <class Run>
static int batch_run(fst_t* f, fst_plan_t* P, int64_t launches, cudaStream_t s, Run run) {
  bool graph = f->batch_graph == 1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (graph && (s == 0 || s == cudaStreamLegacy || cudaStreamIsCapturing(s, &cs) != cudaSuccess ||
                cs != cudaStreamCaptureStatusNone)) {
    (void)cudaGetLastError();
    graph = false;
  }
  if (!graph) return run(s);
  FST_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const int rc = run(s);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
    return cuda_fail(e, "batch graph capture");
  }
  cudaGraphExec_t ge = nullptr;
  cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e2 == cudaSuccess) e2 = cudaGraphLaunch(ge, s);
  if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
  if (ge) cudaGraphExecDestroy(ge);
  if (e2 != cudaSuccess) return cuda_fail(e2, "batch graph launch");
  (void)P;
  return FST_OK;
}

extern "C" int fst_viterbi_batch(fst_t* f, const int32_t* d_ids, const int64_t* d_offsets, int32_t B,
                                 float* d_scores, int32_t* d_paths, int32_t* d_olabels, int32_t* d_status,
                                 void* stream) {
  if (!f) { set_error("fst is NULL"); return FST_ERR_INVALID_ARG; }
  if (B < 0 || !d_offsets) { set_error("fst_viterbi_batch: bad arguments"); return FST_ERR_INVALID_ARG; }
  fst_plan_t* P = nullptr;
  int32_t flags = 0;
  int rc = batch_flags(f, 0, d_offsets, B, as_stream(stream), &flags);
  if (rc) return rc;
  rc = plan_create(f, d_ids, d_offsets, B, f->batch_budget, flags, stream, take_cached(f, 0), &P);
  if (rc) return rc;
  int64_t vl = 0;
  fst_plan_info(P, nullptr, nullptr, nullptr, nullptr, nullptr, &vl, nullptr, nullptr);
  rc = batch_run(f, P, vl, as_stream(stream), [&](cudaStream_t st) {
    return fst_plan_viterbi(P, d_scores, d_paths, d_olabels, d_status, (void*)st);
  });
  cudaError_t e = cudaStreamSynchronize(as_stream(stream));
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "fst_viterbi_batch");
  if (rc) fst_plan_destroy(P); else put_cached(f, 0, P);
  return rc;
}

extern "C" int fst_forward_backward_batch(fst_t* f, const int32_t* d_ids, const int64_t* d_offsets, int32_t B,
                                          const float* d_weights, double* d_logz, float* d_counts,
                                          int32_t* d_status, void* stream) {
  if (!f) { set_error("fst is NULL"); return FST_ERR_INVALID_ARG; }
  if (B < 0 || !d_offsets) { set_error("fst_forward_backward_batch: bad arguments"); return FST_ERR_INVALID_ARG; }
  fst_plan_t* P = nullptr;
  int32_t flags = 0;
  int rc = batch_flags(f, 1, d_offsets, B, as_stream(stream), &flags);
  if (rc) return rc;
  rc = plan_create(f, d_ids, d_offsets, B, f->batch_budget, flags, stream, take_cached(f, 1), &P);
  if (rc) return rc;
  int64_t fl = 0;
  fst_plan_info(P, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, &fl, nullptr);
  rc = batch_run(f, P, fl, as_stream(stream), [&](cudaStream_t st) {
    return fst_plan_forward_backward(P, d_weights, d_logz, d_counts, d_status, (void*)st);
  });
  cudaError_t e = cudaStreamSynchronize(as_stream(stream));
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "fst_forward_backward_batch");
  if (rc) fst_plan_destroy(P); else put_cached(f, 1, P);
  return rc;
}

extern "C" int fst_plan_live_work(fst_plan_t* P, int64_t* entries, int64_t* arcs, void* stream) {
  if (!P) { set_error("plan is NULL"); return FST_ERR_INVALID_ARG; }
  if (!P->parts.empty()) {
    int64_t e = 0, a = 0;
    for (fst_plan_s* q : P->parts) {
      int64_t qe = 0, qa = 0;
      const int rc = fst_plan_live_work(q, &qe, &qa, stream);
      if (rc) return rc;
      e += qe;
      a = (a < 0 || qa < 0) ? -1 : a + qa;
    }
    if (entries) *entries = e;
    if (arcs) *arcs = a;
    return FST_OK;
  }
  cudaStream_t s = as_stream(stream);
  int64_t top = 0;
  FST_CUDA(cudaMemcpyAsync(&top, P->pool_top, 8, cudaMemcpyDeviceToHost, s));
  FST_CUDA(cudaStreamSynchronize(s));
  top = std::min(top, P->pool_cap);
  if (entries) *entries = top;
  if (arcs) {
    *arcs = -1;
    if (P->want_fb) {
      unsigned long long* d_sum = nullptr;
      int rc = dalloc(&d_sum, 1);
      if (rc) return rc;
      unsigned long long h = 0;
      cudaError_t e = cudaMemsetAsync(d_sum, 0, 8, s);
      if (e == cudaSuccess && top > 0) {
        k_sum_i32<<<(unsigned)std::min<int64_t>(1024, (top + TB - 1) / TB), TB, 0, s>>>(P->pool_n, top, d_sum);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_sum, 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      dfree(d_sum);
      if (rc) return rc;
      if (e != cudaSuccess) return cuda_fail(e, "fst_plan_live_work");
      *arcs = (int64_t)h;
    }
  }
  return FST_OK;
}

extern "C" int fst_plan_limit_pool(fst_plan_t* P, int64_t entries) {
  if (!P || entries < 0) { set_error("fst_plan_limit_pool: bad arguments"); return FST_ERR_INVALID_ARG; }
  P->pool_limit = entries;
  for (fst_plan_s* q : P->parts) q->pool_limit = entries;
  return FST_OK;
}

extern "C" int fst_plan_set_pull(fst_plan_t* P, int64_t min_live) {
  if (!P || min_live < -1) { set_error("fst_plan_set_pull: bad arguments"); return FST_ERR_INVALID_ARG; }
  P->pull_min = min_live;
  for (fst_plan_s* q : P->parts) q->pull_min = min_live;
  return FST_OK;
}

extern "C" int fst_plan_limit_table(fst_plan_t* P, int64_t slots) {
  if (!P || slots < 0) { set_error("fst_plan_limit_table: bad arguments"); return FST_ERR_INVALID_ARG; }
  P->table_limit = slots;
  for (fst_plan_s* q : P->parts) q->table_limit = slots;
  return FST_OK;
}

extern "C" int fst_plan_table_slots(const fst_plan_t* P, int64_t* slots) {
  if (!P || !slots) { set_error("fst_plan_table_slots: bad arguments"); return FST_ERR_INVALID_ARG; }
  int64_t n = P->compact ? P->cap_hslots : 0;
  for (const fst_plan_s* q : P->parts) n = std::max(n, q->compact ? q->cap_hslots : 0);
  *slots = n;
  return FST_OK;
}

extern "C" int fst_plan_set_driver(fst_plan_t* P, int32_t driver, int32_t grid_blocks, int64_t barrier_timeout_us) {
  if (!P || (driver != FST_DRIVER_LAUNCH && driver != FST_DRIVER_PERSISTENT) || grid_blocks < 0 ||
      barrier_timeout_us < 0) {
    set_error("fst_plan_set_driver: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  if (driver == FST_DRIVER_PERSISTENT && P->parts.size() > 1) {
    set_error("the persistent driver runs one pass at a time: a plan of several parts cannot use it");
    return FST_ERR_UNSUPPORTED;
  }
  if (driver == FST_DRIVER_PERSISTENT) {
    int dev = 0, coop = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) { set_error("the device cannot launch cooperative kernels"); return FST_ERR_UNSUPPORTED; }
    const int cap = std::min(persist_grid_limit(0), std::min(persist_grid_limit(1), persist_grid_limit(2)));
    if (cap <= 0) { set_error("no co-resident grid for the persistent passes"); return FST_ERR_UNSUPPORTED; }
    if (grid_blocks > cap) {
      set_error("a grid of %d blocks cannot be co-resident (at most %d)", grid_blocks, cap);
      return FST_ERR_UNSUPPORTED;
    }
  }
  P->driver = driver;
  P->persist_grid = grid_blocks;
  if (barrier_timeout_us > 0) P->barrier_limit_ns = (uint64_t)barrier_timeout_us * 1000ull;
  return FST_OK;
}

// ------------------------------------------------------------- autotuner
// A configuration of a plan's driver: which driver, the persistent grid, and
// the launch driver's grid density.  Results are cached per device name,
// FST shape and batch shape, in this process and, when FSTGPU_TUNE_CACHE
// names a file, across processes (one tab-separated line per key).
namespace {
struct TuneConf {
  int32_t driver = FST_DRIVER_LAUNCH, grid = 0, density = 64;
  double ms = 0.0;
};
std::mutex g_tune_mu;
std::map<std::string, TuneConf> g_tune;
bool g_tune_loaded = false;

void tune_load_file() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("FSTGPU_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* fh = fopen(path, "r");
  if (!fh) return;
  char line[1024];
  while (fgets(line, sizeof(line), fh)) {
    char key[768];
    TuneConf c;
    if (sscanf(line, "%767[^\t]\t%d\t%d\t%d\t%lf", key, &c.driver, &c.grid, &c.density, &c.ms) == 5 &&
        (c.driver == FST_DRIVER_LAUNCH || c.driver == FST_DRIVER_PERSISTENT) && c.grid >= 0 && c.density > 0)
      g_tune[key] = c;
  }
  fclose(fh);
}

void tune_store_file(const std::string& key, const TuneConf& c) {
  const char* path = getenv("FSTGPU_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* fh = fopen(path, "a");
  if (!fh) return;
  fprintf(fh, "%s\t%d\t%d\t%d\t%.6f\n", key.c_str(), c.driver, c.grid, c.density, c.ms);
  fclose(fh);
}

std::string tune_key(const fst_plan_s* P) {
  int dev = 0;
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  else (void)cudaGetLastError();
  for (char& ch : name)
    if (ch == '\t' || ch == '\n') ch = ' ';
  const fst_s* f = P->fst;
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|Q=%d|A=%lld|m=%d|B=%d|N=%lld|T=%d|waves=%d|%s", name.c_str(), f->Q,
           (long long)f->A, f->m, P->B, (long long)P->N, P->max_len, (int)P->waves.size(),
           P->want_vit ? (P->want_fb ? "both" : "viterbi") : "forward-backward");
  return buf;
}
}  // namespace

// One run of the plan's own passes (Viterbi and/or forward-backward with
// counts) into scratch outputs, timed with CUDA events on `s`.
static int tune_time(fst_plan_s* P, cudaStream_t s, int reps, float* d_scores, int32_t* d_paths, int32_t* d_status,
                     double* d_logz, float* d_counts, double* ms_out) {
  cudaEvent_t e0, e1;
  FST_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "cudaEventCreate");
  }
  int rc = FST_OK;
  float best = 1e30f;
  for (int r = 0; r < reps + 1 && !rc; ++r) {
    cudaEventRecord(e0, s);
    if (P->want_vit) rc = fst_plan_viterbi(P, d_scores, d_paths, nullptr, d_status, s);
    if (!rc && P->want_fb) rc = fst_plan_forward_backward(P, nullptr, d_logz, d_counts, d_status, s);
    cudaEventRecord(e1, s);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { rc = cuda_fail(e, "autotune run"); break; }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (r > 0) best = std::min(best, t);  // the first run warms the caches
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = best;
  return rc;
}

extern "C" int fst_plan_autotune(fst_plan_t* P, void* stream, int32_t flags, int32_t* driver, int32_t* grid_blocks,
                                 double* best_ms) {
  if (!P || (flags & ~FST_TUNE_REFRESH)) { set_error("fst_plan_autotune: bad arguments"); return FST_ERR_INVALID_ARG; }
  if (!P->parts.empty()) { set_error("fst_plan_autotune: a plan of several parts is not tuned"); return FST_ERR_UNSUPPORTED; }
  cudaStream_t s = as_stream(stream);
  const std::string key = tune_key(P);
  TuneConf best;
  bool have = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_file();
    auto it = g_tune.find(key);
    if (it != g_tune.end() && !(flags & FST_TUNE_REFRESH)) {
      best = it->second;
      have = true;
    }
  }
  int rc = FST_OK;
  if (!have) {
    // scratch outputs of the candidate runs
    fst_s* f = P->fst;
    float *d_scores = nullptr, *d_counts = nullptr;
    int32_t *d_paths = nullptr, *d_status = nullptr;
    double* d_logz = nullptr;
    const bool prof = P->prof.on;
    P->prof.on = false;
    const uint32_t extra = P->barrier_extra;
    P->barrier_extra = 0;
    const TuneConf saved{P->driver, P->persist_grid, P->density, 0.0};
    do {
      if ((rc = dalloc(&d_status, P->B)) || (rc = dalloc(&d_scores, P->B)) || (rc = dalloc(&d_paths, P->N)) ||
          (rc = dalloc(&d_logz, P->B)) || (rc = dalloc(&d_counts, f->A)))
        break;
      std::vector<TuneConf> cands;
      for (int32_t d : {16, 64, 256}) cands.push_back(TuneConf{FST_DRIVER_LAUNCH, 0, d, 0.0});
      int dev = 0, coop = 0;
      if (cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop) {
        const int cap = std::min(persist_grid_limit(0), std::min(persist_grid_limit(1), persist_grid_limit(2)));
        std::vector<int32_t> grids;
        for (int k = 1; k * f->num_sms <= cap; ++k) grids.push_back(k * f->num_sms);
        if (cap > 0) grids.push_back(cap);
        int32_t est = 1;
        for (const Wave& w : P->waves) est = std::max(est, w.grid_est);
        if (cap > 0) grids.push_back(std::min(est, cap));
        std::sort(grids.begin(), grids.end());
        grids.erase(std::unique(grids.begin(), grids.end()), grids.end());
        for (int32_t g : grids) cands.push_back(TuneConf{FST_DRIVER_PERSISTENT, g, 64, 0.0});
      } else {
        (void)cudaGetLastError();
      }
      best.ms = 1e30;
      for (TuneConf& c : cands) {
        P->driver = c.driver;
        P->persist_grid = c.grid;
        P->density = c.density;
        if ((rc = tune_time(P, s, 2, d_scores, d_paths, d_status, d_logz, d_counts, &c.ms))) break;
        if (c.ms < best.ms) best = c;
      }
    } while (0);
    dfree(d_scores); dfree(d_paths); dfree(d_status); dfree(d_logz); dfree(d_counts);
    P->prof.on = prof;
    P->barrier_extra = extra;
    if (rc) {
      P->driver = saved.driver;
      P->persist_grid = saved.grid;
      P->density = saved.density;
      return rc;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = best;
    tune_store_file(key, best);
  }
  P->driver = best.driver;
  P->persist_grid = best.grid;
  P->density = best.density;
  if (driver) *driver = best.driver;
  if (grid_blocks) *grid_blocks = best.driver == FST_DRIVER_PERSISTENT ? best.grid : 0;
  if (best_ms) *best_ms = best.ms;
  return FST_OK;
}

extern "C" int fst_plan_get_driver(const fst_plan_t* P, int32_t* driver, int32_t* grid_blocks) {
  if (!P) { set_error("plan is NULL"); return FST_ERR_INVALID_ARG; }
  if (driver) *driver = P->driver;
  if (grid_blocks) {
    int32_t g = 0;
    if (P->driver == FST_DRIVER_PERSISTENT)
      for (const Wave& w : P->waves) g = std::max(g, persist_grid(P, w, 1));
    *grid_blocks = g;
  }
  return FST_OK;
}

extern "C" int fst_plan_fault_inject(fst_plan_t* P, int32_t kind, int64_t value) {
  if (!P || kind < FST_FAULT_NONE || kind > FST_FAULT_BARRIER_STALL || value < 0 || value > 1024) {
    set_error("fst_plan_fault_inject: bad arguments");
    return FST_ERR_INVALID_ARG;
  }
  P->barrier_extra = kind == FST_FAULT_BARRIER_STALL ? (uint32_t)value : 0u;
  for (fst_plan_s* q : P->parts) q->barrier_extra = P->barrier_extra;
  return FST_OK;
}

extern "C" int fst_plan_profile(fst_plan_t* P, int32_t enable) {
  if (!P) { set_error("plan is NULL"); return FST_ERR_INVALID_ARG; }
  P->prof.on = enable != 0;
  P->prof.used = 0;
  for (fst_plan_s* q : P->parts) {
    q->prof.on = P->prof.on;
    q->prof.used = 0;
  }
  return FST_OK;
}

extern "C" int fst_plan_profile_read(fst_plan_t* P, double* ms_by_kind, int64_t* launches_by_kind) {
  if (!P) { set_error("plan is NULL"); return FST_ERR_INVALID_ARG; }
  double ms[FST_PROF_KINDS];
  int64_t n[FST_PROF_KINDS];
  int rc = P->prof.read(ms, n);
  for (fst_plan_s* q : P->parts) {
    double qm[FST_PROF_KINDS];
    int64_t qn[FST_PROF_KINDS];
    if (rc || (rc = q->prof.read(qm, qn))) return rc;
    for (int k = 0; k < FST_PROF_KINDS; ++k) {
      ms[k] += qm[k];
      n[k] += qn[k];
    }
  }
  for (int k = 0; k < FST_PROF_KINDS; ++k) {
    if (ms_by_kind) ms_by_kind[k] = ms[k];
    if (launches_by_kind) launches_by_kind[k] = n[k];
  }
  return rc;
}

extern "C" int fst_set_batch_budget(fst_t* f, int64_t mem_budget_bytes) {
  if (!f || mem_budget_bytes < 0) { set_error("fst_set_batch_budget: bad arguments"); return FST_ERR_INVALID_ARG; }
  f->batch_budget = mem_budget_bytes;
  return FST_OK;
}
