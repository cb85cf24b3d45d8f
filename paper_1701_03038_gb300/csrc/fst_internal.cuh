// fst_internal.cuh -- shared definitions of the fstgpu CUDA library.
//
// Arc store (built once per FST on the device, Sec. 4 / Fig. 2 redesigned):
// the arcs of every input symbol a (the slice delta[a], R[a]..R[a+1]-1 in
// the paper) are sorted by (segment state, arc id) and cut into segments of
// equal segment state.  Two layouts exist:
//   forward  -- segments by destination (the column-major / CSC reading of
//               Sec. 4: one reduction per destination state), arcs carry src;
//   backward -- segments by source, arcs carry dst.
// Segments are packed into windows of WIN = 128 arcs.  A segment never
// straddles a window unless it is longer than WIN ("long" segment): then it
// starts on a window boundary and owns whole windows.  The tail of a window
// is padded with arcs of weight -inf.  Each window has a 128-bit head mask
// (bit i set = arc i starts a segment) and the index of its first segment;
// the windows serve the float64 check kernels (fd64.cu).  The step kernels
// use the backward layout only, through its packed 16-byte arc records and
// a (symbol, state) hash of its segments.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "fstgpu.h"

namespace fstgpu {

constexpr int WARP = 32;
constexpr int APL = 4;            // arcs per lane
constexpr int WIN = WARP * APL;   // arcs per window
constexpr unsigned FULL = 0xffffffffu;

// Window metadata, 32 bytes: two 16-byte loads.
struct __align__(16) WinMeta {
  int32_t seg;     // first segment starting in this window (or the long segment)
  int32_t lseg;    // long windows: slice-local index of the long segment; -1 otherwise
  int32_t lwin0;   // long windows: slice-local index of the segment's first long window
  int32_t lcnt;    // long windows: number of windows of the segment
  uint32_t mask[4];
};

struct Layout {
  int64_t P = 0;         // padded arcs = nwin * WIN
  int64_t nwin = 0;
  int64_t nseg = 0;
  int32_t* other = nullptr;   // [P] gathered state (src for forward, dst for backward); 0 on padding
  float* theta = nullptr;     // [P] log-weight; -inf on padding
  int32_t* arc_id = nullptr;  // [P] caller arc id; -1 on padding
  double* theta64 = nullptr;  // [P] optional float64 weights (finite-difference variant)
  WinMeta* win = nullptr;     // [nwin]
  int32_t* seg_state = nullptr;  // [nseg] dst (forward) / src (backward)
  int32_t* seg_pos = nullptr;    // [nseg] padded start position
  int32_t* seg_len = nullptr;    // [nseg] arcs in the segment
  // (symbol, state) -> arcs of the segment, open addressing: slot = {key,
  // len << 32 | first position}; key = symbol << 32 | state, empty slots
  // hold ~0 (source-segmented layout only)
  ulonglong2* seg_hash = nullptr;
  // [P] the arcs packed for one 16-byte load each: {other, theta bits,
  // caller id, 0} (source-segmented layout only)
  int4* arcs = nullptr;
  int64_t hash_mask = 0;
  int64_t* sym_win = nullptr;    // [m+1]
  int64_t* sym_seg = nullptr;    // [m+1]
  int64_t* sym_lseg = nullptr;   // [m+1] long segments
  int64_t* sym_lwin = nullptr;   // [m+1] long windows
  // host copies
  int64_t* h_sym_win = nullptr;
  int64_t* h_sym_seg = nullptr;
  int64_t* h_sym_lseg = nullptr;
  int64_t* h_sym_lwin = nullptr;
};

// Per-launch timing (the tracing subsystem): with `on`, every launch that a
// run brackets with begin/end gets two CUDA events on its stream; read()
// waits for the last one and sums device milliseconds and launches per
// kernel kind (FST_PROF_*), then starts over.
struct LaunchProfile {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  size_t used = 0;
  ~LaunchProfile() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  long begin(int k, cudaStream_t s) {
    if (!on) return -1;
    const size_t i = used;
    while (ev.size() < 2 * (i + 1)) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      ev.push_back(e);
    }
    if (kind.size() < i + 1) kind.resize(i + 1);
    kind[i] = k;
    cudaEventRecord(ev[2 * i], s);
    used = i + 1;
    return (long)i;
  }
  void end(long i, cudaStream_t s) {
    if (i >= 0) cudaEventRecord(ev[2 * i + 1], s);
  }
  // ms_by_kind / launches_by_kind: FST_PROF_KINDS entries each, or NULL
  int read(double* ms_by_kind, int64_t* launches_by_kind);
};

}  // namespace fstgpu

struct fst_s {
  int32_t Q = 0;
  int64_t A = 0;
  int32_t m = 0;
  int device = 0;
  int num_sms = 0;
  fstgpu::Layout fwd, bwd;
  float* theta_s = nullptr;    // [Q]
  float* theta_f = nullptr;    // [Q]
  int32_t* start_q = nullptr;  // [nstart] states with a finite start weight
  int32_t nstart = 0;
  int32_t* olabel = nullptr;   // [A] by caller arc id
  int32_t* src_by_id = nullptr;  // [A] source state by caller arc id
  int64_t* sym_arc = nullptr;  // [m+1] R offsets (device)
  int64_t* h_sym_arc = nullptr;
  int32_t max_seg_len = 0;
  // per-handle state for the single-string calls
  struct PlainWs* plain = nullptr;
  // launch timing of the single-string calls (fst_profile)
  fstgpu::LaunchProfile prof;
  // the last plan of each batch call kind (Viterbi, forward-backward), whose
  // storage the next call of that kind takes over
  struct fst_plan_s* batch_plan[2] = {nullptr, nullptr};
  int64_t batch_budget = 0;  // plan storage budget of the batch calls (0 = the plan default)
  int32_t batch_parts[2] = {0, 0};  // fst_set_batch_plan: parts of the Viterbi / FB batch plans (0 = by size)
  int32_t batch_layout = -1;        // accumulators of the batch plans: -1 by budget, 0 compact, 1 dense
  int32_t batch_graph = 0;          // batch runs recorded into a CUDA graph and launched: 0 never, 1 always
  // an output-clamped FST (fst_create_clamped): the (input, output) label
  // pair of each of its input symbols, ((uint64)ilabel << 32 | olabel), sorted
  std::vector<uint64_t>* pair_keys = nullptr;
  std::mutex* batch_mu = nullptr;
  // the paper's slice-wide relaxation (fst_viterbi_slice): per-arc records
  // {src, dst, id} in the destination-segmented layout's order, and the
  // packed keys of every position of the last string
  int4* slice_arcs = nullptr;      // in the destination-segmented (column-major) order
  int4* slice_arcs_src = nullptr;  // in the source-segmented (row-major) order
  int32_t slice_order = 0;         // FST_SLICE_BY_DESTINATION or FST_SLICE_BY_SOURCE
  unsigned long long* slice_keys = nullptr;
  int64_t slice_cap = 0;
  float* slice_fb = nullptr;       // forward and backward tables of fst_forward_backward_slice
  int64_t slice_fb_cap = 0;
  int32_t* slice_out = nullptr;    // slice Viterbi outputs: score, path and output labels
  int64_t slice_out_cap = 0;
  // one-block kernels (block.cu): the string and its outputs; backpointers
  // or forward values
  int32_t* block_ids = nullptr;
  int64_t block_ids_cap = 0;
  unsigned long long* block_ws = nullptr;
  int64_t block_ws_cap = 0;
  // single-string Viterbi: frontier kernels, the slice-wide kernel, or the
  // cheaper of the two by a cost model fitted by fst_autotune_plain
  int32_t plain_method = 0;
  int32_t plain_fb_driver = 0;   // single-string forward-backward: FST_DRIVER_LAUNCH or _PERSISTENT
  int32_t plain_fb_grid = 0;     // persistent grid (0 = one block per SM)
  bool plain_tuned = false;
  bool plain_block = false;  // FST_PLAIN_AUTO, calibrated: the one-block kernels for both calls
  double plain_coef[5] = {0, 0, 0, 0, 0};  // frontier d0 + d1 n; slice c0 + c1 n + c2 (slice arcs)
};

namespace fstgpu {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
#define FST_CUDA(call)                                          \
  do {                                                          \
    cudaError_t e__ = (call);                                   \
    if (e__ != cudaSuccess) return ::fstgpu::cuda_fail(e__, #call); \
  } while (0)

// ------------------------------------------------------------ device math
// Order-preserving map float -> uint32 (total order, -0 < +0).
__device__ __forceinline__ uint32_t fkey(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}
constexpr uint32_t FKEY_NEG_INF = 0x007fffffu;  // fkey(-inf)

// Order-preserving map float64 -> uint64 (as fkey for float32); no finite
// value or -inf maps to 0, which therefore means "nothing yet".
__device__ __forceinline__ unsigned long long dkey(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  const unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)u);
}

// exp(v - m), v <= m, as a 2^-40 fixed-point integer: sums of these are exact
// and so independent of the order in which they are added.  A sum of fewer
// than 2^24 terms cannot overflow (the store refuses longer segments).  The
// value and the maximum m are float64: the forward and backward values
// carried from position to position are float64 (a float32 value rounds by
// up to 2^-24 of its size at every position, and over a 200-position string
// those roundings shift alpha + beta - log Z by ~1e-5, the whole posterior
// tolerance), and so is the term, whose relative error would otherwise add
// to the same drift.  The maximal term is exactly 2^40 and costs no
// exponential (most destinations of a sparse frontier have one live arc;
// float64 arithmetic is scarce on this GPU).
__device__ __forceinline__ unsigned long long fix_exp64(double v, double m) {
  if (v == -INFINITY) return 0ull;
  if (v == m) return 1099511627776ull;  // 2^40
  return __double2ull_rn(exp(v - m) * 1099511627776.0);
}
// -inf tests on the bit patterns: integer compares (a float64 compare takes
// the float64 pipe, narrow on this part).
__device__ __forceinline__ bool dead64(double v) { return __double_as_longlong(v) == (long long)0xfff0000000000000ull; }
__device__ __forceinline__ bool dead32(float v) { return __float_as_uint(v) == 0xff800000u; }

// m + log(s / 2^40), in float64.  A sum that is the maximal term alone
// (s = 2^40, the usual case on a sparse frontier: one live arc into the
// state) is m itself and takes no logarithm.
__device__ __forceinline__ double fix_log_sum64(double m, unsigned long long s) {
  if (__double_as_longlong(m) == (long long)0xfff0000000000000ull || s == 0ull) return -INFINITY;
  return s == 1099511627776ull ? m : m + log((double)s * 0x1p-40);
}


// ------------------------------------------------------------ primitives
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the key.
int radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s);
// Exclusive scan of n int64 values (out may alias in); *total gets the sum (host).
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, cudaStream_t s);
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);

// Slot of key k in a power-of-two table (Fibonacci hashing).
__host__ __device__ __forceinline__ uint64_t seg_hash_slot(uint64_t k, int64_t mask) {
  return (k * 0x9E3779B97F4A7C15ull >> 17) & (uint64_t)mask;
}
__host__ __device__ __forceinline__ uint64_t seg_hash_key(int32_t sym, int32_t state) {
  return ((uint64_t)(uint32_t)sym << 32) | (uint64_t)(uint32_t)state;
}

// Device memory helpers (plain cudaMalloc; every buffer is owned by a handle).
template <class T>
int dalloc(T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, (size_t)n * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    set_error("cudaMalloc of %lld bytes failed: %s", (long long)((size_t)n * sizeof(T)),
              cudaGetErrorString(e));
    return FST_ERR_OOM;
  }
  return FST_OK;
}
template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// ------------------------------------------------------------ arc store
int build_store(fst_s* f, const int32_t* d_src, const int32_t* d_dst, const int32_t* d_il,
                const float* d_theta, cudaStream_t s);
void free_layout(Layout& L);
int set_layout_weights(fst_s* f, const float* d_theta_by_id, cudaStream_t s);
int set_layout_weights64(fst_s* f, const double* d_theta_by_id, cudaStream_t s);

int grid_for(int64_t work_warps, int block_threads, int num_sms, int max_blocks_per_sm);

// Every arc of every slice as one record {source, destination, id} (id -1 on
// padding) with its log-weight, in the order fst_set_slice_order chose;
// symbol a's records are [h_sym_win[a] * WIN, h_sym_win[a+1] * WIN).  Built
// on first use (slice.cu).
struct SliceView {
  const int4* arcs;
  const float* theta;
  const int64_t* h_sym_win;
};
int slice_view(fst_s* f, cudaStream_t s, SliceView* out);
// The destination-ordered slice records (fst_s::slice_arcs), built on first
// use whatever order the slice kernels are set to.
int slice_records_dst(fst_s* f, cudaStream_t s);

// Viterbi of one string by the paper's slice-wide relaxation (slice.cu);
// host outputs, olabels may be NULL.
int viterbi_slice_run(fst_s* f, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path,
                      int32_t* olabels);

// One string in one thread block (block.cu), for FSTs of at most
// BLOCK_QMAX states, host outputs: Viterbi (olabels may be NULL; *status
// FST_OK or FST_ERR_NO_PATH) and forward-backward (arc_posteriors [A] or
// NULL, log Z, *status).
constexpr int32_t BLOCK_QMAX = FST_BLOCK_MAX_STATES;
bool block_fits(const fst_s* f);
int viterbi_block_run(fst_s* f, const int32_t* ids, int32_t n, float* best_score, int32_t* arc_path,
                      int32_t* olabels, int32_t* status);
int fb_block_run(fst_s* f, const int32_t* ids, int32_t n, float* arc_posteriors, double* log_z, int32_t* status);

// Input label, destination and log-weight of every arc by caller id (any
// output may be NULL; train.cu).
int arcs_by_id(fst_s* f, int32_t* il, int32_t* dst, float* th, cudaStream_t s);

}  // namespace fstgpu
