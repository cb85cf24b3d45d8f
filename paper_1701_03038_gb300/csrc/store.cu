// store.cu -- building the device arc store of an FST.
//
// The paper keeps the arcs of each input symbol contiguous (the CSR offsets
// R over symbols with COO arrays S, T, O, P; Sec. 4, Fig. 2) and sorts each
// slice by source and then target (Sec. 5).  Here each slice is instead
// sorted by (segment state, arc id) on the device -- destination for the
// forward layout, source for the backward layout -- and packed into
// 128-arc windows (their head masks serve the float64 check kernels).  The
// backward layout also gets packed 16-byte arc records and a (symbol,
// state) hash of its segments, which the step kernels read.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "fst_internal.cuh"

namespace fstgpu {
namespace {

constexpr int TB = 256;

inline unsigned blocks_for(int64_t n, int tb = TB) {
  int64_t b = (n + tb - 1) / tb;
  if (b < 1) b = 1;
  return (unsigned)b;
}

inline int bits_for(int64_t maxval) {  // bits needed for values in [0, maxval]
  int b = 0;
  while (b < 63 && ((int64_t)1 << b) <= maxval) ++b;
  return b;
}

__global__ void k_make_keys(const int32_t* __restrict__ il, const int32_t* __restrict__ st, int64_t A,
                            int sbits, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= A) return;
  keys[k] = ((uint64_t)(uint32_t)il[k] << sbits) | (uint64_t)(uint32_t)st[k];
  vals[k] = (uint32_t)k;
}

__global__ void k_heads(const uint64_t* __restrict__ keys, int64_t A, int64_t* __restrict__ hd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A) return;
  hd[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// For head i: record the segment's first arc, symbol and state.
__global__ void k_seg_info(const uint64_t* __restrict__ keys, const int64_t* __restrict__ hd,
                           const int64_t* __restrict__ segx, int64_t A, int sbits,
                           int64_t* __restrict__ seg_first, int32_t* __restrict__ seg_sym,
                           int32_t* __restrict__ seg_state) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A || !hd[i]) return;
  const int64_t s = segx[i];
  seg_first[s] = i;
  seg_sym[s] = (int32_t)(keys[i] >> sbits);
  seg_state[s] = (int32_t)(keys[i] & (((uint64_t)1 << sbits) - 1));
}

// sym_seg[a] = first segment whose symbol is >= a (lower bound), a in [0, m].
__global__ void k_sym_lower_bound(const int32_t* __restrict__ seg_sym, int64_t nseg, int32_t m,
                                  int64_t* __restrict__ sym_seg) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a > m) return;
  int64_t lo = 0, hi = nseg;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (seg_sym[mid] < a) lo = mid + 1; else hi = mid;
  }
  sym_seg[a] = lo;
}

// Greedy packing of one symbol's segments into windows (one thread per
// symbol).  A segment that fits in a window never straddles one; a longer
// segment starts on a boundary and owns whole windows.
__global__ void k_pack(const int64_t* __restrict__ sym_seg, const int64_t* __restrict__ seg_first,
                       int32_t m, int64_t* __restrict__ seg_ppos, int64_t* __restrict__ sym_nwin,
                       int64_t* __restrict__ is_long, int64_t* __restrict__ long_nwin,
                       int32_t* __restrict__ max_len) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= m) return;
  int64_t cur = 0;
  int64_t mx = 0;
  for (int64_t s = sym_seg[a]; s < sym_seg[a + 1]; ++s) {
    const int64_t len = seg_first[s + 1] - seg_first[s];
    mx = len > mx ? len : mx;
    const int64_t off = cur % WIN;
    if (len > WIN) {
      if (off) cur += WIN - off;
      seg_ppos[s] = cur;
      const int64_t nw = (len + WIN - 1) / WIN;
      cur += nw * WIN;
      is_long[s] = 1;
      long_nwin[s] = nw;
    } else {
      if (off + len > WIN) cur += WIN - off;
      seg_ppos[s] = cur;
      cur += len;
      is_long[s] = 0;
      long_nwin[s] = 0;
    }
  }
  sym_nwin[a] = (cur + WIN - 1) / WIN;
  atomicMax(max_len, (int32_t)(mx < 0x7fffffff ? mx : 0x7fffffff));
}

__global__ void k_fill_padding(int32_t* __restrict__ other, float* __restrict__ theta,
                               int32_t* __restrict__ id, int64_t P) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  other[i] = 0;
  theta[i] = -INFINITY;
  id[i] = -1;
}

__global__ void k_seg_pos(const int32_t* __restrict__ seg_sym, const int64_t* __restrict__ seg_ppos,
                          const int64_t* __restrict__ sym_win, int64_t nseg, int32_t* __restrict__ seg_pos) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  seg_pos[s] = (int32_t)(sym_win[seg_sym[s]] * WIN + seg_ppos[s]);
}

__global__ void k_seg_len(const int64_t* __restrict__ seg_first, int64_t nseg, int32_t* __restrict__ len) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nseg) len[s] = (int32_t)(seg_first[s + 1] - seg_first[s]);
}

// Insert every segment (symbol, state) -> (first position, length) into the
// open-addressing table; one thread per segment.
__global__ void k_hash_insert(const int64_t* __restrict__ sym_seg, int32_t m, const int32_t* __restrict__ seg_state,
                              const int32_t* __restrict__ seg_pos, const int32_t* __restrict__ seg_len,
                              int64_t nseg, ulonglong2* __restrict__ tab, int64_t mask) {
  const int64_t sg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sg >= nseg) return;
  int32_t lo = 0, hi = m;  // symbol of segment sg: last a with sym_seg[a] <= sg
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (sym_seg[mid] <= sg) lo = mid; else hi = mid;
  }
  const uint64_t k = seg_hash_key(lo, seg_state[sg]);
  uint64_t h = seg_hash_slot(k, mask);
  for (int64_t probe = 0; probe <= mask; ++probe) {
    const unsigned long long old = atomicCAS(&tab[h].x, ~0ull, (unsigned long long)k);
    if (old == ~0ull || old == k) {
      tab[h].y = ((unsigned long long)(uint32_t)seg_len[sg] << 32) | (unsigned long long)(uint32_t)seg_pos[sg];
      return;
    }
    h = (h + 1) & (uint64_t)mask;
  }
}

__global__ void k_scatter_arcs(const uint32_t* __restrict__ perm, const int64_t* __restrict__ hd,
                               const int64_t* __restrict__ segx, const int64_t* __restrict__ seg_first,
                               const int32_t* __restrict__ seg_pos, const int32_t* __restrict__ oth_by_id,
                               const float* __restrict__ th_by_id, int64_t A, int32_t* __restrict__ other,
                               float* __restrict__ theta, int32_t* __restrict__ id) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A) return;
  const int64_t s = segx[i] + hd[i] - 1;
  const int64_t pos = (int64_t)seg_pos[s] + (i - seg_first[s]);
  const uint32_t k = perm[i];
  other[pos] = oth_by_id[k];
  theta[pos] = th_by_id[k];
  id[pos] = (int32_t)k;
}

__global__ void k_win_init(WinMeta* __restrict__ win, int64_t nwin) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwin) return;
  WinMeta z;
  z.seg = -1; z.lseg = -1; z.lwin0 = -1; z.lcnt = 0;
  z.mask[0] = z.mask[1] = z.mask[2] = z.mask[3] = 0u;
  win[w] = z;
}

__global__ void k_win_meta(const int32_t* __restrict__ seg_pos, const int32_t* __restrict__ seg_sym,
                           const int64_t* __restrict__ is_long, const int64_t* __restrict__ long_nwin,
                           const int64_t* __restrict__ long_x, const int64_t* __restrict__ lwin_x,
                           const int64_t* __restrict__ sym_seg, int64_t nseg, WinMeta* __restrict__ win) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const int64_t pos = seg_pos[s];
  const int64_t w0 = pos / WIN;
  const int bit = (int)(pos % WIN);
  atomicOr(&win[w0].mask[bit >> 5], 1u << (bit & 31));
  if (bit == 0) win[w0].seg = (int32_t)s;
  if (is_long[s]) {
    const int64_t a = seg_sym[s];
    const int64_t s0 = sym_seg[a];
    const int32_t lseg = (int32_t)(long_x[s] - long_x[s0]);
    const int32_t lwin0 = (int32_t)(lwin_x[s] - lwin_x[s0]);
    const int64_t nw = long_nwin[s];
    for (int64_t j = 0; j < nw; ++j) {
      WinMeta* wm = &win[w0 + j];
      wm->seg = (int32_t)s;
      wm->lseg = lseg;
      wm->lwin0 = lwin0;
      wm->lcnt = (int32_t)nw;
    }
  }
}

// sym_x[a] = x[sym_seg[a]] for a in [0, m] (x has a valid entry at nseg).
__global__ void k_gather_sym(const int64_t* __restrict__ x, const int64_t* __restrict__ sym_seg, int32_t m,
                             int64_t* __restrict__ out) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a > m) return;
  out[a] = x[sym_seg[a]];
}

__global__ void k_pack_arcs(const int32_t* __restrict__ other, const float* __restrict__ theta,
                            const int32_t* __restrict__ arc_id, int64_t P, int4* __restrict__ arcs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) arcs[i] = make_int4(other[i], __float_as_int(theta[i]), arc_id[i], 0);
}

__global__ void k_set_weights(const int32_t* __restrict__ id, const float* __restrict__ th_by_id, int64_t P,
                              float* __restrict__ theta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const int32_t k = id[i];
  theta[i] = k >= 0 ? th_by_id[k] : -INFINITY;
}

__global__ void k_set_weights64(const int32_t* __restrict__ id, const double* __restrict__ th_by_id, int64_t P,
                                double* __restrict__ theta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const int32_t k = id[i];
  theta[i] = k >= 0 ? th_by_id[k] : -INFINITY;
}

int copy_to_host(int64_t** h, const int64_t* d, int64_t n) {
  *h = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!*h) { set_error("host allocation failed"); return FST_ERR_OOM; }
  FST_CUDA(cudaMemcpy(*h, d, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToHost));
  return FST_OK;
}

struct Tmp {
  uint64_t* keys = nullptr;
  uint32_t* perm = nullptr;
  int64_t* hd = nullptr;
  int64_t* segx = nullptr;
  int64_t* seg_first = nullptr;
  int32_t* seg_sym = nullptr;
  int64_t* seg_ppos = nullptr;
  int64_t* sym_nwin = nullptr;
  int64_t* is_long = nullptr;
  int64_t* long_nwin = nullptr;
  int64_t* long_x = nullptr;
  int64_t* lwin_x = nullptr;
  int32_t* max_len = nullptr;
  ~Tmp() {
    dfree(keys); dfree(perm); dfree(hd); dfree(segx); dfree(seg_first); dfree(seg_sym);
    dfree(seg_ppos); dfree(sym_nwin); dfree(is_long); dfree(long_nwin); dfree(long_x);
    dfree(lwin_x); dfree(max_len);
  }
};

// Build one layout: segments keyed by `seg_st` (dst for forward, src for
// backward); arcs carry `oth` (the state they gather from).
int build_layout(fst_s* f, Layout& L, const int32_t* d_il, const int32_t* seg_st, const int32_t* oth,
                 const float* d_theta, int64_t** h_sym_arc_out, int64_t* d_sym_arc_out, cudaStream_t s) {
  const int64_t A = f->A;
  const int32_t m = f->m;
  Tmp t;
  int rc = FST_OK;
  const int sbits = bits_for(f->Q - 1 > 0 ? f->Q - 1 : 1);
  const int lbits = bits_for(m - 1 > 0 ? m - 1 : 1);
  if (sbits + lbits > 64) { set_error("key too wide"); return FST_ERR_UNSUPPORTED; }
  if ((rc = dalloc(&t.keys, A)) || (rc = dalloc(&t.perm, A)) || (rc = dalloc(&t.hd, A)) ||
      (rc = dalloc(&t.segx, A + 1)))
    return rc;
  if (A > 0) {
    k_make_keys<<<blocks_for(A), TB, 0, s>>>(d_il, seg_st, A, sbits, t.keys, t.perm);
    if ((rc = radix_sort_pairs(t.keys, t.perm, A, sbits + lbits, s))) return rc;
    k_heads<<<blocks_for(A), TB, 0, s>>>(t.keys, A, t.hd);
  }
  int64_t nseg = 0;
  if ((rc = exclusive_scan_i64(t.hd, t.segx, A, &nseg, s))) return rc;
  L.nseg = nseg;
  if ((rc = dalloc(&t.seg_first, nseg + 1)) || (rc = dalloc(&t.seg_sym, nseg + 1)) ||
      (rc = dalloc(&L.seg_state, nseg + 1)) || (rc = dalloc(&L.sym_seg, (int64_t)m + 1)))
    return rc;
  if (A > 0)
    k_seg_info<<<blocks_for(A), TB, 0, s>>>(t.keys, t.hd, t.segx, A, sbits, t.seg_first, t.seg_sym,
                                            L.seg_state);
  FST_CUDA(cudaMemcpyAsync(t.seg_first + nseg, &A, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  k_sym_lower_bound<<<blocks_for((int64_t)m + 1), TB, 0, s>>>(t.seg_sym, nseg, m, L.sym_seg);
  // R offsets (Fig. 2): first arc of each symbol
  if (d_sym_arc_out) {
    k_gather_sym<<<blocks_for((int64_t)m + 1), TB, 0, s>>>(t.seg_first, L.sym_seg, m, d_sym_arc_out);
    if ((rc = copy_to_host(h_sym_arc_out, d_sym_arc_out, (int64_t)m + 1))) return rc;
  }
  // window packing
  if ((rc = dalloc(&t.seg_ppos, nseg + 1)) || (rc = dalloc(&t.sym_nwin, (int64_t)m + 1)) ||
      (rc = dalloc(&t.is_long, nseg + 1)) || (rc = dalloc(&t.long_nwin, nseg + 1)) ||
      (rc = dalloc(&t.max_len, 1)) || (rc = dalloc(&L.sym_win, (int64_t)m + 1)) ||
      (rc = dalloc(&t.long_x, nseg + 1)) || (rc = dalloc(&t.lwin_x, nseg + 1)) ||
      (rc = dalloc(&L.sym_lseg, (int64_t)m + 1)) || (rc = dalloc(&L.sym_lwin, (int64_t)m + 1)))
    return rc;
  FST_CUDA(cudaMemsetAsync(t.max_len, 0, sizeof(int32_t), s));
  k_pack<<<blocks_for(m, 64), 64, 0, s>>>(L.sym_seg, t.seg_first, m, t.seg_ppos, t.sym_nwin, t.is_long,
                                          t.long_nwin, t.max_len);
  int64_t nwin = 0;
  if ((rc = exclusive_scan_i64(t.sym_nwin, L.sym_win, m, &nwin, s))) return rc;
  FST_CUDA(cudaMemcpyAsync(L.sym_win + m, &nwin, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  int64_t nlong = 0, nlwin = 0;
  if ((rc = exclusive_scan_i64(t.is_long, t.long_x, nseg, &nlong, s))) return rc;
  if ((rc = exclusive_scan_i64(t.long_nwin, t.lwin_x, nseg, &nlwin, s))) return rc;
  FST_CUDA(cudaMemcpyAsync(t.long_x + nseg, &nlong, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  FST_CUDA(cudaMemcpyAsync(t.lwin_x + nseg, &nlwin, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  k_gather_sym<<<blocks_for((int64_t)m + 1), TB, 0, s>>>(t.long_x, L.sym_seg, m, L.sym_lseg);
  k_gather_sym<<<blocks_for((int64_t)m + 1), TB, 0, s>>>(t.lwin_x, L.sym_seg, m, L.sym_lwin);
  int32_t mx = 0;
  FST_CUDA(cudaMemcpyAsync(&mx, t.max_len, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FST_CUDA(cudaStreamSynchronize(s));
  f->max_seg_len = std::max(f->max_seg_len, mx);
  L.nwin = nwin;
  L.P = nwin * WIN;
  if (L.P >= ((int64_t)1 << 31) - WIN) {
    set_error("padded arc count %lld is beyond 2^31", (long long)L.P);
    return FST_ERR_UNSUPPORTED;
  }
  if ((rc = dalloc(&L.other, L.P)) || (rc = dalloc(&L.theta, L.P)) || (rc = dalloc(&L.arc_id, L.P)) ||
      (rc = dalloc(&L.seg_pos, nseg + 1)) || (rc = dalloc(&L.win, nwin)) || (rc = dalloc(&L.seg_len, nseg + 1)))
    return rc;
  if (nseg > 0) k_seg_len<<<blocks_for(nseg), TB, 0, s>>>(t.seg_first, nseg, L.seg_len);
  if (L.P > 0) k_fill_padding<<<blocks_for(L.P), TB, 0, s>>>(L.other, L.theta, L.arc_id, L.P);
  if (nseg > 0) k_seg_pos<<<blocks_for(nseg), TB, 0, s>>>(t.seg_sym, t.seg_ppos, L.sym_win, nseg, L.seg_pos);
  if (A > 0)
    k_scatter_arcs<<<blocks_for(A), TB, 0, s>>>(t.perm, t.hd, t.segx, t.seg_first, L.seg_pos, oth, d_theta,
                                                A, L.other, L.theta, L.arc_id);
  if (nwin > 0) k_win_init<<<blocks_for(nwin), TB, 0, s>>>(L.win, nwin);
  if (nseg > 0)
    k_win_meta<<<blocks_for(nseg), TB, 0, s>>>(L.seg_pos, t.seg_sym, t.is_long, t.long_nwin, t.long_x, t.lwin_x,
                                               L.sym_seg, nseg, L.win);
  FST_CUDA(cudaGetLastError());
  FST_CUDA(cudaStreamSynchronize(s));
  if ((rc = copy_to_host(&L.h_sym_win, L.sym_win, (int64_t)m + 1))) return rc;
  if ((rc = copy_to_host(&L.h_sym_seg, L.sym_seg, (int64_t)m + 1))) return rc;
  if ((rc = copy_to_host(&L.h_sym_lseg, L.sym_lseg, (int64_t)m + 1))) return rc;
  if ((rc = copy_to_host(&L.h_sym_lwin, L.sym_lwin, (int64_t)m + 1))) return rc;
  return FST_OK;
}

}  // namespace

void free_layout(Layout& L) {
  dfree(L.other); dfree(L.theta); dfree(L.arc_id); dfree(L.theta64); dfree(L.win);
  dfree(L.seg_state); dfree(L.seg_pos); dfree(L.seg_len); dfree(L.seg_hash); dfree(L.arcs); dfree(L.sym_win); dfree(L.sym_seg); dfree(L.sym_lseg);
  dfree(L.sym_lwin);
  free(L.h_sym_win); free(L.h_sym_seg); free(L.h_sym_lseg); free(L.h_sym_lwin);
  L.h_sym_win = L.h_sym_seg = L.h_sym_lseg = L.h_sym_lwin = nullptr;
  L.P = L.nwin = L.nseg = 0;
}

int build_store(fst_s* f, const int32_t* d_src, const int32_t* d_dst, const int32_t* d_il,
                const float* d_theta, cudaStream_t s) {
  int rc;
  if ((rc = dalloc(&f->sym_arc, (int64_t)f->m + 1))) return rc;
  // forward: segments by destination, arcs carry their source
  if ((rc = build_layout(f, f->fwd, d_il, d_dst, d_src, d_theta, &f->h_sym_arc, f->sym_arc, s))) return rc;
  // backward: segments by source, arcs carry their destination
  if ((rc = build_layout(f, f->bwd, d_il, d_src, d_dst, d_theta, nullptr, nullptr, s))) return rc;
  // the fixed-point sums of the step kernels add at most one term of at
  // most 2^40 per arc of a segment: 2^24 arcs would overflow 64 bits
  if (f->max_seg_len >= (1 << 24)) {
    set_error("a state has %d arcs on one symbol, beyond the 2^24 the step kernels support", f->max_seg_len);
    return FST_ERR_UNSUPPORTED;
  }
  // source state by caller arc id (the backtrace follows arc ids)
  if ((rc = dalloc(&f->src_by_id, f->A))) return rc;
  if (f->A > 0) FST_CUDA(cudaMemcpyAsync(f->src_by_id, d_src, (size_t)f->A * 4, cudaMemcpyDeviceToDevice, s));
  // (symbol, state) -> segment of the source-segmented layout: the step
  // kernels find a live state's arcs on a symbol with about one probe
  {
    Layout& L = f->bwd;
    int64_t size = 2;
    while (size < 2 * std::max<int64_t>(L.nseg, 1)) size <<= 1;
    if ((rc = dalloc(&L.seg_hash, size))) return rc;
    L.hash_mask = size - 1;
    FST_CUDA(cudaMemsetAsync(L.seg_hash, 0xff, (size_t)size * sizeof(ulonglong2), s));
    if (L.nseg > 0)
      k_hash_insert<<<blocks_for(L.nseg), TB, 0, s>>>(L.sym_seg, f->m, L.seg_state, L.seg_pos, L.seg_len, L.nseg,
                                                      L.seg_hash, L.hash_mask);
    if ((rc = dalloc(&L.arcs, L.P))) return rc;
    if (L.P > 0) k_pack_arcs<<<blocks_for(L.P), TB, 0, s>>>(L.other, L.theta, L.arc_id, L.P, L.arcs);
    FST_CUDA(cudaStreamSynchronize(s));
  }
  return FST_OK;
}

int set_layout_weights(fst_s* f, const float* d_theta_by_id, cudaStream_t s) {
  Layout* Ls[2] = {&f->fwd, &f->bwd};
  for (Layout* L : Ls) {
    if (L->P > 0) k_set_weights<<<blocks_for(L->P), TB, 0, s>>>(L->arc_id, d_theta_by_id, L->P, L->theta);
    if (L->P > 0 && L->arcs) k_pack_arcs<<<blocks_for(L->P), TB, 0, s>>>(L->other, L->theta, L->arc_id, L->P, L->arcs);
  }
  FST_CUDA(cudaGetLastError());
  return FST_OK;
}

int set_layout_weights64(fst_s* f, const double* d_theta_by_id, cudaStream_t s) {
  Layout* Ls[2] = {&f->fwd, &f->bwd};
  for (Layout* L : Ls) {
    if (!L->theta64) {
      int rc = dalloc(&L->theta64, L->P);
      if (rc) return rc;
    }
    if (L->P > 0) k_set_weights64<<<blocks_for(L->P), TB, 0, s>>>(L->arc_id, d_theta_by_id, L->P, L->theta64);
  }
  FST_CUDA(cudaGetLastError());
  return FST_OK;
}

}  // namespace fstgpu
