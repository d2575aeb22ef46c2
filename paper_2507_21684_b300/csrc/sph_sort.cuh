// Device-side building blocks of the cell-structure rebuild (cell keys, radix-sort tiles,
// permute), shared by the stand-alone kernels of sph_kernels.cu and the single-launch rebuild of
// sph_rebuild.cu.
#pragma once
#include "sph_device.cuh"

namespace sph {

// Coordinate q of x = hi + lo folded into the primary box, rounded to FP32, and the fold offset
// o = L floor((x - lo_box) / L) (decided in FP64; in_primary_box() settles the common case 0
// without the FP64 division and gives the same result).  With o = 0 the result is hi + lo rounded
// once to FP32, which one FP32 addition gives exactly (IEEE addition rounds the exact sum; B300's
// FP64 rate is low, and this runs for every particle of every rebuild).
__device__ __forceinline__ float fold_coord(const DevSeg& s, int q, float hi, float lo, double* o_out) {
  if (!((s.periodic_mask >> q) & 1) || in_primary_box(s, q, hi)) {
    *o_out = 0.0;
    return __fadd_rn(hi, lo);
  }
  const double x = __dadd_rn((double)hi, (double)lo);
  const double f = floor(__ddiv_rn(__dsub_rn(x, s.lo_d[q]), s.L_d[q]));
  const double o = __dmul_rn(s.L_d[q], f);
  *o_out = o;
  return (float)__dsub_rn(x, o);
}

// Cell key of particle i, decided in FP64 from x = hi + lo exactly as floor(((x wrapped) - lo) /
// cell edge), clamped to the grid.  Fast path: an FP32 estimate from hi alone decides the floor
// whenever it lies farther than a margin from an integer; the margin, 2^-18 (|x| + |lo|) /
// cell edge + 2^-18, exceeds the estimate's error (five FP32 roundings, and |lo part| <= 2^-24
// |hi|) by more than ten times, so the FP64 decision is only taken near a cell face (and for
// NaN or huge coordinates).  Both paths give the same key.
// XB: the key with the particle's x sub-bin, cell * kXBins + bin, the bin taken from the position
// folded into the box exactly as the permute folds it (fold_coord), so the sorted cells are
// ordered by sub-bin as the sweep's x windows see them.
template <int D, bool XB = false>
__device__ __forceinline__ uint32_t cell_key_of(const DevSeg* __restrict__ segs, const Arrays& a, int i) {
  const DevSeg& s = segs[a.meta[i].y];
  Cold c = load_cold<D>(a, i);
  int cc3[3] = {0, 0, 0};
  bool fast = true;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float d = c.hi[k] - s.lo[k];
    const float mag = fabsf(c.hi[k]) + fabsf(s.lo[k]);
    if ((s.periodic_mask >> k) & 1) fast = fast && in_primary_box(s, k, c.hi[k]);  // no wrap
    const float t = d * s.invcs[k];
    const float f = floorf(t);
    const float fr = t - f;
    const float mt = 0x1p-18f * fmaf(mag, s.invcs[k], 1.f);
    fast = fast && fr >= mt && fr <= 1.f - mt && fabsf(t) < 0x1p30f;
    cc3[k] = fast ? min(max((int)f, 0), s.n[k] - 1) : 0;
  }
  if (!fast) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double x = __dadd_rn((double)c.hi[k], (double)c.lo[k]);
      double xw = x;
      if ((s.periodic_mask >> k) & 1) {
        double f = floor(__ddiv_rn(__dsub_rn(x, s.lo_d[k]), s.L_d[k]));
        xw = __dsub_rn(x, __dmul_rn(s.L_d[k], f));
      }
      double cc = floor(__ddiv_rn(__dsub_rn(xw, s.lo_d[k]), s.cs_d[k]));
      cc = fmin(fmax(cc, 0.0), (double)(s.n[k] - 1));
      cc3[k] = (int)cc;
    }
  }
  const uint32_t key = (uint32_t)(s.cell_base + (cc3[2] * s.n[1] + cc3[1]) * s.n[0] + cc3[0]);
  if (!XB) return key;
  double o;
  const float xh = fold_coord(s, 0, c.hi[0], c.lo[0], &o);
  const int b = min(max(line_xbin<kXBins>(s, xh) - cc3[0] * kXBins, 0), kXBins - 1);
  return key * kXBins + (uint32_t)b;
}

// ---- stable LSD radix sort, 8-bit digits, 2048-key tiles ---------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortIPT = 8;
constexpr int kSortTile = kSortThreads * kSortIPT;

// Histogram of one digit over sort tile `tile` (2048 keys), 256 threads; h: 256 words of shared
// memory.  KEYS_FROM_STATE: the keys are the cell keys of the current storage order (2: with x
// sub-bins), computed here (first pass of a rebuild) instead of read; with kcache they are also
// stored there, for the pass's scatter in a later launch.
template <int D, int KEYS_FROM_STATE>
__device__ __forceinline__ void sort_hist_tile(int tile, const uint32_t* __restrict__ keys, int N, int shift,
                                               uint32_t* __restrict__ hist, int nblocks,
                                               const DevSeg* __restrict__ segs, const Arrays& a, uint32_t* h,
                                               uint32_t* kcache = nullptr) {
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = tile * kSortTile;
#pragma unroll
  for (int k = 0; k < kSortIPT; ++k) {
    int i = base + k * kSortThreads + threadIdx.x;
    if (i < N) {
      const uint32_t key = KEYS_FROM_STATE ? cell_key_of<D, KEYS_FROM_STATE == 2>(segs, a, i) : keys[i];
      if (KEYS_FROM_STATE && kcache) kcache[i] = key;
      atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + tile] = h[threadIdx.x];
}

// Shared memory of one scatter tile.
struct ScatterSmem {
  uint32_t cnt[kSortThreads / 32][257];
  uint32_t goff[256];
};

// Scatter of sort tile `tile` with stable ranks: warp w owns the contiguous sub-tile
// [w*256, w*256+256) and walks it in 8 rounds of 32; within a round, equal digits are ranked by
// lane via match_any.  hist holds the exclusive offsets of (digit, tile).  256 threads.
// KEYS_FROM_STATE: the first pass; the keys come from kcache (stored by the histogram launch) or,
// without it, are computed again from the state.
template <int D, int KEYS_FROM_STATE>
__device__ __forceinline__ void sort_scatter_tile(int tile, const uint32_t* __restrict__ kin,
                                                  const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                                                  uint32_t* __restrict__ vout, int N, int shift,
                                                  const uint32_t* __restrict__ hist, int nblocks,
                                                  const DevSeg* __restrict__ segs, const Arrays& a, ScatterSmem& sm,
                                                  const uint32_t* __restrict__ kcache = nullptr) {
  constexpr int W = kSortThreads / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < W * 257; k += kSortThreads) (&sm.cnt[0][0])[k] = 0;
  sm.goff[threadIdx.x] = hist[threadIdx.x * nblocks + tile];
  __syncthreads();
  uint32_t kk[kSortIPT], vv[kSortIPT], rk[kSortIPT];
  const int base = tile * kSortTile + w * 32 * kSortIPT;
#pragma unroll
  for (int r = 0; r < kSortIPT; ++r) {
    int i = base + r * 32 + lane;
    bool ok = i < N;
    if (KEYS_FROM_STATE) {
      kk[r] = ok ? (kcache ? kcache[i] : cell_key_of<D, KEYS_FROM_STATE == 2>(segs, a, i)) : 0u;
      vv[r] = (uint32_t)i;
    } else {
      kk[r] = ok ? kin[i] : 0u;
      vv[r] = ok ? vin[i] : 0u;
    }
    uint32_t dg = ok ? ((kk[r] >> shift) & 255u) : 256u;
    uint32_t peers = __match_any_sync(kFull, dg);
    uint32_t before = __popc(peers & ((1u << lane) - 1u));
    rk[r] = sm.cnt[w][dg] + before;
    __syncwarp();
    if (before == 0) sm.cnt[w][dg] += __popc(peers);
    __syncwarp();
    rk[r] |= dg << 20;  // keep the digit beside the warp-local rank (rank < 256 per warp)
  }
  __syncthreads();
  // exclusive prefix over warps for each digit (thread t handles digit t)
  {
    uint32_t run = 0;
    for (int q = 0; q < W; ++q) {
      uint32_t c = sm.cnt[q][threadIdx.x];
      sm.cnt[q][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortIPT; ++r) {
    uint32_t dg = rk[r] >> 20;
    if (dg < 256u) {
      uint32_t pos = sm.goff[dg] + sm.cnt[w][dg] + (rk[r] & 0xfffffu);
      kout[pos] = kk[r];
      vout[pos] = vv[r];
    }
  }
}

// Element k (0 <= k <= N) of the sorted keys writes the CSR offsets of the cells in
// (key[k-1], key[k]] (off[c] = first index with key >= c).
__device__ __forceinline__ void cell_offsets_one(int k, int N, const uint32_t* __restrict__ keys, int C,
                                                 int* __restrict__ off) {
  const int lo = (k == 0) ? 0 : (int)keys[k - 1] + 1;
  const int hi = (k < N) ? (int)keys[k] : C;
  for (int c = lo; c <= hi; ++c) off[c] = k;
}

// Gather element k of the sorted state and re-fold its position into the primary box; element k
// (0 <= k <= N) also writes the cells' CSR offsets (cell_offsets_one) and, when xb is set, the
// folded position (the reference of the displacement check).  boff set: the keys carry x
// sub-bins; off gets the offsets of the cells (keys >> kXShift), boff those of the sub-bins.
template <int D>
__device__ __forceinline__ void permute_one(int k, const DevSeg* __restrict__ segs, int N,
                                            const uint32_t* __restrict__ perm, const Arrays& in, const Arrays& out,
                                            const uint32_t* __restrict__ keys, int C, int* __restrict__ off,
                                            float4* __restrict__ xb, int* __restrict__ boff = nullptr) {
  if (boff) {
    cell_offsets_one(k, N, keys, C * kXBins, boff);
    const int lo = (k == 0) ? 0 : (int)(keys[k - 1] >> kXShift) + 1;
    const int hi = (k < N) ? (int)(keys[k] >> kXShift) : C;
    for (int c = lo; c <= hi; ++c) off[c] = k;
  } else {
    cell_offsets_one(k, N, keys, C, off);
  }
  if (k >= N) return;
  int src = (int)perm[k];
  uint2 m = in.meta[src];
  const DevSeg& s = segs[m.y];
  float4 a = in.A[src], b = in.B[src];
  Cold c = load_cold<D>(in, src);
  float xh[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < D; ++q) {
    double o;
    xh[q] = fold_coord(s, q, c.hi[q], c.lo[q], &o);
    c.off[q] = (float)o;
  }
  if (D == 2) {
    out.A[k] = make_float4(xh[0], xh[1], a.z, a.w);
    if (xb) xb[k] = make_float4(xh[0], xh[1], 0.f, 0.f);
  } else {
    out.A[k] = make_float4(xh[0], xh[1], xh[2], a.w);
    out.C[k] = in.C[src];
    if (xb) xb[k] = make_float4(xh[0], xh[1], xh[2], 0.f);
  }
  store_cold<D>(out, k, c);
  out.B[k] = b;
  out.meta[k] = m;
}

// Copy of element k of every state array.
template <int D>
__device__ __forceinline__ void copy_state_one(int k, const Arrays& src, const Arrays& dst) {
  dst.A[k] = src.A[k];
  dst.B[k] = src.B[k];
  dst.X[k] = src.X[k];
  dst.O[k] = src.O[k];
  dst.meta[k] = src.meta[k];
  if (D == 3) {
    dst.C[k] = src.C[k];
    dst.XL[k] = src.XL[k];
  }
}

}  // namespace sph
