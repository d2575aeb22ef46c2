// Cell-block traversal with shared-memory staging (the neighbour loop of every pass).
//
// The sorted particles of one cell line (fixed y[, z] cell, x varying) are cut into tiles of at
// most TP consecutive particles; one CTA owns one tile at a time.  The CTA stages, into shared
// memory, every particle of the 3^(d-1) neighbouring lines whose x cell lies in
// [cx_first - 1, cx_last + 1] (with periodic images), as contiguous "columns" in stencil order,
// so each target particle's own 3^d cells are 3^(d-1) contiguous runs of shared memory.
// LANES threads serve one target: they split its candidates, test |r| < H, collect the hits in
// per-lane lists and evaluate the pair terms (Body::pair) from shared memory; the partial sums
// of the LANES threads are then combined with shuffles.  Tiles whose staged region would not fit
// fall back to the warp traversal on global memory.
#pragma once
#include "sph_device.cuh"

namespace sph {

// One tile: particle range [p0, p1) inside one cell line of one scene.
struct Tile {
  int p0, p1, line, seg;
};

template <int D>
struct TileCfg;
template <>
struct TileCfg<2> {
  static constexpr int TP = 64, LANES = 4, THREADS = 256, CAP = 1024, LIST = 24, NL = 3;
};
template <>
struct TileCfg<3> {
  static constexpr int TP = 32, LANES = 8, THREADS = 256, CAP = 1024, LIST = 16, NL = 9;
};

// Maximum columns per staged line: TP targets can span TP cells, plus the two neighbours.
template <int D>
constexpr int tile_cols() { return TileCfg<D>::TP + 2; }

// Shared-memory layout of a staged tile.  EXTRA: number of additional float4 payloads per
// staged particle (adjoint seeds).
template <int D, int EXTRA>
struct TileSmem {
  static constexpr int CAP = TileCfg<D>::CAP;
  static constexpr int NCOL = tile_cols<D>() + 1;
  float4 A[CAP];
  float4 B[CAP];
  float2 C[D == 3 ? CAP : 1];
  float4 E[EXTRA > 0 ? EXTRA * CAP : 1];
  int gidx[CAP];
  int colstart[TileCfg<D>::NL * NCOL + 1];
  unsigned short list[TileCfg<D>::LIST * TileCfg<D>::THREADS];
  float tshift[TileCfg<D>::NL][3];  // target shift of each line (applied to the target, +L)
  float cshift[TileCfg<D>::NL][3];  // candidate shift of each line (applied at staging, -L)
  int ncols, colbase, total, fallback;
  int linecell[TileCfg<D>::NL];     // global cell id of column 0 of each line (-1: no line)
};

template <int D, int EXTRA>
constexpr size_t tile_smem_bytes() { return sizeof(TileSmem<D, EXTRA>); }

// Per-scene line indexing: global line id = seg_line_base + cz * ny + cy.
__device__ __forceinline__ void line_coords(const DevSeg& s, int line_local, int& cy, int& cz) {
  cy = line_local % s.n[1];
  cz = line_local / s.n[1];
}

// Build the column table of a tile and stage its particles.  Returns false (fallback) when the
// staged region exceeds the shared-memory capacity.  Must be called by all threads of the CTA.
template <int D, int EXTRA>
__device__ bool stage_tile(TileSmem<D, EXTRA>& sm, const DevSeg& s, const Tile& T, const Arrays& a,
                           const uint32_t* __restrict__ keys, const int* __restrict__ cell_off,
                           const float4* __restrict__ extra0, const float* __restrict__ extra1) {
  constexpr int NL = TileCfg<D>::NL;
  constexpr int NCOL = TileSmem<D, EXTRA>::NCOL;
  constexpr int CAP = TileCfg<D>::CAP;
  const int tid = threadIdx.x;
  const int nx = s.n[0], ny = s.n[1], nz = s.n[2];
  int c_first[3], c_last[3];
  key_coords(s, keys[T.p0], c_first);
  key_coords(s, keys[T.p1 - 1], c_last);
  const int colbase = c_first[0] - 1;
  const int ncols = c_last[0] - c_first[0] + 3;  // columns colbase .. colbase + ncols - 1
  const int cy = c_first[1], cz = c_first[2];
  if (ncols > NCOL - 1) {  // a sparse line: the tile spans more cells than the table holds
    __syncthreads();
    if (tid == 0) sm.fallback = 1;
    __syncthreads();
    return false;
  }
  const bool px = s.periodic_mask & 1, py = (s.periodic_mask >> 1) & 1, pz = (s.periodic_mask >> 2) & 1;
  if (tid < NL) {
    const int dy = (D == 2) ? tid - 1 : tid % 3 - 1;
    const int dz = (D == 2) ? 0 : tid / 3 - 1;
    int ly = cy + dy, lz = cz + dz;
    float ty = 0.f, tz = 0.f, cyv = 0.f, czv = 0.f;
    bool ok = true;
    if (ly < 0) { if (py) { ly += ny; cyv = -s.L[1]; } else ok = false; }
    else if (ly >= ny) { if (py) { ly -= ny; ty = s.L[1]; } else ok = false; }
    if (D == 3) {
      if (lz < 0) { if (pz) { lz += nz; czv = -s.L[2]; } else ok = false; }
      else if (lz >= nz) { if (pz) { lz -= nz; tz = s.L[2]; } else ok = false; }
    }
    sm.linecell[tid] = ok ? s.cell_base + (lz * ny + ly) * nx : -1;
    sm.tshift[tid][0] = 0.f; sm.tshift[tid][1] = ty; sm.tshift[tid][2] = tz;
    sm.cshift[tid][0] = 0.f; sm.cshift[tid][1] = cyv; sm.cshift[tid][2] = czv;
  }
  __syncthreads();
  // counts of every (line, column) cell, then an exclusive scan in stencil order
  const int nent = NL * ncols;
  for (int e = tid; e < nent; e += blockDim.x) {
    const int l = e / ncols, c = e % ncols;
    const int lc = sm.linecell[l];
    int cnt = 0;
    if (lc >= 0) {
      int col = colbase + c;
      bool ok = true;
      if (col < 0) { if (px) col += nx; else ok = false; }
      else if (col >= nx) { if (px) col -= nx; else ok = false; }
      if (ok) cnt = cell_off[lc + col + 1] - cell_off[lc + col];
    }
    sm.colstart[l * NCOL + c] = cnt;
  }
  __syncthreads();
  if (tid < 32) {
    // warp scan over the (line, column) entries in order
    int run = 0;
    for (int base = 0; base < nent; base += 32) {
      const int e = base + tid;
      const int l = e / ncols, c = e % ncols;
      int v = (e < nent) ? sm.colstart[l * NCOL + c] : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, incl, o);
        if (tid >= o) incl += t;
      }
      if (e < nent) sm.colstart[l * NCOL + c] = run + incl - v;
      run += __shfl_sync(kFull, incl, 31);
    }
    if (tid == 0) {
      sm.total = run;
      sm.ncols = ncols;
      sm.colbase = colbase;
      sm.fallback = run > CAP;
    }
  }
  __syncthreads();
  // the end of each line's last column = start of the next line's first column
  const int total = sm.total;
  if (sm.fallback) return false;
  // stage: staged index k -> (line, column) by binary search over the scanned starts
  for (int k = tid; k < total; k += blockDim.x) {
    int lo = 0, hi = nent - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      const int l = mid / ncols, c = mid % ncols;
      if (sm.colstart[l * NCOL + c] <= k) lo = mid; else hi = mid - 1;
    }
    const int l = lo / ncols, c = lo % ncols;
    int col = colbase + c;
    float sx = 0.f;
    if (col < 0) { col += nx; sx = -s.L[0]; }  // left image: x_j - L is exact near L
    else if (col >= nx) { col -= nx; }         // right image: the target takes off L
    const int cell = sm.linecell[l] + col;
    const int j = cell_off[cell] + (k - sm.colstart[l * NCOL + c]);
    float4 A = __ldg(a.A + j), B = __ldg(a.B + j);
    A.x += sx;
    A.y += sm.cshift[l][1];
    if (D == 3) A.z += sm.cshift[l][2];
    sm.A[k] = A;
    sm.B[k] = B;
    if (D == 3) sm.C[k] = __ldg(a.C + j);
    if (EXTRA > 0) sm.E[k] = __ldg(extra0 + j);
    if (EXTRA > 1) sm.E[CAP + k] = make_float4(__ldg(extra1 + j), 0.f, 0.f, 0.f);
    sm.gidx[k] = j;
  }
  __syncthreads();
  return true;
}

// Column runs of one target in line l (target in column ccol of the tile): the staged indices
// of its three cells.  The column right of the box's last cell (periodic) is staged without a
// shift; its run is returned separately so the caller can take L off the target instead
// (x_i - L is exact for x_i near L, x_j + L is not for x_j near 0).
template <int D, int EXTRA>
__device__ __forceinline__ void target_runs(const TileSmem<D, EXTRA>& sm, int l, int ccol, int nx, int& lo, int& mid,
                                            int& hi) {
  constexpr int NCOL = TileSmem<D, EXTRA>::NCOL;
  const int ncols = sm.ncols;
  lo = sm.colstart[l * NCOL + (ccol - 1)];
  const int endc = ccol + 2;
  if (endc < ncols)
    hi = sm.colstart[l * NCOL + endc];
  else
    hi = (l + 1 < TileCfg<D>::NL) ? sm.colstart[(l + 1) * NCOL] : sm.total;
  // absolute column of ccol + 1; if it lies past the box (wrapped), split it off
  const int abs_right = sm.colbase + ccol + 1;
  mid = (abs_right >= nx) ? sm.colstart[l * NCOL + ccol + 1] : hi;
}

}  // namespace sph
