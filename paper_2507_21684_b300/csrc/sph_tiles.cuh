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

// One tile: particle range [p0, p1) inside one cell line of one scene, with the x cells of its
// first and last particle and the line's (y, z) cell (filled when the tile table is built).
struct Tile {
  int p0, p1, seg, line;
  int cx0, cx1, cy, cz;
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
// staged particle (adjoint seeds).  Each staged line holds up to three runs in stencil order:
// the left periodic image cell, the in-box columns (one contiguous range of sorted particles),
// the right periodic image cell.
template <int D, int EXTRA>
struct TileSmem {
  static constexpr int CAP = TileCfg<D>::CAP;
  static constexpr int NCOL = tile_cols<D>() + 1;
  static constexpr int NL = TileCfg<D>::NL;
  static constexpr int NRUN = 3 * NL;
  float4 A[CAP];
  float4 B[CAP];
  float2 C[D == 3 ? CAP : 1];
  float4 E[EXTRA > 0 ? EXTRA * CAP : 1];
  int colstart[NL * NCOL + 1];      // staged index of each (line, column) cell start
  unsigned short list[TileCfg<D>::LIST * TileCfg<D>::THREADS];
  int run_g[NRUN];                  // global start of each run
  int run_n[NRUN];                  // length of each run
  int run_s[NRUN + 1];              // staged start of each run (exclusive scan)
  float run_sx[NRUN];               // x shift applied at staging (-L for the left image)
  float tshift[NL][3];              // target shift of each line (upper periodic image: +L)
  float cshift[NL][3];              // candidate shift of each line (lower periodic image: -L)
  int ncols, colbase, total, fallback;
  int linecell[NL];                 // global cell id of column 0 of each line (-1: no line)
};

template <int D, int EXTRA>
constexpr size_t tile_smem_bytes() { return sizeof(TileSmem<D, EXTRA>); }

// Build the run table of a tile and stage its particles (two dependent global round trips:
// the cell offsets, then the particle records).  Returns 1 when staged, 0 (fallback) when the
// staged region exceeds the shared-memory capacity or the column table, -1 when no thread
// passed want (no target of the pass in this tile: nothing is staged; the decision rides on
// the first barrier, so it costs no extra round trip).  All threads of the CTA call it.
template <int D, int EXTRA>
__device__ int stage_tile(TileSmem<D, EXTRA>& sm, const DevSeg& s, const Tile& T, const Arrays& a,
                          const int* __restrict__ cell_off, const float4* __restrict__ extra0,
                          const float* __restrict__ extra1, bool want) {
  constexpr int NL = TileCfg<D>::NL;
  constexpr int NCOL = TileSmem<D, EXTRA>::NCOL;
  constexpr int NRUN = TileSmem<D, EXTRA>::NRUN;
  constexpr int CAP = TileCfg<D>::CAP;
  const int tid = threadIdx.x;
  const int nx = s.n[0], ny = s.n[1], nz = s.n[2];
  const int colbase = T.cx0 - 1;
  const int ncols = T.cx1 - T.cx0 + 3;  // columns colbase .. colbase + ncols - 1
  if (ncols > NCOL - 1) {               // a sparse line: more cells than the table holds
    if (tid == 0) sm.fallback = 1;
    return __syncthreads_or(want) ? 0 : -1;
  }
  const bool px = s.periodic_mask & 1, py = (s.periodic_mask >> 1) & 1, pz = (s.periodic_mask >> 2) & 1;
  // in-box column range of the tile and its periodic image cells
  const int mc0 = max(colbase, 0), mc1 = min(colbase + ncols - 1, nx - 1);
  const bool left_img = px && colbase < 0;
  const bool right_img = px && colbase + ncols - 1 >= nx;
  // 1) line geometry (threads 0..NL-1) and every needed cell offset (one round trip)
  if (tid < NL) {
    const int dy = (D == 2) ? tid - 1 : tid % 3 - 1;
    const int dz = (D == 2) ? 0 : tid / 3 - 1;
    int ly = T.cy + dy, lz = T.cz + dz;
    float ty = 0.f, tz = 0.f, cyv = 0.f, czv = 0.f;
    bool ok = true;
    if (ly < 0) { if (py) { ly += ny; cyv = -s.L[1]; } else ok = false; }
    else if (ly >= ny) { if (py) { ly -= ny; ty = s.L[1]; } else ok = false; }
    if (D == 3) {
      if (lz < 0) { if (pz) { lz += nz; czv = -s.L[2]; } else ok = false; }
      else if (lz >= nz) { if (pz) { lz -= nz; tz = s.L[2]; } else ok = false; }
    }
    const int lc = ok ? s.cell_base + (lz * ny + ly) * nx : -1;
    sm.linecell[tid] = lc;
    sm.tshift[tid][0] = 0.f; sm.tshift[tid][1] = ty; sm.tshift[tid][2] = tz;
    sm.cshift[tid][0] = 0.f; sm.cshift[tid][1] = cyv; sm.cshift[tid][2] = czv;
    // runs: left image cell (nx-1), in-box columns [mc0, mc1], right image cell (0)
    int g0 = 0, n0 = 0, g1 = 0, n1 = 0, g2 = 0, n2 = 0;
    if (ok) {
      if (left_img) { g0 = cell_off[lc + nx - 1]; n0 = cell_off[lc + nx] - g0; }
      g1 = cell_off[lc + mc0];
      n1 = cell_off[lc + mc1 + 1] - g1;
      if (right_img) { g2 = cell_off[lc]; n2 = cell_off[lc + 1] - g2; }
    }
    sm.run_g[3 * tid + 0] = g0; sm.run_n[3 * tid + 0] = n0; sm.run_sx[3 * tid + 0] = -s.L[0];
    sm.run_g[3 * tid + 1] = g1; sm.run_n[3 * tid + 1] = n1; sm.run_sx[3 * tid + 1] = 0.f;
    sm.run_g[3 * tid + 2] = g2; sm.run_n[3 * tid + 2] = n2; sm.run_sx[3 * tid + 2] = 0.f;
  }
  // in-box column boundaries of every line: colstart is filled relative to the run start
  // after the scan; here the raw offsets are kept in colstart.
  const int nb = NL * (ncols + 1);
  if (!__syncthreads_or(want)) return -1;
  for (int e = tid; e < nb; e += blockDim.x) {
    const int l = e / (ncols + 1), c = e - l * (ncols + 1);
    const int lc = sm.linecell[l];
    int v = 0;
    if (lc >= 0) {
      const int col = min(max(colbase + c, mc0), mc1 + 1);  // clamp into the in-box range
      v = cell_off[lc + col];
    }
    sm.colstart[l * NCOL + c] = v;
  }
  // 2) exclusive scan of the run lengths (one warp, NRUN <= 27)
  if (tid < 32) {
    const int v = tid < NRUN ? sm.run_n[tid] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (tid >= o) incl += t;
    }
    if (tid < NRUN) sm.run_s[tid] = incl - v;
    const int total = __shfl_sync(kFull, incl, 31);
    if (tid == 0) {
      sm.run_s[NRUN] = total;
      sm.total = total;
      sm.ncols = ncols;
      sm.colbase = colbase;
      sm.fallback = total > CAP;
    }
  }
  __syncthreads();
  if (sm.fallback) return 0;
  const int total = sm.total;
  // 3) column starts as staged indices: image columns map to their own runs
  for (int e = tid; e < nb; e += blockDim.x) {
    const int l = e / (ncols + 1), c = e - l * (ncols + 1);
    const int col = colbase + c;
    int v;
    if (col < 0) v = sm.run_s[3 * l + 0];                           // start of the left image
    else if (col > nx) v = sm.run_s[3 * l + 2] + sm.run_n[3 * l + 2];  // end of the right image
    else if (col == nx) v = sm.run_s[3 * l + 2];                    // start of the right image
    else v = sm.run_s[3 * l + 1] + (sm.colstart[l * NCOL + c] - sm.run_g[3 * l + 1]);
    if (sm.linecell[l] < 0) v = sm.run_s[3 * l + 0];
    sm.colstart[l * NCOL + c] = v;
  }
  // 4) copy: every thread takes staged indices, finds its run (at most 3 NL runs)
  for (int k = tid; k < total; k += blockDim.x) {
    int r = 0;
#pragma unroll 1
    while (r + 1 < NRUN && sm.run_s[r + 1] <= k) ++r;
    const int j = sm.run_g[r] + (k - sm.run_s[r]);
    const int l = r / 3;
    float4 A = __ldg(a.A + j), B = __ldg(a.B + j);
    A.x += sm.run_sx[r];
    A.y += sm.cshift[l][1];
    if (D == 3) A.z += sm.cshift[l][2];
    sm.A[k] = A;
    sm.B[k] = B;
    if (D == 3) sm.C[k] = __ldg(a.C + j);
    if (EXTRA > 0) sm.E[k] = __ldg(extra0 + j);
    if (EXTRA > 1) sm.E[CAP + k] = make_float4(__ldg(extra1 + j), 0.f, 0.f, 0.f);
  }
  __syncthreads();
  return 1;
}

// Global index of staged particle k (for predicates that exclude the target by index).
template <int D, int EXTRA>
__device__ __forceinline__ int staged_gidx(const TileSmem<D, EXTRA>& sm, int k) {
  int r = 0;
  while (r + 1 < TileSmem<D, EXTRA>::NRUN && sm.run_s[r + 1] <= k) ++r;
  return sm.run_g[r] + (k - sm.run_s[r]);
}


}  // namespace sph
