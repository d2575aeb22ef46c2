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
#include <cstddef>

#include "sph_device.cuh"

namespace sph {

// One tile: particle range [p0, p1) inside one cell line of one scene, with the x cells of its
// first and last particle and the line's (y, z) cell (filled when the tile table is built).
struct Tile {
  int p0, p1, seg, line;
  int cx0, cx1, cy, cz;
};

// Tile shape per dimension: targets per tile (TP), threads per target (LANES, TP x LANES = THREADS
// per CTA), staged-particle capacity (CAP) and hit-list entries per thread (LIST).  Set per build (SPH_TILE2_* / SPH_TILE3_*) so that the
// autotuner can time library variants against each other; the defaults are the shapes measured
// best on the B300 for the dam break and the 3D Taylor-Green vortex.
#ifndef SPH_TILE2_TP
#define SPH_TILE2_TP 64
#define SPH_TILE2_LANES 4
#define SPH_TILE2_LIST 24
#endif
#ifndef SPH_TILE2_THREADS
#define SPH_TILE2_THREADS 256
#define SPH_TILE2_CAP 1024
#endif
#ifndef SPH_TILE3_TP
#define SPH_TILE3_TP 32
#define SPH_TILE3_LANES 8
#define SPH_TILE3_LIST 18
#endif
#ifndef SPH_TILE3_THREADS
#define SPH_TILE3_THREADS 256
#define SPH_TILE3_CAP 1024
#endif

// SPH_W3: the 3D sweep (and rate evaluation) on the warp-per-tile traversal (sph_warptiles.cuh);
// 0 keeps them on the staged traversal (a library variant, timed against it by the autotuner).
#ifndef SPH_W3
#define SPH_W3 1
#endif
// CUT: how cell lines are cut into tiles (0 whole cells, 1 balanced tiles cut between particles).
// 3D: balanced tiles fill the warps of the warp-per-tile sweep (a warp of a whole-cell tile of
// two cells of about 15 particles leaves a fifth of its lanes idle); whole cells with the staged
// sweep.
#ifndef SPH_TILE2_CUT
#define SPH_TILE2_CUT 1
#endif
#ifndef SPH_TILE3_CUT
#define SPH_TILE3_CUT (SPH_W3 ? 1 : 0)
#endif
// MINB: CTAs per SM the tiled kernels are compiled for (register budget 64K / (MINB x THREADS)).
#ifndef SPH_TILE2_MINB
#define SPH_TILE2_MINB (1024 / SPH_TILE2_THREADS)
#endif
#ifndef SPH_TILE3_MINB
#define SPH_TILE3_MINB (1024 / SPH_TILE3_THREADS)
#endif

template <int D>
struct TileCfg;
template <>
struct TileCfg<2> {
  static constexpr int TP = SPH_TILE2_TP, LANES = SPH_TILE2_LANES, THREADS = SPH_TILE2_THREADS, CAP = SPH_TILE2_CAP,
                       LIST = SPH_TILE2_LIST, NL = 3, MINB = SPH_TILE2_MINB, CUT = SPH_TILE2_CUT;
};
template <>
struct TileCfg<3> {
  static constexpr int TP = SPH_TILE3_TP, LANES = SPH_TILE3_LANES, THREADS = SPH_TILE3_THREADS, CAP = SPH_TILE3_CAP,
                       LIST = SPH_TILE3_LIST, NL = 9, MINB = SPH_TILE3_MINB, CUT = SPH_TILE3_CUT;
};

// The records of a tile's own targets (a contiguous range of sorted particles), copied into
// shared memory with cp.async while the neighbour lines are staged, so that a pass's prologue
// and epilogue read them without a global round trip.  E0/E1: per-target extras of the pass.
template <int D>
struct TargetCache {
  static constexpr int TP = TileCfg<D>::TP;
  float4 A[TP], B[TP], X[TP], O[TP];
  float4 XL[D == 3 ? TP : 1];
  float2 C[D == 3 ? TP : 1];
  uint2 meta[TP];
  float4 E0[TP], E1[TP];
  // the cache seen through the Arrays interface (local index = i - tile start)
  __device__ __forceinline__ Arrays view() {
    Arrays v;
    v.A = A; v.B = B; v.C = C; v.X = X; v.XL = XL; v.O = O; v.meta = meta;
    return v;
  }
};

// A pass's view of its target in the cache: records (local index k) and the two extras.
struct TgtView {
  Arrays a;
  const float4* e0;
  const float4* e1;
  int k;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Load with acquire semantics at GPU scope: the caller's later accesses (and, through a barrier,
// its CTA's) see every write that preceded the release of the value read.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Record loads of the staging: through the read-only path, or (COH) through L2 only, for
// records that another CTA of the same launch may have rewritten (the fused wall + sweep kernel).
template <bool COH>
__device__ __forceinline__ float4 ld_rec(const float4* p) { return COH ? __ldcg(p) : __ldg(p); }
template <bool COH>
__device__ __forceinline__ float2 ld_rec(const float2* p) { return COH ? __ldcg(p) : __ldg(p); }

// Issue the copies of targets [p0, p0 + n) into the cache (all threads of the CTA; completion is
// awaited by stage_tile before its first barrier).  The 16-byte copies bypass L1; with COH the
// 8-byte records are read through L2 as well.
template <int D, bool COH = false>
__device__ __forceinline__ void fill_target_cache(TargetCache<D>& tc, const Arrays& a, const float4* e0,
                                                  const float4* e1, int p0, int n) {
  constexpr int NF = (D == 3) ? 5 : 4;  // float4 arrays A, B, X, O (, XL)
  for (int e = threadIdx.x; e < n * NF; e += blockDim.x) {
    const int f = e / n, k = e - f * n, g = p0 + k;
    const float4* src = f == 0 ? a.A : f == 1 ? a.B : f == 2 ? a.X : f == 3 ? a.O : a.XL;
    float4* dst = f == 0 ? tc.A : f == 1 ? tc.B : f == 2 ? tc.X : f == 3 ? tc.O : tc.XL;
    cp_async16(dst + k, src + g);
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    cp_async8(&tc.meta[k], a.meta + p0 + k);
    if (D == 3) {
      if (COH) tc.C[k] = __ldcg(a.C + p0 + k);
      else cp_async8(&tc.C[k], a.C + p0 + k);
    }
    if (e0) cp_async16(&tc.E0[k], e0 + p0 + k);
    if (e1) cp_async16(&tc.E1[k], e1 + p0 + k);
  }
  cp_async_commit();
}

// Maximum columns per staged line: TP targets can span TP cells, plus the two neighbours.
template <int D>
constexpr int tile_cols() { return TileCfg<D>::TP + 2; }

// Shared-memory layout of a staged tile.  EXTRA: number of additional float4 payloads per
// staged particle (adjoint seeds).  LN: threads per target of the pass (the tile shape's LANES,
// or more for a pass that wants more parallelism on the same tiles).  Each staged line holds up
// to three runs in stencil order: the left periodic image cell, the in-box columns (one contiguous
// range of sorted particles), the right periodic image cell.
template <int D, int EXTRA, int LN = TileCfg<D>::LANES>
struct TileSmem {
  static constexpr int CAP = TileCfg<D>::CAP;
  static constexpr int THREADS = TileCfg<D>::TP * LN;  // the pass's CTA
  static_assert(CAP <= 8192, "hit-list entries hold the staged index in 13 bits");
  static_assert(LN >= 1 && LN <= 32 && (LN & (LN - 1)) == 0 && THREADS <= 1024, "one group of LN lanes per target");
  static_assert(TileCfg<D>::TP * TileCfg<D>::LANES == TileCfg<D>::THREADS, "one group of LANES per target");
  static constexpr int NCOL = tile_cols<D>() + 1;
  static constexpr int NL = TileCfg<D>::NL;
  static constexpr int NRUN = 3 * NL;
  float4 A[CAP];
  float4 B[CAP];
  float2 C[D == 3 ? CAP : 1];
  float4 E[EXTRA > 0 ? EXTRA * CAP : 1];
  TargetCache<D> tc;
  unsigned short list[TileCfg<D>::LIST * THREADS];
  // From here to img: a tile's staging plan (TilePlan), which depends on the cell structure only
  alignas(16) Tile ptile;           // the tile
  int pvalid, ppad[3];              // whether the rest of the plan (the staging table) is filled
  int colstart[NL * NCOL + 1];      // staged index of each (line, column) cell start
  int run_g[NRUN];                  // global start of each run
  int run_n[NRUN];                  // length of each run
  int run_s[NRUN + 1];              // staged start of each run (exclusive scan)
  float run_sx[NRUN];               // x shift applied at staging (-L for the left image)
  float tshift[NL][3];              // target shift of each line (upper periodic image: +L)
  float cshift[NL][3];              // candidate shift of each line (lower periodic image: -L)
  int ncols, colbase, total, fallback;
  int linecell[NL];                 // global cell id of column 0 of each line (-1: no line)
  int img[NL][4];                   // offsets bounding the left and right periodic image cells
};

template <int D, int EXTRA, int LN = TileCfg<D>::LANES>
constexpr size_t tile_smem_bytes() { return sizeof(TileSmem<D, EXTRA, LN>); }

// A tile's staging plan in global memory, as uint4 words laid out like TileSmem from ptile to img:
// the tile, a flag, and the staging table (column starts as staged indices, the run table and the
// periodic shifts).  The table depends only on the cell structure, so the fused wall + sweep
// launch keeps it from the step after a rebuild to the next rebuild, and a tile then starts
// with one load of its plan instead of its cell offsets and a run-table scan.  Kept in 2D (the
// plans of 3D tiles would outweigh their particles' state); a 3D plan is the tile and the flag.
template <int D>
struct TilePlan {
  using SM = TileSmem<D, 0>;
  static constexpr bool CACHED = D == 2;
  static constexpr size_t BEGIN = offsetof(SM, ptile);
  static constexpr size_t END = offsetof(SM, img) + sizeof(int) * 4 * TileCfg<D>::NL;
  static constexpr int U4 = CACHED ? (int)((END - BEGIN + 15) / 16) : 3;
  static_assert(BEGIN % 16 == 0, "the plan is copied as uint4 words");
};

// Copy of a plan (U4 words from the tile on) into the CTA's shared memory (all threads).
template <int D, int EXTRA, int LN>
__device__ __forceinline__ void load_plan(TileSmem<D, EXTRA, LN>& sm, const uint4* __restrict__ plan) {
  uint4* dst = reinterpret_cast<uint4*>(&sm.ptile);
  for (int e = threadIdx.x; e < TilePlan<D>::U4; e += blockDim.x) dst[e] = plan[e];
}
// The staging table of a staged tile into its plan, and the flag (all threads; read by later launches).
template <int D, int EXTRA, int LN>
__device__ __forceinline__ void store_plan(const TileSmem<D, EXTRA, LN>& sm, uint4* __restrict__ plan) {
  const uint4* src = reinterpret_cast<const uint4*>(&sm.ptile);
  for (int e = 3 + threadIdx.x; e < TilePlan<D>::U4; e += blockDim.x) plan[e] = src[e];
  if (threadIdx.x == 0) reinterpret_cast<int*>(plan + 2)[0] = 1;
}

// Geometry of staged line l of a tile: global cell id of its column 0 (-1 when the line lies
// outside a closed box), the target shift (upper periodic image: +L) and the candidate shift
// (lower periodic image: -L) on the y and z axes.  Pure arithmetic.
template <int D>
__device__ __forceinline__ int tile_line(const DevSeg& s, const Tile& T, int l, float* tsh, float* csh) {
  const int dy = (D == 2) ? l - 1 : l % 3 - 1;
  const int dz = (D == 2) ? 0 : l / 3 - 1;
  const int nx = s.n[0], ny = s.n[1], nz = s.n[2];
  int ly = T.cy + dy, lz = T.cz + dz;
  tsh[0] = tsh[1] = csh[0] = csh[1] = 0.f;
  if (ly < 0) { if ((s.periodic_mask >> 1) & 1) { ly += ny; csh[0] = -s.L[1]; } else return -1; }
  else if (ly >= ny) { if ((s.periodic_mask >> 1) & 1) { ly -= ny; tsh[0] = s.L[1]; } else return -1; }
  if (D == 3) {
    if (lz < 0) { if ((s.periodic_mask >> 2) & 1) { lz += nz; csh[1] = -s.L[2]; } else return -1; }
    else if (lz >= nz) { if ((s.periodic_mask >> 2) & 1) { lz -= nz; tsh[1] = s.L[2]; } else return -1; }
  }
  return s.cell_base + (lz * ny + ly) * nx;
}

// Run containing staged index k: the largest r with run_s[r] <= k (run_s is non-decreasing and
// k < total, so that run is not empty).
template <int D, int EXTRA, int LN>
__device__ __forceinline__ int staged_run(const TileSmem<D, EXTRA, LN>& sm, int k) {
  constexpr int NRUN = TileSmem<D, EXTRA, LN>::NRUN;
  int r = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1)
    if (r + step < NRUN && sm.run_s[r + step] <= k) r += step;
  return r;
}

// Stage particle k of a tile whose run table is built: its records (with the run's periodic
// shifts) and extras.  Returns whether it is a wall particle (mass <= 0).
template <int D, int EXTRA, bool COH, int LN>
__device__ __forceinline__ bool stage_record(TileSmem<D, EXTRA, LN>& sm, const Arrays& a, int k,
                                             const float4* __restrict__ extra0, const float* __restrict__ extra1) {
  constexpr int CAP = TileCfg<D>::CAP;
  const int r = staged_run(sm, k);
  const int j = sm.run_g[r] + (k - sm.run_s[r]);
  const int l = r / 3;
  float4 A = ld_rec<COH>(a.A + j), B = ld_rec<COH>(a.B + j);
  A.x += sm.run_sx[r];
  A.y += sm.cshift[l][1];
  if (D == 3) A.z += sm.cshift[l][2];
  sm.A[k] = A;
  sm.B[k] = B;
  float m = B.w;
  if (D == 3) {
    const float2 C = ld_rec<COH>(a.C + j);
    sm.C[k] = C;
    m = C.y;
  }
  if (EXTRA > 0) sm.E[k] = __ldg(extra0 + j);
  if (EXTRA > 1) sm.E[CAP + k] = make_float4(__ldg(extra1 + j), 0.f, 0.f, 0.f);
  return m <= 0.f;
}

// Stage the records of a tile whose staging table is in shared memory (all threads); returns 1.
template <int D, int EXTRA, bool COH, int LN>
__device__ __forceinline__ int stage_records(TileSmem<D, EXTRA, LN>& sm, const Arrays& a, int total,
                                             const float4* __restrict__ extra0, const float* __restrict__ extra1,
                                             int* wall_seen) {
  int walls = 0;
  for (int k = threadIdx.x; k < total; k += blockDim.x) walls |= stage_record<D, EXTRA, COH>(sm, a, k, extra0, extra1);
  if (wall_seen)
    *wall_seen = __syncthreads_or(walls);
  else
    __syncthreads();
  return 1;
}

// Build the run table of a tile and stage its particles: two dependent global round trips (every
// cell offset the tile needs, then the particle records).  The caller's cp.async copies into the
// target cache are complete and visible after the first barrier.  Returns 1 when staged, 0 (fallback)
// when the staged region exceeds the shared-memory capacity or the column table, -1 when no
// thread passed want (no target of the pass in this tile: nothing is staged; the decision rides
// on the first barrier, so it costs no extra round trip).  All threads of the CTA call it.
// wall_seen (optional): set to whether any staged particle is a wall (mass <= 0).  COH: record
// loads through L2 (see ld_rec).
template <int D, int EXTRA, bool COH = false, int LN = TileCfg<D>::LANES>
__device__ int stage_tile(TileSmem<D, EXTRA, LN>& sm, const DevSeg& s, const Tile& T, const Arrays& a,
                          const int* __restrict__ cell_off, const float4* __restrict__ extra0,
                          const float* __restrict__ extra1, bool want, int* wall_seen = nullptr) {
  constexpr int NL = TileCfg<D>::NL;
  constexpr int NCOL = TileSmem<D, EXTRA, LN>::NCOL;
  constexpr int NRUN = TileSmem<D, EXTRA, LN>::NRUN;
  constexpr int CAP = TileCfg<D>::CAP;
  const int tid = threadIdx.x;
  const int nx = s.n[0];
  const int colbase = T.cx0 - 1;
  const int ncols = T.cx1 - T.cx0 + 3;  // columns colbase .. colbase + ncols - 1
  if (ncols > NCOL - 1) {               // a sparse line: more cells than the table holds
    if (tid == 0) sm.fallback = 1;
    cp_async_wait_all();
    return __syncthreads_or(want) ? 0 : -1;
  }
  const bool px = s.periodic_mask & 1;
  // in-box column range of the tile and its periodic image cells
  const int mc0 = max(colbase, 0), mc1 = min(colbase + ncols - 1, nx - 1);
  const bool left_img = px && colbase < 0;
  const bool right_img = px && colbase + ncols - 1 >= nx;
  // 1) one round trip: the column boundaries of every staged line (clamped into the in-box
  //    range, raw offsets) and the bounds of the two periodic image cells
  if (tid < NL) {
    float tsh[2], csh[2];
    sm.linecell[tid] = tile_line<D>(s, T, tid, tsh, csh);
    sm.tshift[tid][0] = 0.f; sm.tshift[tid][1] = tsh[0]; sm.tshift[tid][2] = tsh[1];
    sm.cshift[tid][0] = 0.f; sm.cshift[tid][1] = csh[0]; sm.cshift[tid][2] = csh[1];
  }
  const int nb = NL * (ncols + 1);
  for (int e = tid; e < nb + 4 * NL; e += blockDim.x) {
    float tsh[2], csh[2];
    if (e < nb) {
      const int l = e / (ncols + 1), c = e - l * (ncols + 1);
      const int lc = tile_line<D>(s, T, l, tsh, csh);
      const int col = min(max(colbase + c, mc0), mc1 + 1);
      sm.colstart[l * NCOL + c] = lc >= 0 ? cell_off[lc + col] : 0;
    } else {
      const int l = (e - nb) >> 2, w = (e - nb) & 3;
      const int lc = tile_line<D>(s, T, l, tsh, csh);
      int v = 0;
      if (lc >= 0 && (w < 2 ? left_img : right_img)) v = cell_off[lc + (w < 2 ? nx - 1 + w : w - 2)];
      sm.img[l][w] = v;
    }
  }
  cp_async_wait_all();  // the target cache (issued by the caller) is complete at this barrier
  if (!__syncthreads_or(want)) return -1;
  // 2) run table (left image, in-box columns, right image per line) and its exclusive scan
  if (tid < 32) {
    int g = 0, n = 0;
    if (tid < NRUN) {
      const int l = tid / 3, kind = tid - 3 * (tid / 3);
      if (sm.linecell[l] >= 0) {
        if (kind == 0) { g = sm.img[l][0]; n = sm.img[l][1] - g; }
        else if (kind == 1) { g = sm.colstart[l * NCOL + (mc0 - colbase)]; n = sm.colstart[l * NCOL + (mc1 + 1 - colbase)] - g; }
        else { g = sm.img[l][2]; n = sm.img[l][3] - g; }
      }
      sm.run_g[tid] = g;
      sm.run_n[tid] = n;
      sm.run_sx[tid] = kind == 0 ? -s.L[0] : 0.f;
    }
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (tid >= o) incl += t;
    }
    if (tid < NRUN) sm.run_s[tid] = incl - n;
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
  // 3) column starts as staged indices (image columns map to their own runs), and the copy of
  //    the records (second round trip)
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
  return stage_records<D, EXTRA, COH>(sm, a, total, extra0, extra1, wall_seen);
}

// Stage the wall particles of a staged tile again, through L2 (their records were rewritten
// after the first staging); the fluid entries stay.  All threads of the CTA call it.
template <int D, int EXTRA, int LN>
__device__ void restage_walls(TileSmem<D, EXTRA, LN>& sm, const Arrays& a, const float4* __restrict__ extra0,
                              const float* __restrict__ extra1) {
  const int total = sm.total;
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const float m = D == 3 ? sm.C[k].y : sm.B[k].w;
    if (m <= 0.f) stage_record<D, EXTRA, true>(sm, a, k, extra0, extra1);
  }
  __syncthreads();
}

// Global index of staged particle k (for predicates that exclude the target by index).
template <int D, int EXTRA, int LN>
__device__ __forceinline__ int staged_gidx(const TileSmem<D, EXTRA, LN>& sm, int k) {
  const int r = staged_run(sm, k);
  return sm.run_g[r] + (k - sm.run_s[r]);
}


}  // namespace sph
