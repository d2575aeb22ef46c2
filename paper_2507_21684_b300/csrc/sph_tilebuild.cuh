// Device-side tile-table builders (one warp per cell line, one warp per tile for the wall
// list), shared by the stand-alone kernels of sph_passes.cu and the single-launch rebuild.
#pragma once
#include "sph_tiles.cuh"

namespace sph {

// Tiles of one cell line, cut in one of two ways (TileCfg<D>::CUT):
// - whole cells (0): greedily from the left, a tile holds at most TP particles and spans at most
//   TP cells (so its column table fits); a cell with more than TP particles is split into tiles
//   of its own.  One warp per line: the lanes hold the offsets of 32 consecutive cells, and each
//   tile boundary is one ballot over them (the conditions "count <= TP" and "span <= TP" are
//   monotone along the line).  Finished tiles wait in the registers of lane (k mod 32) and are
//   written in batches of 32 at slots reserved with one atomic.
// - balanced (1): the line is cut into chunks of TP cells, and the particles of each chunk into
//   ceil(count / TP) tiles of equal size (+-1), cut between particles, not at cell boundaries:
//   full tiles keep every thread of a CTA busy and a line needs ceil(count / TP) tiles, at the
//   price of staging the cells around a cut twice.  One warp per line: lane j reads the bounds
//   of chunk j (lines of up to 32 TP cells in one round trip), one atomic reserves the line's
//   tiles, and the tiles are spread over the lanes, each finding its first and last cell by
//   binary search over its chunk.
// Either way a tile's targets are one contiguous range of sorted particles whose cells lie in
// [cx0, cx1], and the order of the tiles in the table affects no result.
__device__ __forceinline__ int seg_of_line(const int* __restrict__ line_base, int S, int l) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (line_base[mid] <= l) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Cell of particle p in cells [c0, c1) of a line (cell_off[first + c1] > p >= cell_off[first + c0]):
// the largest c with cell_off[first + c] <= p.
__device__ __forceinline__ int cell_of(const int* __restrict__ cell_off, int first, int c0, int c1, int p) {
  int lo = c0, hi = c1 - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cell_off[first + mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Balanced tiles of line l (one warp, all 32 lanes call it; lane = lane index).
template <int D>
__device__ __forceinline__ void tiles_line_balanced(int l, int lane, const DevSeg* __restrict__ segs, int S,
                                           const int* __restrict__ line_base, const int* __restrict__ cell_off,
                                           Tile* __restrict__ tiles, int* __restrict__ ntiles) {
  constexpr int TP = TileCfg<D>::TP;
  const int sg = seg_of_line(line_base, S, l);
  const DevSeg& s = segs[sg];
  const int ll = l - line_base[sg];
  const int nx = s.n[0];
  const int first = s.cell_base + ll * nx;
  const int cy = ll % s.n[1], cz = ll / s.n[1];
  for (int w0 = 0; w0 < nx; w0 += 32 * TP) {  // windows of 32 chunks (warp-uniform)
    const int c0 = min(w0 + lane * TP, nx), c1 = min(c0 + TP, nx);
    int a = 0, cnt = 0;
    if (c0 < nx) {
      a = cell_off[first + c0];
      cnt = cell_off[first + c1] - a;
    }
    const int n = (cnt + TP - 1) / TP;
    int incl = n;  // tiles before this lane's chunk: exclusive scan over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    if (total == 0) continue;
    int base = 0;
    if (lane == 0) base = atomicAdd(ntiles, total);
    base = __shfl_sync(kFull, base, 0);
    // the window's tiles, 32 at a time over the lanes (one tile per lane and round): tile t lies
    // in the chunk of the first lane whose inclusive count passes t
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int t = t0 + lane;
      int j = 0;
#pragma unroll 8
      for (int q = 0; q < 32; ++q) j += __shfl_sync(kFull, incl, q) <= t;
      j = min(j, 31);
      const int ja = __shfl_sync(kFull, a, j), jcnt = __shfl_sync(kFull, cnt, j), jn = __shfl_sync(kFull, n, j);
      const int jex = __shfl_sync(kFull, incl, j) - jn, jc0 = __shfl_sync(kFull, c0, j);
      if (t < total) {
        const int jc1 = min(jc0 + TP, nx);
        const int k = t - jex;
        const int p0 = ja + (int)((long long)jcnt * k / jn), p1 = ja + (int)((long long)jcnt * (k + 1) / jn);
        Tile T;
        T.p0 = p0; T.p1 = p1; T.seg = sg; T.line = l;
        T.cx0 = cell_of(cell_off, first, jc0, jc1, p0);
        T.cx1 = cell_of(cell_off, first, jc0, jc1, p1 - 1);
        T.cy = cy; T.cz = cz;
        tiles[base + t] = T;
      }
    }
  }
}

// Whole-cell tiles of line l (one warp, all 32 lanes call it; lane = lane index).
template <int D>
__device__ __forceinline__ void tiles_line_cells(int l, int lane, const DevSeg* __restrict__ segs, int S,
                                           const int* __restrict__ line_base, const int* __restrict__ cell_off,
                                           Tile* __restrict__ tiles, int* __restrict__ ntiles) {
  constexpr int TP = TileCfg<D>::TP;
  const int sg = seg_of_line(line_base, S, l);
  const DevSeg& s = segs[sg];
  const int ll = l - line_base[sg];
  const int nx = s.n[0];
  const int first = s.cell_base + ll * nx;
  const int cy = ll % s.n[1], cz = ll / s.n[1];
  Tile mine;  // the pending tile this lane holds
  int pending = 0;
  auto emit = [&](int p0, int p1, int c0, int c1) {  // warp-uniform arguments
    if (lane == pending) {
      mine.p0 = p0; mine.p1 = p1; mine.seg = sg; mine.line = l;
      mine.cx0 = c0; mine.cx1 = c1; mine.cy = cy; mine.cz = cz;
    }
    if (++pending == 32) {
      int base = 0;
      if (lane == 0) base = atomicAdd(ntiles, 32);
      base = __shfl_sync(kFull, base, 0);
      tiles[base + lane] = mine;
      pending = 0;
    }
  };
  // open tile: first cell, first particle, last non-empty cell and its end offset
  bool open = false;
  int t_a = 0, t_p = 0, t_last = 0, t_end = 0;
  auto window = [&](int w0, int o0, int o1) {
    const int c = w0 + lane;
    const bool in = c < nx;
    const unsigned nonempty = __ballot_sync(kFull, in && o1 > o0);
    const bool last_window = w0 + 32 >= nx;
    int cur = 0;  // first lane not yet consumed
    while (cur < 32) {
      if (!open) {
        const unsigned m = nonempty & (~0u << cur);
        if (!m) break;
        const int j = __ffs(m) - 1;
        const int p0 = __shfl_sync(kFull, o0, j), p1 = __shfl_sync(kFull, o1, j);
        if (p1 - p0 > TP) {  // an over-full cell: tiles of its own
          for (int k = p0; k < p1; k += TP) emit(k, min(k + TP, p1), w0 + j, w0 + j);
          cur = j + 1;
          continue;
        }
        open = true;
        t_a = w0 + j; t_p = p0; t_last = w0 + j; t_end = p1;
        cur = j + 1;
        continue;
      }
      // extend the open tile over lanes cur..hi
      const bool ok = in && lane >= cur && o1 - t_p <= TP && c - t_a <= TP - 1;
      const unsigned okm = __ballot_sync(kFull, ok);
      const int hi = okm ? 31 - __clz(okm) : cur - 1;  // contiguous from cur
      const unsigned ne = nonempty & okm;
      if (ne) {
        const int j = 31 - __clz(ne);
        t_last = w0 + j;
        t_end = __shfl_sync(kFull, o1, j);
      }
      if (hi == 31 && !last_window) break;  // the tile may continue in the next window
      emit(t_p, t_end, t_a, t_last);
      open = false;
      cur = hi + 1;
    }
  };
  // the offsets of the first kPre windows are loaded up front (one round trip for lines of up
  // to 32 kPre cells); longer lines load the rest window by window
  constexpr int kPre = 6;
  int o0s[kPre], o1s[kPre];
#pragma unroll
  for (int w = 0; w < kPre; ++w) {
    const int c = 32 * w + lane;
    o0s[w] = c < nx ? cell_off[first + c] : 0;
    o1s[w] = c < nx ? cell_off[first + c + 1] : 0;
  }
#pragma unroll
  for (int w = 0; w < kPre; ++w)
    if (32 * w < nx) window(32 * w, o0s[w], o1s[w]);
  for (int w0 = 32 * kPre; w0 < nx; w0 += 32) {
    const int c = w0 + lane;
    window(w0, c < nx ? cell_off[first + c] : 0, c < nx ? cell_off[first + c + 1] : 0);
  }
  if (open) emit(t_p, t_end, t_a, t_last);
  if (pending) {
    int base = 0;
    if (lane == 0) base = atomicAdd(ntiles, pending);
    base = __shfl_sync(kFull, base, 0);
    if (lane < pending) tiles[base + lane] = mine;
  }
}


template <int D>
__device__ __forceinline__ void tiles_line(int l, int lane, const DevSeg* __restrict__ segs, int S,
                                           const int* __restrict__ line_base, const int* __restrict__ cell_off,
                                           Tile* __restrict__ tiles, int* __restrict__ ntiles) {
  if (TileCfg<D>::CUT)
    tiles_line_balanced<D>(l, lane, segs, S, line_base, cell_off, tiles, ntiles);
  else
    tiles_line_cells<D>(l, lane, segs, S, line_base, cell_off, tiles, ntiles);
}

// What tile T holds (the same on all lanes; one warp): bit 0 a wall particle, bit 1 a fluid one.
__device__ __forceinline__ unsigned tile_kinds(const Tile& T, int lane, const uint2* __restrict__ meta) {
  bool wall = false, fluid = false;
  for (int k = T.p0 + lane; k < T.p1; k += 32) {
    const bool w = (meta[k].x & kWallBit) != 0;
    wall |= w;
    fluid |= !w;
  }
  return (__any_sync(kFull, wall) ? 1u : 0u) | (__any_sync(kFull, fluid) ? 2u : 0u);
}
// The task lists of a scene with walls (one warp per tile): tiles holding a wall particle
// (list[0..count[0]) by index, for the wall pass, and wall_p[0..count[0]) as plans) and tiles
// holding a fluid particle (fluid_p[0..count[1]), plans): the two task lists of the fused wall +
// sweep kernel, whose sweep has nothing to do on tiles of walls alone.  A plan starts as the tile
// with its flag cleared; the fused kernel fills in the staging table the first time it stages it.
template <int D>
__device__ __forceinline__ void list_tile(const Tile& T, int w, int lane, const uint2* __restrict__ meta, int* list,
                                          uint4* wall_p, uint4* fluid_p, int* count) {
  const unsigned k = tile_kinds(T, lane, meta);
  if (lane == 0) {
    if (k & 1u) {
      const int q = atomicAdd(count, 1);
      list[q] = w;
      uint4* b = wall_p + (size_t)q * TilePlan<D>::U4;
      *reinterpret_cast<Tile*>(b) = T;
      reinterpret_cast<int*>(b + 2)[0] = 0;
    }
    if (k & 2u) {
      uint4* b = fluid_p + (size_t)atomicAdd(count + 1, 1) * TilePlan<D>::U4;
      *reinterpret_cast<Tile*>(b) = T;
      reinterpret_cast<int*>(b + 2)[0] = 0;
    }
  }
}

}  // namespace sph
