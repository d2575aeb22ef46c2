// Device side of the single-launch rebuild (grid barrier, grid scan, the phases), used by the
// stand-alone cooperative rebuild and by the fused step kernel.  Every wait is bounded: a barrier
// that gives up sets status bit 1 and the whole grid leaves.
#pragma once
#include "sph_rebuild.cuh"
#include "sph_sort.cuh"
#include "sph_tilebuild.cuh"

namespace sph {


constexpr int kRbThreads = 256;
constexpr long long kRbBarrierSpins = 1LL << 22;  // x ~100 ns sleep: the barrier gives up after ~0.5 s

// Grid-wide barrier over a cooperative launch (all CTAs resident).  bar[0] counts arrivals,
// bar[1] is the generation.  Returns false when the wait gave up (status bit 1 set); every CTA
// then leaves the kernel, so nothing runs on half-built data.
__device__ inline bool grid_barrier(unsigned* bar, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*vgen == g) {
        if (++it > kRbBarrierSpins) {
          atomicOr(status, 2);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

union RebuildSmem {
  ScatterSmem scatter;
  uint32_t hist[256];
  uint32_t wsum[kRbThreads / 32 + 1];
};

// Exclusive scan of a[0, n) in place by one CTA of 256 threads, in rounds of 4096 values
// (16 consecutive per thread) with a running carry; returns the total.  wsum: 9 words of shared
// memory (the warp offsets and the round total).
__device__ inline uint32_t cta_scan(uint32_t* __restrict__ a, int n, uint32_t* wsum) {
  constexpr int NW = kRbThreads / 32;
  uint32_t carry = 0;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int r0 = 0; r0 < n; r0 += 16 * kRbThreads) {
    const int base = r0 + t * 16;
    uint32_t v[16], run = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t x = (base + k < n) ? a[base + k] : 0u;
      v[k] = run;
      run += x;
    }
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      const uint32_t ws = lane < NW ? wsum[lane] : 0u;
      uint32_t wi = ws;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, wi, o);
        if (lane >= o) wi += y;
      }
      __syncwarp();
      if (lane < NW) wsum[lane] = wi - ws;
      if (lane == NW - 1) wsum[NW] = wi;  // the round's total
    }
    __syncthreads();
    const uint32_t off = carry + wsum[w] + incl - run;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (base + k < n) a[base + k] = v[k] + off;
    carry += wsum[NW];
    __syncthreads();  // wsum is rewritten by the next round
  }
  return carry;
}

// Exclusive scan of a[0, n) across the grid: one CTA when n is small, else chunk scans, a scan
// of the chunk totals and the chunk offsets (two more barriers).
__device__ inline bool grid_scan(uint32_t* __restrict__ a, int n, uint32_t* __restrict__ sums, uint32_t* wsum,
                          unsigned* bar, int* status) {
  if (n <= 4 * 16 * kRbThreads) {
    if (blockIdx.x == 0) cta_scan(a, n, wsum);
    return grid_barrier(bar, status);
  }
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int b0 = min(n, blockIdx.x * per), b1 = min(n, b0 + per);
  const uint32_t tot = cta_scan(a + b0, b1 - b0, wsum);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
  if (!grid_barrier(bar, status)) return false;
  if (blockIdx.x == 0) cta_scan(sums, gridDim.x, wsum);
  if (!grid_barrier(bar, status)) return false;
  const uint32_t add = sums[blockIdx.x];
  for (int k = b0 + threadIdx.x; k < b1; k += kRbThreads) a[k] += add;
  return grid_barrier(bar, status);
}

// The rebuild over the whole grid (all CTAs resident, 256 threads each).  Returns false when a
// barrier gave up; the caller then leaves at once.
template <int D>
__device__ bool rebuild_body(const RebuildArgs& r, RebuildSmem& sm) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *r.ntiles = 0;
    if (r.nwall) r.nwall[0] = r.nwall[1] = 0;
    if (r.ctl) {
      r.ctl->rebuilds += 1;
      r.ctl->call_rebuilds += 1;
    }
  }
  uint32_t *ki = r.kA, *vi = r.vA, *ko = r.kB, *vo = r.vB;
  const int M = 256 * r.nb;
  for (int p = 0; p < r.passes; ++p) {
    for (int tile = blockIdx.x; tile < r.nb; tile += gridDim.x) {
      if (p == 0 && D == 3 && r.boff)
        sort_hist_tile<D, 2>(tile, ki, r.N, 0, r.hist, r.nb, r.segs, r.in, sm.hist);
      else if (p == 0)
        sort_hist_tile<D, 1>(tile, ki, r.N, 0, r.hist, r.nb, r.segs, r.in, sm.hist);
      else
        sort_hist_tile<D, false>(tile, ki, r.N, 8 * p, r.hist, r.nb, r.segs, r.in, sm.hist);
      __syncthreads();
    }
    if (!grid_barrier(r.bar, r.status)) return false;
    if (!grid_scan(r.hist, M, r.sums, sm.wsum, r.bar, r.status)) return false;
    for (int tile = blockIdx.x; tile < r.nb; tile += gridDim.x) {
      if (p == 0 && D == 3 && r.boff)
        sort_scatter_tile<D, 2>(tile, ki, vi, ko, vo, r.N, 0, r.hist, r.nb, r.segs, r.in, sm.scatter);
      else if (p == 0)
        sort_scatter_tile<D, 1>(tile, ki, vi, ko, vo, r.N, 0, r.hist, r.nb, r.segs, r.in, sm.scatter);
      else
        sort_scatter_tile<D, false>(tile, ki, vi, ko, vo, r.N, 8 * p, r.hist, r.nb, r.segs, r.in, sm.scatter);
      __syncthreads();
    }
    if (!grid_barrier(r.bar, r.status)) return false;
    uint32_t* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  // permute into `out` with the cell ranges and the displacement reference
  for (int k = blockIdx.x * kRbThreads + threadIdx.x; k <= r.N; k += gridDim.x * kRbThreads)
    permute_one<D>(k, r.segs, r.N, vi, r.in, r.out, ki, r.C, r.off, r.xb, D == 3 ? r.boff : nullptr);
  if (!grid_barrier(r.bar, r.status)) return false;
  // back into `in` (the buffer parity of the step does not depend on the rebuild), and the tiles
  if (r.copy_back)
    for (int k = blockIdx.x * kRbThreads + threadIdx.x; k < r.N; k += gridDim.x * kRbThreads)
      copy_state_one<D>(k, r.out, r.in);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kRbThreads + threadIdx.x) >> 5, nwarps = gridDim.x * (kRbThreads / 32);
  for (int l = warp; l < r.n_lines; l += nwarps)
    tiles_line<D>(l, lane, r.segs, r.S, r.line_base, r.off, r.tiles, r.ntiles);
  if (r.wall_list) {
    if (!grid_barrier(r.bar, r.status)) return false;
    const int nt = *(volatile int*)r.ntiles;
    for (int w = warp; w < nt; w += nwarps)
      list_tile<D>(r.tiles[w], w, lane, r.out.meta, r.wall_list, r.wall_plans, r.fluid_plans, r.nwall);
  }
  return true;
}


}  // namespace sph
