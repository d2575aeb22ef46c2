// Neighbour passes of the WCSPH step on the cell-block tiles (sph_tiles.cuh):
//   tile table      (built after every rebuild from the cell offsets)
//   walls           Shepard extrapolation of the fluid pressure onto wall particles
//   walls + sweep   both in one launch (wall tiles first; sweep tiles near walls wait for them)
//   mDBC walls      first-order extrapolation from ghost nodes (a warp per wall particle)
//   density         summation density rho_i = sum_j m_j W_ij            (Sec. 2.3)
//   gradient        renormalised density gradient <grad rho>^L (kernel renormalisation, App. A)
//   sweep           continuity + delta diffusion, Tait pressure, viscosity, gravity, and the
//                   kick-drift epilogue (Sec. 2.3, Sec. 3.4); also the rate-only evaluation
//   shift           explicit particle shifting at the end of a step (free-surface aware)
//   opt P1..P4      shifting by optimisation: objective, its gradient, a descent step
//   pairs           exact pair export (FP64 predicate in a guard band; per-particle radii too)
//   variable support   search radius and super-symmetric / gather densities with radii H_i
//   adjoint sweep   vector-Jacobian product of one step, gathered per particle (Sec. 2.2)
#include <algorithm>
#include <map>

#include "sph_passes.cuh"
#include "sph_tilebuild.cuh"
#include "sph_warptiles.cuh"

namespace sph {

// Bounded wait of a sweep tile on the wall tasks of the fused kernel: ~0.1 s, then status bit 1.
constexpr long long kGateSpins = 1LL << 22;
// One thread waits until *gate >= n (then a fence orders its later reads), or gives up after
// kGateSpins polls, sets status bit 1 and returns false.
__device__ __noinline__ bool gate_wait(const unsigned* gate, unsigned n, int* status) {
  long long it = 0;
  while (*(volatile const unsigned*)gate < n) {
    if (++it > kGateSpins) {
      atomicOr(status, 2);
      return false;
    }
    __nanosleep(32);
  }
  __threadfence();
  return true;
}

// Test hook of the bounded waits: a gate that no task opens.
__global__ void k_debug_gate(const unsigned* gate, int* status) {
  if (threadIdx.x == 0) gate_wait(gate, 1u, status);
}
void launch_debug_gate(const unsigned* gate, int* status, cudaStream_t st) { k_debug_gate<<<1, 32, 0, st>>>(gate, status); }
// Relative cut-off of the pseudo-inverses (renormalisation, mDBC): eigen-directions with
// |lambda| <= kPinvRtol max|lambda| (or singular values <= kPinvRtol max) are dropped.
constexpr float kPinvRtol = 1e-3f;

// ================================================================== tile table
// (builders in sph_tilebuild.cuh)
template <int D>
__global__ void __launch_bounds__(256) k_tiles(const DevSeg* __restrict__ segs, int S,
                                               const int* __restrict__ line_base, int n_lines,
                                               const int* __restrict__ cell_off, Tile* __restrict__ tiles,
                                               int* __restrict__ ntiles) {
  const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (l < n_lines) tiles_line<D>(l, threadIdx.x & 31, segs, S, line_base, cell_off, tiles, ntiles);  // warp-uniform
}

// ================================================================== staged particle data
template <int D, int E, int LN>
__device__ __forceinline__ PD<D> smem_pd(const TileSmem<D, E, LN>& sm, int k) {
  PD<D> r;
  const float4 A = sm.A[k], B = sm.B[k];
  if (D == 2) {
    r.x[0] = A.x; r.x[1] = A.y; r.v[0] = A.z; r.v[1] = A.w;
    r.rho = B.x; r.p = B.y; r.V = B.z; r.m = B.w;
  } else {
    const float2 C = sm.C[k];
    r.x[0] = A.x; r.x[1] = A.y; r.x[2] = A.z; r.V = A.w;
    r.v[0] = B.x; r.v[1] = B.y; r.v[2] = B.z; r.p = B.w;
    r.rho = C.x; r.m = C.y;
  }
  return r;
}

// Candidate gathering of one target (this thread = one of LANES for the target): its own 3^d
// cells in shared memory, split across the LANES threads, hits collected in a per-thread list and
// evaluated by body.pair(pj, extra, pp, j_global).  Returns the number of pairs evaluated.
// Neighbour lines and side cells that lie farther than the reach from the target (distance to
// the cell faces) are skipped.  List entries carry the staged index and, in bits 13..15, which
// axes take the box length off the target (periodic images on the upper side).
// SELF: 0 = exclude r^2 == 0 (gradient terms vanish there anyway), 1 = exclude by index,
// 2 = exact FP64 predicate in the guard band (pair export).
template <int D, int E, int SELF, class Body, int LN>
__device__ __forceinline__ int gather_staged(TileSmem<D, E, LN>& sm, const DevSeg& s, const Arrays& a, int i, int ccol,
                                             const float* xt0, const float* face_lo, const float* face_hi,
                                             Body& body) {
  using Cfg = TileCfg<D>;
  constexpr int CAP = Cfg::CAP;
  constexpr int THREADS = TileSmem<D, E, LN>::THREADS;
  const int lane = threadIdx.x % LN;
  unsigned short* list = sm.list + threadIdx.x;
  int cnt = 0, npair = 0;
  const float H2 = s.H2;
  const float R2 = s.trimR2;
  auto drain = [&]() {
    for (int e = 0; e < cnt; ++e) {
      const unsigned code = list[e * THREADS];
      const int k = (int)(code & 0x1fffu);  // bits 0..12: staged index (CAP <= 8192)
      PD<D> pj = smem_pd(sm, k);
      // periodic image of the entry: the target takes off the box length on the flagged axes
      // (an exact shift: the target lies in the upper half of the box on those axes)
      float xs[D];
      if (D == 2) {  // (2D: most entries carry no shift)
#pragma unroll
        for (int q = 0; q < D; ++q) xs[q] = xt0[q];
        if (code >> 13) {
#pragma unroll
          for (int q = 0; q < D; ++q)
            if ((code >> (13 + q)) & 1u) xs[q] -= s.L[q];
        }
      } else {
#pragma unroll
        for (int q = 0; q < D; ++q) xs[q] = xt0[q] - ((code >> (13 + q)) & 1u ? s.L[q] : 0.f);
      }
      float4 ex = make_float4(0.f, 0.f, 0.f, 0.f);
      float pp = 0.f;
      if (E > 0) ex = sm.E[k];
      if (E > 1) pp = sm.E[CAP + k].x;
      body.pair_at(xs, pj, ex, pp, SELF == 2 ? staged_gidx(sm, k) : 0);
    }
    npair += cnt;
    cnt = 0;
  };
  // squared distances of the target to its own cell's faces (0 if it has drifted past one)
  float fl[3], fh[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float a0 = q < D ? fmaxf(xt0[q] - face_lo[q], 0.f) : 0.f;
    const float a1 = q < D ? fmaxf(face_hi[q] - xt0[q], 0.f) : 0.f;
    fl[q] = a0 * a0;
    fh[q] = a1 * a1;
  }
  // Each lane of the target's group sets up the candidate runs of one staged line (lane j: lines
  // j, j + LANES, ...): [lo, hi) in staged order, mid = start of the right periodic image (the
  // target takes off L in x from there on), and the line's y/z image bits.  The loop over lines
  // then fetches each line's run with two shuffles instead of every lane redoing the setup.
  constexpr int NL = Cfg::NL, LANES = LN;
  constexpr int NSLOT = (NL + LANES - 1) / LANES;
  static_assert(NSLOT <= 2, "a lane sets up at most two lines");
  const unsigned gmask = (LANES == 32 ? 0xffffffffu : ((1u << LANES) - 1u)) << ((threadIdx.x & 31) & ~(LANES - 1));
  unsigned runA[NSLOT], runB[NSLOT];
#pragma unroll
  for (int q = 0; q < NSLOT; ++q) {
    const int l = lane + q * LANES;
    unsigned A = 0u, B = 0u;  // empty run
    if (l < NL && sm.linecell[l] >= 0) {
      const int dy = (D == 2) ? l - 1 : l % 3 - 1;
      const int dz = (D == 2) ? 0 : l / 3 - 1;
      const float dyz = (dy < 0 ? fl[1] : dy > 0 ? fh[1] : 0.f) + (dz < 0 ? fl[2] : dz > 0 ? fh[2] : 0.f);
      if (dyz < R2) {
        const bool need_left = fl[0] + dyz < R2, need_right = fh[0] + dyz < R2;
        constexpr int NCOL = TileSmem<D, E, LN>::NCOL;
        const int lo = sm.colstart[l * NCOL + (need_left ? ccol - 1 : ccol)];
        const int hi = sm.colstart[l * NCOL + (need_right ? ccol + 2 : ccol + 1)];
        const bool wrap_right = need_right && (sm.colbase + ccol + 1 >= s.n[0]);
        const int mid = wrap_right ? sm.colstart[l * NCOL + ccol + 1] : hi;
        const unsigned lbits = (sm.tshift[l][1] != 0.f ? 2u : 0u) | (D == 3 && sm.tshift[l][2] != 0.f ? 4u : 0u);
        A = (unsigned)lo | ((unsigned)hi << 16);
        B = (unsigned)mid | (lbits << 16);
      }
    }
    runA[q] = A;
    runB[q] = B;
  }
#pragma unroll 1
  for (int l = 0; l < NL; ++l) {
    const int src = l % LANES;
    const bool second = NSLOT > 1 && l >= LANES;
    const unsigned A = __shfl_sync(gmask, second ? runA[NSLOT - 1] : runA[0], src, LANES);
    const unsigned B = __shfl_sync(gmask, second ? runB[NSLOT - 1] : runB[0], src, LANES);
    const int lo = (int)(A & 0xffffu), hi = (int)(A >> 16), mid = (int)(B & 0xffffu);
    if (lo >= hi) continue;
    const unsigned lshift = (B >> 16) << 13;
    float tx = xt0[0];
    const float ty = (lshift & (1u << 14)) ? xt0[1] - s.L[1] : xt0[1];
    const float tz = (D == 3) ? ((lshift & (1u << 15)) ? xt0[2] - s.L[2] : xt0[2]) : 0.f;
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      const int b = part == 0 ? lo : mid, en = part == 0 ? mid : hi;
      unsigned shift_bits = lshift;
      if (part == 1) {
        if (b >= en) break;
        tx -= s.L[0];
        shift_bits |= 1u << 13;
      }
      for (int k0 = b + lane; k0 < en; k0 += 4 * LN) {
        if (cnt > Cfg::LIST - 4) drain();
        if constexpr (D == 3 && SELF == 0) {
          // branch-free in 3D (-1 % there, +1.5 % in 2D): every slot is tested (an index past the
          // run is clamped to a valid one and rejected) and written at the list's end, which only
          // a hit advances (cnt <= LIST - 4 here, so the four writes stay in the list); the list
          // is the same as the branching form's
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int k = k0 + u * LN;
            const int kc = min(k, en - 1);
            const float4 P = sm.A[kc];
            const float dx = tx - P.x, dy2 = ty - P.y, dz2 = tz - P.z;
            const float r2 = fmaf(dz2, dz2, fmaf(dy2, dy2, dx * dx));
            list[cnt * THREADS] = (unsigned short)(kc | shift_bits);
            cnt += (k < en && r2 < H2 && r2 > 0.f) ? 1 : 0;
          }
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int k = k0 + u * LN;
            if (k < en) {
              const float4 P = sm.A[k];
              const float dx = tx - P.x, dy2 = ty - P.y;
              float r2 = fmaf(dy2, dy2, dx * dx);
              if (D == 3) {
                const float dz2 = tz - P.z;
                r2 = fmaf(dz2, dz2, r2);
              }
              bool in;
              if (SELF == 2) {
                in = r2 < s.band_hi;
                if (in) {
                  const int gj = staged_gidx(sm, k);
                  in = gj != i;
                  if (in && r2 >= s.band_lo) in = exact_pair<D>(s, a, i, gj);
                }
              } else if (SELF == 1) {
                in = r2 < H2 && (r2 > 0.f || staged_gidx(sm, k) != i);
              } else {
                in = r2 < H2 && r2 > 0.f;
              }
              if (in) {
                list[cnt * THREADS] = (unsigned short)(k | shift_bits);
                ++cnt;
              }
            }
          }
        }
      }
    }
  }
  drain();
  return npair;
}

// Fallback for tiles whose staged region does not fit: the target's own 3^d cells straight from
// global memory, one thread per target (the caller lets only lane 0 of the group do this).
template <int D, int SELF, bool COH, class Body>
__device__ int gather_global(const DevSeg& s, const Arrays& a, const uint32_t* __restrict__ keys, int kshift,
                             const int* __restrict__ cell_off, const float4* __restrict__ extra0,
                             const float* __restrict__ extra1, int i, const float* xi, Body& body) {
  int c[3];
  key_coords(s, keys[i] >> kshift, c);
  int npair = 0;
  const int zlo = (D == 3) ? -1 : 0, zhi = (D == 3) ? 1 : 0;
  for (int oz = zlo; oz <= zhi; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        int cc[3] = {c[0] + ox, c[1] + oy, c[2] + oz};
        bool skip = false;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          if (cc[k] < 0 || cc[k] >= s.n[k]) {
            if (!((s.periodic_mask >> k) & 1)) skip = true;
            cc[k] = (cc[k] + s.n[k]) % s.n[k];
          }
        }
        if (skip) continue;
        const int cell = s.cell_base + (cc[2] * s.n[1] + cc[1]) * s.n[0] + cc[0];
        for (int j = cell_off[cell]; j < cell_off[cell + 1]; ++j) {
          const PD<D> pj = load_pd<D, COH>(a, j);
          float r[D];
          const float r2 = separation<D>(s, xi, pj.x, r);
          bool in;
          if (SELF == 2) {
            in = j != i && r2 < s.band_hi;
            if (in && r2 >= s.band_lo) in = exact_pair<D>(s, a, i, j);
          } else if (SELF == 1) {
            in = j != i && r2 < s.H2;
          } else {
            in = r2 < s.H2 && r2 > 0.f;
          }
          if (in) {
            float4 ex = extra0 ? __ldg(extra0 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
            float pp = extra1 ? __ldg(extra1 + j) : 0.f;
            // place the neighbour at its nearest image relative to the target
            PD<D> pm = pj;
#pragma unroll
            for (int q = 0; q < D; ++q) pm.x[q] = xi[q] - r[q];
            body.pair_at(xi, pm, ex, pp, j);
            ++npair;
          }
        }
      }
  return npair;
}

// sum over the LANES threads of one target (all threads of the warp call this)
template <int LANES>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
template <int LANES>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// One tile of a pass: stage, gather per target, reduce, epilogue (or skip).  Returns the pairs
// evaluated by this thread.  gate (fused wall + sweep kernel): the tile may read records that the
// launch's wall tasks rewrite; unless all gate_n wall tasks had finished when the tile started
// (an acquire load of the counter), a tile whose staged region holds a wall particle waits for
// them (bounded) and loads its wall particles again, through L2 (COH); one that falls back to
// global memory waits before it reads any neighbour.  A tile without a target of the pass does not wait: the fused sweep's
// skip touches nothing.  (Only wall records change: the fluid entries and the target cache, whose
// wall targets the sweep does not use, stay valid.)
template <int D, int E, int SELF, bool COH, class Pass, int LN>
__device__ __forceinline__ int tile_task(const TravArgs& t, const Tile& T, TileSmem<D, E, LN>& sm,
                                         const float4* __restrict__ extra0, const float* __restrict__ extra1,
                                         Pass& pass, const unsigned* gate = nullptr, unsigned gate_n = 0,
                                         uint4* plan = nullptr, int gate_ready = -1) {
  using Cfg = TileCfg<D>;
  __shared__ int s_ready;
  const DevSeg& s = t.segs[T.seg];
  const int tgt = threadIdx.x / LN;
  const int lane = threadIdx.x % LN;
  const int i = T.p0 + tgt;
  const bool valid = i < T.p1;
  // (gate_ready: the caller's reading of the gate, taken before a barrier that precedes every load
  // of this task; a plan's records are loaded without a barrier of their own before them)
  if (gate && threadIdx.x == 0) s_ready = gate_ready >= 0 ? gate_ready : ld_acquire(gate) >= gate_n;
  // the targets' own records go to the cache while the neighbours are staged; the key and the
  // meta word (for the skip decision) are requested now so that their loads overlap too
  fill_target_cache<D, COH>(sm.tc, t.a, pass.tex0(), pass.tex1(), T.p0, T.p1 - T.p0);
  const int key = valid ? (int)(t.keys[i] >> t.kshift) : 0;
  // tiles without a target of this pass (walls only, fluid only) are skipped unstaged
  const bool want = valid && lane == 0 && Pass::wants(t.a.meta[i].x);
  int seen = 1;
  int stg;
  if (TilePlan<D>::CACHED && plan && sm.pvalid) {
    // the staging table is the plan's (loaded with the tile): the records at once, then one
    // barrier for the records, the target cache and the decisions
    stg = 1;
    if (sm.fallback) {
      stg = 0;
      cp_async_wait_all();
    } else {
      int walls = 0;
      for (int k = threadIdx.x; k < sm.total; k += blockDim.x) walls |= stage_record<D, E, COH>(sm, t.a, k, extra0, extra1);
      cp_async_wait_all();
      seen = __syncthreads_or(walls);
    }
    if (!__syncthreads_or(want)) stg = -1;
  } else {
    stg = stage_tile<D, E, COH>(sm, s, T, t.a, t.cell_off, extra0, extra1, want, gate ? &seen : nullptr);
    if (TilePlan<D>::CACHED && plan && stg == 1) store_plan(sm, plan);  // for the steps up to the next rebuild
  }
  if (gate && !s_ready && (stg == 0 || (stg == 1 && seen))) {  // uniform over the CTA (barrier results)
    if (threadIdx.x == 0) gate_wait(gate, gate_n, t.status);
    __syncthreads();
    if (stg == 1) restage_walls(sm, t.a, extra0, extra1);
  }
  const TgtView tv{sm.tc.view(), sm.tc.E0, sm.tc.E1, tgt};
  int np = 0;
  if (stg >= 0) {
    const bool staged = stg > 0;
    typename Pass::Body body;
    bool active = false;
    int ccol = 0;
    float xi[3] = {0.f, 0.f, 0.f}, flo[3] = {0.f, 0.f, 0.f}, fhi[3] = {0.f, 0.f, 0.f};
    if (valid) {
      active = pass.init(body, s, i, tv);
      const float4 A = tv.a.A[tgt];
      xi[0] = A.x; xi[1] = A.y; xi[2] = A.z;
      const int c[3] = {key - (s.cell_base + (T.cz * s.n[1] + T.cy) * s.n[0]), T.cy, T.cz};
      ccol = c[0] - (staged ? sm.colbase : 0);
#pragma unroll
      for (int q = 0; q < D; ++q) {
        flo[q] = s.lo[q] + s.cs[q] * (float)c[q];
        fhi[q] = flo[q] + s.cs[q];
      }
    }
    if (active) {
      if (staged)
        np = gather_staged<D, E, SELF>(sm, s, t.a, i, ccol, xi, flo, fhi, body);
      else if (lane == 0)
        np = gather_global<D, SELF, COH>(s, t.a, t.keys, t.kshift, t.cell_off, extra0, extra1, i, xi, body);
    }
    __syncwarp();
    body.template reduce<LN>();
    if (valid && lane == 0) pass.finish(body, s, i, tv);
  } else if (valid && lane == 0) {
    pass.skip(i, tv);
  }
  return np;
}

// The end of a tiled launch: the pass's partial results, the pair count, and the last CTA to
// finish zeroes the tile counters (ctr[0] task counter, ctr[1] finished CTAs, ctr[2] finished
// wall tasks of the fused kernel) for the next launch: every CTA has taken its last task index,
// and flushed its partial results, before it counts itself done.
template <class Pass>
__device__ __forceinline__ void end_tiles(const TravArgs& t, Pass& pass, long long pairs_cta) {
  pass.flush();
  if (t.pair_count) {
    long long v = pairs_cta;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(t.pair_count, (unsigned long long)v);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(t.tile_ctr + 1, 1) == (int)gridDim.x - 1) {
      __threadfence();
      t.tile_ctr[0] = 0;
      t.tile_ctr[1] = 0;
      t.tile_ctr[2] = 0;
      pass.last_cta();
    }
  }
}

// Common skeleton of a tiled pass: tiles are handed out dynamically (one atomic per CTA and tile)
// after a first tile per CTA by block index: load balance whatever the occupancy and the tile
// sizes, and no atomic on the first tile's path.  A list selects a subset of the tiles.
template <int D, int E, int SELF, class Pass, int LN = TileCfg<D>::LANES>
__device__ __forceinline__ void run_tiles(const TravArgs& t, const Tile* __restrict__ tiles, const int* __restrict__ ntiles,
                                          const float4* __restrict__ extra0, const float* __restrict__ extra1,
                                          Pass& pass, const int* __restrict__ tile_list = nullptr) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TileSmem<D, E, LN>& sm = *reinterpret_cast<TileSmem<D, E, LN>*>(smraw);
  __shared__ int s_tile;
  const int nt = *ntiles;
  long long pairs_cta = 0;
  int ti = blockIdx.x;
  while (ti < nt) {
    const Tile T = tiles[tile_list ? tile_list[ti] : ti];
    pairs_cta += tile_task<D, E, SELF, false>(t, T, sm, extra0, extra1, pass);
    __syncthreads();  // shared memory is restaged for the next tile
    if (threadIdx.x == 0) s_tile = gridDim.x + atomicAdd(t.tile_ctr, 1);
    __syncthreads();
    ti = s_tile;
  }
  end_tiles(t, pass, pairs_cta);
}

// ================================================================== mDBC walls
// One warp per wall particle b of the wall tiles: the fluid particles within H of its ghost node g
// (the 3^d cells around g's cell, read from global memory and split over the lanes) give the
// first-order system of the paper's boundary section for q = rho - rho0, in units of H:
//   [ <1>          <x_jg>^T / H    ] [ f    ]   [ <q>          ]
//   [ H <grad 1>   <grad (x) x_jg> ] [ H f' ] = [ H <grad q>   ]
// (<q> = sum_j V_j q_j W(x_g - x_j), grad = grad_g, x_jg = x_j - x_g), summed in FP32 and solved
// by a pseudo-inverse (one-sided Jacobi SVD; singular values at or below kPinvRtol of the largest
// dropped); rho_b = rho0 + f + x_bg . f' with x_bg = x_b - x_g, rho0 when no fluid is in
// range.  The density deviation q (exact in FP32 for densities near rho0) keeps the right-hand
// side small, so the FP32 sums lose nothing against the large rest density, and the pressure is
// taken from the deviation directly.  The walls' records are rewritten in place (only their
// density, pressure and volume change).
// Minimum-norm least-squares solution u = pinv(A) b of the n x n system by one-sided Jacobi
// (Hestenes): plane rotations A V make the columns orthogonal, so A = U S V^T with the column
// norms as singular values; u = sum_k v_k (a_k . b) / s_k^2 over s_k > kPinvRtol max s (the same
// cut-off as the oracle's).  FP32, registers only; the condition number enters once (no normal
// equations).
template <int N>
__device__ __forceinline__ void mdbc_solve(const float (&A)[N][N], const float (&b)[N], float (&u)[N]) {
  float a[N][N], v[N][N];
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c < N; ++c) {
      a[r][c] = A[r][c];
      v[r][c] = r == c ? 1.f : 0.f;
    }
#pragma unroll 1
  for (int sweep = 0; sweep < 12; ++sweep) {
    bool rotated = false;
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
      for (int q = p + 1; q < N; ++q) {
        float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          al = fmaf(a[k][p], a[k][p], al);
          be = fmaf(a[k][q], a[k][q], be);
          ga = fmaf(a[k][p], a[k][q], ga);
        }
        if (!(fabsf(ga) > 1e-7f * sqrtf(al) * sqrtf(be))) continue;
        rotated = true;
        const float zeta = (be - al) / (2.f * ga);
        const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
        const float c = rsqrtf(fmaf(t, t, 1.f)), sn = c * t;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const float ap = a[k][p], aq = a[k][q];
          a[k][p] = c * ap - sn * aq;
          a[k][q] = sn * ap + c * aq;
          const float vp = v[k][p], vq = v[k][q];
          v[k][p] = c * vp - sn * vq;
          v[k][q] = sn * vp + c * vq;
        }
      }
    if (!rotated) break;
  }
  float s2[N], s2max = 0.f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float n2 = 0.f;
#pragma unroll
    for (int r = 0; r < N; ++r) n2 = fmaf(a[r][k], a[r][k], n2);
    s2[k] = n2;
    s2max = fmaxf(s2max, n2);
  }
#pragma unroll
  for (int r = 0; r < N; ++r) u[r] = 0.f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (!(s2[k] > kPinvRtol * kPinvRtol * s2max)) continue;
    float ab = 0.f;
#pragma unroll
    for (int r = 0; r < N; ++r) ab = fmaf(a[r][k], b[r], ab);
    const float coef = ab / s2[k];
#pragma unroll
    for (int r = 0; r < N; ++r) u[r] = fmaf(coef, v[r][k], u[r]);
  }
}

// Tasks: slices of 8 consecutive particles of the wall tiles, one warp per particle.
template <int D, int KERN>
__global__ void __launch_bounds__(256) k_mdbc(TravArgs t, const Tile* __restrict__ tiles,
                                              const int* __restrict__ wall_tiles, const int* __restrict__ n_wall_tiles,
                                              const float4* __restrict__ ghost, const int* __restrict__ orig_base) {
  constexpr int N = D + 1, NS = N * N + N;  // the system and its right-hand side
  constexpr int SLICES = TileCfg<D>::TP / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntask = *n_wall_tiles * SLICES;
  for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
    const Tile T = tiles[wall_tiles[task / SLICES]];
    const DevSeg& s = t.segs[T.seg];
    const int i = T.p0 + (task % SLICES) * 8 + warp;
    if (i < T.p1) {
      const uint2 m = t.a.meta[i];
      if (!(m.x & kWallBit)) continue;  // warp-uniform (the whole warp has this particle)
      const float4 G4 = __ldg(ghost + orig_base[m.y] + (int)(m.x & ~kWallBit));
      float xg[3] = {G4.x, G4.y, G4.z};
      int c[3] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < D; ++k) {
        if ((s.periodic_mask >> k) & 1) xg[k] -= s.L[k] * floorf((xg[k] - s.lo[k]) * s.invL[k]);
        c[k] = min(max((int)floorf((xg[k] - s.lo[k]) * s.invcs[k]), 0), s.n[k] - 1);
      }
      float acc[NS];
#pragma unroll
      for (int e = 0; e < NS; ++e) acc[e] = 0.f;
      // the 3^d cells around the ghost node in one round trip: lane k < NC holds cell k's first
      // particle and count; the warp then walks their concatenation, 32 candidates per round
      constexpr int NC = D == 3 ? 27 : 9;
      int cfirst = 0, ccount = 0;
      if (lane < NC) {
        int cc[3] = {c[0] + lane % 3 - 1, c[1] + (lane / 3) % 3 - 1, c[2] + (D == 3 ? lane / 9 - 1 : 0)};
        bool skip = false;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          if (cc[k] < 0 || cc[k] >= s.n[k]) {
            if (!((s.periodic_mask >> k) & 1)) skip = true;
            cc[k] = (cc[k] + s.n[k]) % s.n[k];
          }
        }
        if (!skip) {
          const int cell = s.cell_base + (cc[2] * s.n[1] + cc[1]) * s.n[0] + cc[0];
          cfirst = t.cell_off[cell];
          ccount = t.cell_off[cell + 1] - cfirst;
        }
      }
      int incl = ccount;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      const int excl = incl - ccount;
      for (int base = 0; base < total; base += 32) {
        const int idx = base + lane;
        // the cell holding walk position idx: the smallest b with incl_b > idx (incl is
        // non-decreasing over the lanes, and only a non-empty cell raises it), by a binary
        // search over the lanes' prefix sums; then that cell's first particle and offset
        int lo = 0, hi = NC - 1;
#pragma unroll
        for (int step = 0; step < 5; ++step) {  // NC <= 32
          const int mid = (lo + hi) >> 1;
          if (__shfl_sync(kFull, incl, mid) > idx) hi = mid;
          else lo = mid + 1;
        }
        const int fb = __shfl_sync(kFull, cfirst, hi), eb = __shfl_sync(kFull, excl, hi);
        if (idx >= total) continue;
        const int j = fb + (idx - eb);
        const PD<D> pj = load_pd<D>(t.a, j);
        if (!(pj.m > 0.f)) continue;  // fluid only
        float r[D];
        const float r2 = separation<D>(s, xg, pj.x, r);  // x_g - x_j
        if (!(r2 < s.H2)) continue;
        const float q = safe_q(r2, s.invH);
        const float VW = pj.V * (s.Kw * kern_w<KERN>(q));
        const float VgH = pj.V * (s.Kg * kern_gt<KERN>(q)) * s.H;  // V grad W / r, times H
        acc[0] += VW;
#pragma unroll
        for (int l = 0; l < D; ++l) acc[1 + l] = fmaf(-VW * s.invH, r[l], acc[1 + l]);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          acc[(1 + k) * N] = fmaf(VgH, r[k], acc[(1 + k) * N]);
#pragma unroll
          for (int l = 0; l < D; ++l)
            acc[(1 + k) * N + 1 + l] = fmaf(-VgH * s.invH * r[k], r[l], acc[(1 + k) * N + 1 + l]);
        }
        const float qj = pj.rho - s.rho0;
        acc[N * N] = fmaf(VW, qj, acc[N * N]);
#pragma unroll
        for (int k = 0; k < D; ++k) acc[N * N + 1 + k] = fmaf(VgH * qj, r[k], acc[N * N + 1 + k]);
      }
#pragma unroll
      for (int e = 0; e < NS; ++e)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[e] += __shfl_xor_sync(kFull, acc[e], o);
      if (lane == 0) {
        PD<D> me = load_pd<D>(t.a, i);
        double q = 0.0;  // rho_b - rho0
        if (acc[0] > 0.f) {
          float A[N][N], bb[N], u[N];
#pragma unroll
          for (int a = 0; a < N; ++a) {
#pragma unroll
            for (int cix = 0; cix < N; ++cix) A[a][cix] = acc[a * N + cix];
            bb[a] = acc[N * N + a];
          }
          mdbc_solve<N>(A, bb, u);
          float xb[D];
          const float rbg2 = separation<D>(s, me.x, xg, xb);  // x_b - x_g
          (void)rbg2;
          q = (double)u[0];
#pragma unroll
          for (int k = 0; k < D; ++k) q += (double)xb[k] * (double)u[1 + k] / (double)s.H;
        }
        const float rb = (float)((double)s.rho0 + q);
        me.rho = rb;
        me.p = s.B * expm1f(s.gamma * log1pf((float)(q / (double)s.rho0)));
        me.V = fabsf(me.m) / rb;
        store_pd<D>(t.a, i, me);
      }
      __syncwarp();
    }
  }
}

// ================================================================== walls
template <int D, int KERN>
struct WallPass {
  struct Body {
    const DevSeg* s;
    float xi[D];
    float sW, sp, sh;
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4, float, int) {
      if (pj.m < 0.f) return;  // wall neighbour
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      const float W = s->Kw * kern_w<KERN>(safe_q(r2, s->invH));
      float gr = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) gr = fmaf(s->g[k], r[k], gr);
      sW += W;
      sp = fmaf(pj.p, W, sp);
      sh = fmaf(pj.rho * gr, W, sh);
    }
    template <int L>
    __device__ __forceinline__ void reduce() {
      sW = group_sum<L>(sW);
      sp = group_sum<L>(sp);
      sh = group_sum<L>(sh);
    }
  };
  Arrays a;
  Arrays out{};  // optional: the records are written here too
  // superset of the targets init() activates, from the meta word alone
  __device__ static __forceinline__ bool wants(uint32_t m) { return (m & kWallBit) != 0; }
  __device__ __forceinline__ void skip(int, const TgtView&) {}
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return nullptr; }
  __device__ __forceinline__ const float4* tex1() const { return nullptr; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int, const TgtView& tv) {
    b.s = &s;
    b.sW = b.sp = b.sh = 0.f;
    const uint2 m = tv.a.meta[tv.k];
    const float4 A = tv.a.A[tv.k];
    b.xi[0] = A.x; b.xi[1] = A.y;
    if (D == 3) b.xi[2] = A.z;
    return (m.x & kWallBit) != 0;
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    const uint2 m = tv.a.meta[tv.k];
    if (!(m.x & kWallBit)) return;
    const float pw = b.sW > 0.f ? (b.sp + b.sh) / b.sW : 0.f;
    const float rw = tait_rho(s, pw);
    PD<D> me = load_pd_plain<D>(tv.a, tv.k);
    me.rho = rw;
    me.p = pw;
    me.V = fabsf(me.m) / rw;
    store_pd<D>(a, i, me);
    if (out.A) {  // the step's output buffer as well (the fused sweep does not copy walls)
      store_pd<D>(out, i, me);
      store_cold<D>(out, i, load_cold<D>(tv.a, tv.k));
      out.meta[i] = m;
    }
  }
};

// ================================================================== density
template <int D, int KERN>
struct DensityPass {
  struct Body {
    const DevSeg* s;
    float xi[D];
    float rh, rl;  // compensated FP32 sum (FP64 accuracy without FP64 arithmetic per pair)
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4, float, int) {
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      two_sum_acc(rh, rl, fabsf(pj.m) * (s->Kw * kern_w<KERN>(safe_q(r2, s->invH))));
    }
    template <int L>
    __device__ __forceinline__ void reduce() {
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(kFull, rh, o), ol = __shfl_xor_sync(kFull, rl, o);
        two_sum_merge(rh, rl, oh, ol);
      }
    }
  };
  Arrays a;
  __device__ static __forceinline__ bool wants(uint32_t m) { return (m & kWallBit) == 0; }
  __device__ __forceinline__ void skip(int, const TgtView&) {}
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return nullptr; }
  __device__ __forceinline__ const float4* tex1() const { return nullptr; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int, const TgtView& tv) {
    b.s = &s;
    b.rh = b.rl = 0.f;
    const float4 A = tv.a.A[tv.k];
    b.xi[0] = A.x; b.xi[1] = A.y;
    if (D == 3) b.xi[2] = A.z;
    return !(tv.a.meta[tv.k].x & kWallBit);
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    if (tv.a.meta[tv.k].x & kWallBit) return;
    PD<D> me = load_pd_plain<D>(tv.a, tv.k);
    const double rho = ((double)b.rh + (double)b.rl) + (double)(me.m * s.Kw);  // self term, w(0) = 1
    const float e = (float)((rho - (double)s.rho0) / (double)s.rho0);
    me.rho = (float)rho;
    me.p = s.B * expm1f(s.gamma * log1pf(e));
    me.V = me.m / me.rho;
    store_pd<D>(a, i, me);
    Cold c = load_cold<D>(tv.a, tv.k);
    c.rlo = (float)(rho - (double)me.rho);
    store_cold<D>(a, i, c);
  }
};

// ================================================================== renormalised density gradient
// Kernel renormalisation (App. A, after Marrone et al.), for every particle (fluid and wall):
//   M_i = sum_j V_j (x_j - x_i) (x) grad_i W_ij = -sum_j V_j gK r (x) r      (symmetric)
//   s_i = sum_j V_j (rho_j - rho_i) grad_i W_ij,       <grad rho>_i^L = pinv(M_i) s_i
// (L_i applies to every term of the sum, so it is taken out of it).  The pseudo-inverse keeps
// the eigen-directions with |lambda| > kPinvRtol max|lambda|.

// pinv of the symmetric 2x2 [a b; b c] in closed form: (Lxx, Lxy, Lyy)
__device__ __forceinline__ void pinv_sym2(float a, float b, float c, float* L) {
  const float mean = 0.5f * (a + c), half = 0.5f * (a - c);
  const float rt = sqrtf(fmaf(half, half, b * b));
  const float l1 = mean + rt, l2 = mean - rt;
  const float cut = kPinvRtol * fmaxf(fabsf(l1), fabsf(l2));
  const bool k1 = fabsf(l1) > cut, k2 = fabsf(l2) > cut;
  L[0] = L[1] = L[2] = 0.f;
  if (k1 && k2) {
    const float inv = 1.f / fmaf(a, c, -b * b);
    L[0] = c * inv;
    L[1] = -b * inv;
    L[2] = a * inv;
  } else if (k1 || k2) {
    const float l = k1 ? l1 : l2;
    // eigenvector of l: (b, l - a) or (l - c, b), whichever is longer
    float ex = b, ey = l - a;
    const float fx = l - c, fy = b;
    if (fmaf(fx, fx, fy * fy) > fmaf(ex, ex, ey * ey)) {
      ex = fx;
      ey = fy;
    }
    const float n2 = fmaf(ex, ex, ey * ey);
    if (n2 > 0.f) {
      const float w = 1.f / (n2 * l);
      L[0] = ex * ex * w;
      L[1] = ex * ey * w;
      L[2] = ey * ey * w;
    } else {  // b = 0 and l on the diagonal
      L[0] = fabsf(a) > cut ? 1.f / a : 0.f;
      L[2] = fabsf(c) > cut ? 1.f / c : 0.f;
    }
  }
}

// Eigen-decomposition of a symmetric 3x3 by cyclic Jacobi rotations (Golub & Van Loan,
// Sec. 8.5), FP32: A becomes diagonal (the eigenvalues), Q (if wanted) collects the eigenvectors
// as columns.  m = (xx, xy, xz, yy, yz, zz).
template <bool VECTORS>
__device__ __forceinline__ void jacobi_sym3(const float* m, float A[3][3], float Q[3][3]) {
  A[0][0] = m[0]; A[0][1] = m[1]; A[0][2] = m[2];
  A[1][0] = m[1]; A[1][1] = m[3]; A[1][2] = m[4];
  A[2][0] = m[2]; A[2][1] = m[4]; A[2][2] = m[5];
  if (VECTORS) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Q[a][b] = a == b ? 1.f : 0.f;
  }
#pragma unroll 1
  for (int sweep = 0; sweep < 8; ++sweep) {
    const float off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const float dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (!(off > 1e-14f * dia)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const float apq = A[p][q];
      if (apq == 0.f) continue;
      const float tau = (A[q][q] - A[p][p]) / (2.f * apq);
      const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
      const float c = rsqrtf(fmaf(t, t, 1.f)), sn = t * c;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float akp = A[k][p], akq = A[k][q];
        A[k][p] = c * akp - sn * akq;
        A[k][q] = sn * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float apk = A[p][k], aqk = A[q][k];
        A[p][k] = c * apk - sn * aqk;
        A[q][k] = sn * apk + c * aqk;
      }
      if (VECTORS) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float qkp = Q[k][p], qkq = Q[k][q];
          Q[k][p] = c * qkp - sn * qkq;
          Q[k][q] = sn * qkp + c * qkq;
        }
      }
    }
  }
}

// pinv of a symmetric 3x3, m = (xx, xy, xz, yy, yz, zz) in and L (same packing) out.
__device__ __forceinline__ void pinv_sym3(const float* m, float* L) {
  float A[3][3], Q[3][3];
  jacobi_sym3<true>(m, A, Q);
  const float lam[3] = {A[0][0], A[1][1], A[2][2]};
  const float cut = kPinvRtol * fmaxf(fabsf(lam[0]), fmaxf(fabsf(lam[1]), fabsf(lam[2])));
#pragma unroll
  for (int e = 0; e < 6; ++e) L[e] = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (!(fabsf(lam[k]) > cut)) continue;
    const float w = 1.f / lam[k];
    L[0] = fmaf(Q[0][k] * Q[0][k], w, L[0]);
    L[1] = fmaf(Q[0][k] * Q[1][k], w, L[1]);
    L[2] = fmaf(Q[0][k] * Q[2][k], w, L[2]);
    L[3] = fmaf(Q[1][k] * Q[1][k], w, L[3]);
    L[4] = fmaf(Q[1][k] * Q[2][k], w, L[4]);
    L[5] = fmaf(Q[2][k] * Q[2][k], w, L[5]);
  }
}

template <int D, int KERN>
struct GradPass {
  static constexpr int NM = D * (D + 1) / 2;  // packed upper triangle of M
  struct Body {
    const DevSeg* s;
    float rho_i;
    float m[NM], g[D];
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4, float, int) {
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      const float VgK = pj.V * (s->Kg * kern_gt<KERN>(safe_q(r2, s->invH)));
      int e = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b, ++e) m[e] = fmaf(-VgK * r[a], r[b], m[e]);
      const float dr = VgK * (pj.rho - rho_i);
#pragma unroll
      for (int k = 0; k < D; ++k) g[k] = fmaf(dr, r[k], g[k]);
    }
    template <int L>
    __device__ __forceinline__ void reduce() {
#pragma unroll
      for (int e = 0; e < NM; ++e) m[e] = group_sum<L>(m[e]);
#pragma unroll
      for (int k = 0; k < D; ++k) g[k] = group_sum<L>(g[k]);
    }
  };
  float4* grad;
  __device__ static __forceinline__ bool wants(uint32_t) { return true; }
  __device__ __forceinline__ void skip(int, const TgtView&) {}
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return nullptr; }
  __device__ __forceinline__ const float4* tex1() const { return nullptr; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int, const TgtView& tv) {
    b.s = &s;
    b.rho_i = load_pd_plain<D>(tv.a, tv.k).rho;
#pragma unroll
    for (int e = 0; e < NM; ++e) b.m[e] = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) b.g[k] = 0.f;
    return true;
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg&, int i, const TgtView&) {
    float L[6];
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (D == 2) {
      pinv_sym2(b.m[0], b.m[1], b.m[2], L);
      out.x = fmaf(L[0], b.g[0], L[1] * b.g[1]);
      out.y = fmaf(L[1], b.g[0], L[2] * b.g[1]);
    } else {
      pinv_sym3(b.m, L);
      out.x = fmaf(L[0], b.g[0], fmaf(L[1], b.g[1], L[2] * b.g[2]));
      out.y = fmaf(L[1], b.g[0], fmaf(L[3], b.g[1], L[4] * b.g[2]));
      out.z = fmaf(L[2], b.g[0], fmaf(L[4], b.g[1], L[5] * b.g[2]));
    }
    grad[i] = out;
  }
};

// ================================================================== fused sweep
// a_i    = (1/rho_i) sum_j V_j gK (Cv w s - (p_i + p_j)) r + g
// drho_i = rho_i sum_j V_j gK w - 2 Cdel sum_j V_j gK (rho_j - rho_i) r^2 s
// (r = x_i - x_j, grad_i W_ij = gK r, w = (v_i - v_j).r, s = 1/(r^2 + eps h^2),
//  Cv = 2(d+2) nu rho0, Cdel = delta h c0): the paper's terms regrouped per pair.
// RENORM: the renormalised diffusion, rho_j - rho_i -> rho_j - rho_i + (g_i + g_j).r / 2 with
// g = <grad rho>^L of both ends (g_j staged with the neighbour records, g_i in the target cache).
// FUSED: the wall tasks of the same launch write the wall records of the output, so the sweep
// writes fluid targets only (and skips tiles without fluid without touching them).
template <int D, int KERN, bool INTEGRATE, bool RENORM, bool FUSED = false>
struct SweepPass {
  struct Body {
    const DevSeg* s;
    float xi[D], vi[D], rho_i, p_i;
    float acc[D], c1, c2;
    float gi[D];              // RENORM: half the target's renormalised density gradient
    float invH, Kg, Cv, eH2;  // the scene's constants, kept in registers
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4 gj, float, int) {
      const float cinvH = invH, cKg = Kg, cCv = Cv, ceH2 = eH2;
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      const float q = safe_q(r2, cinvH);
      const float gK = cKg * kern_gt<KERN>(q);
      float w = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) w = fmaf(vi[k] - pj.v[k], r[k], w);
      const float sd = __fdividef(1.f, r2 + ceH2);
      const float VgK = pj.V * gK;
      const float tt = VgK * fmaf(cCv * w, sd, -(p_i + pj.p));
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] = fmaf(tt, r[k], acc[k]);
      c1 = fmaf(VgK, w, c1);
      float drho_ji = pj.rho - rho_i;
      if (RENORM) {
        const float gjs[3] = {gj.x, gj.y, gj.z};
#pragma unroll
        for (int k = 0; k < D; ++k) drho_ji = fmaf(fmaf(0.5f, gjs[k], gi[k]), r[k], drho_ji);
      }
      c2 = fmaf(VgK * drho_ji, r2 * sd, c2);
    }
#if SPH_W_PAIR2
    // Two hits at once (a in .x, b in .y) with the paired FP32 operations (one instruction for
    // both hits wherever the scalar form in pair_at has one; the square roots and reciprocals stay
    // scalar); vb = false drops b.  The sums take a, then b, as two pair_at calls would.
    static constexpr bool kPaired = !RENORM;
    __device__ __forceinline__ static float2 sub2(float2 a, float2 b) {  // a - b, rounded once
      return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
    }
    __device__ __forceinline__ void pair_at2(const float* xsa, const PD<D>& pa, const float* xsb, const PD<D>& pb,
                                             bool vb) {
      float2 r[D];
#pragma unroll
      for (int k = 0; k < D; ++k) r[k] = sub2(make_float2(xsa[k], xsb[k]), make_float2(pa.x[k], pb.x[k]));
      float2 r2 = __fmul2_rn(r[0], r[0]);
#pragma unroll
      for (int k = 1; k < D; ++k) r2 = __ffma2_rn(r[k], r[k], r2);
      const float2 q = make_float2(safe_q(r2.x, invH), safe_q(r2.y, invH));
      const float2 om = __ffma2_rn(q, make_float2(-1.f, -1.f), make_float2(1.f, 1.f));
      const float2 om2 = __fmul2_rn(om, om);
      float2 g = __fmul2_rn(om2, om);
      if (KERN == 0) g = __fmul2_rn(__fmul2_rn(__fmul2_rn(om2, om2), om), __ffma2_rn(make_float2(5.f, 5.f), q, make_float2(1.f, 1.f)));
      const float2 gK = __fmul2_rn(make_float2(Kg, Kg), g);
      float2 w = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < D; ++k) w = __ffma2_rn(sub2(make_float2(vi[k], vi[k]), make_float2(pa.v[k], pb.v[k])), r[k], w);
      const float2 r2e = __fadd2_rn(r2, make_float2(eH2, eH2));
      const float2 sd = make_float2(__fdividef(1.f, r2e.x), __fdividef(1.f, r2e.y));
      const float2 VgK = __fmul2_rn(make_float2(pa.V, vb ? pb.V : 0.f), gK);
      const float2 npp = __ffma2_rn(make_float2(pa.p, pb.p), make_float2(-1.f, -1.f), make_float2(-p_i, -p_i));
      const float2 tt = __fmul2_rn(VgK, __ffma2_rn(__fmul2_rn(make_float2(Cv, Cv), w), sd, npp));
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] = fmaf(tt.y, r[k].y, fmaf(tt.x, r[k].x, acc[k]));
      c1 = fmaf(VgK.y, w.y, fmaf(VgK.x, w.x, c1));
      const float2 drho = sub2(make_float2(pa.rho, pb.rho), make_float2(rho_i, rho_i));
      const float2 t2 = __fmul2_rn(VgK, drho), u2 = __fmul2_rn(r2, sd);
      c2 = fmaf(t2.y, u2.y, fmaf(t2.x, u2.x, c2));
    }
#else
    static constexpr bool kPaired = false;
#endif
    template <int L>
    __device__ __forceinline__ void reduce() {
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] = group_sum<L>(acc[k]);
      c1 = group_sum<L>(c1);
      c2 = group_sum<L>(c2);
    }
  };
  Arrays a, out;
  RateOut ro;
  int* status;
  Displace disp;
  const float4* grad;  // RENORM: <grad rho>^L per particle (sorted order)
  float dmax = 0.f;  // largest scaled displacement of this thread's targets
  // with the decision on the device: every CTA has folded its maximum in, so the last one
  // decides whether the next step rebuilds (interval reached or a displacement past skin/2)
  __device__ __forceinline__ void last_cta() {
    if (!INTEGRATE) return;
    if (disp.sticky) {  // a replayed step on a fixed rebuild schedule: record a violation
      if (__uint_as_float(*(volatile unsigned*)disp.maxr) > 1.f) *disp.sticky = 1;
      *disp.maxr = 0u;
      return;
    }
    if (!disp.ctl) return;
    RebuildCtl* c = disp.ctl;
    const int since = c->since + 1;
    const bool r = since >= disp.interval || __uint_as_float(*(volatile unsigned*)&c->maxr) > 1.f;
    c->flag = r ? 1 : 0;
    c->since = r ? 0 : since;
    c->maxr = 0u;
  }
  // the CTA's warps fold their maxima into the scene's running maximum
  __device__ __forceinline__ void flush() {
    if (!INTEGRATE || !disp.maxr) return;
    const unsigned v = __reduce_max_sync(kFull, __float_as_uint(dmax));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(disp.maxr, v);
  }
  // fluid targets only (walls carry m <= 0); a skipped wall keeps its state
  __device__ static __forceinline__ bool wants(uint32_t m) { return (m & kWallBit) == 0; }
  __device__ __forceinline__ void skip(int i, const TgtView& tv) {
    if (!INTEGRATE || FUSED) return;
    store_pd<D>(out, i, load_pd_plain<D>(tv.a, tv.k));
    store_cold<D>(out, i, load_cold<D>(tv.a, tv.k));
    out.meta[i] = tv.a.meta[tv.k];
  }
  __device__ __forceinline__ const float4* tex0() const { return INTEGRATE ? disp.xb : nullptr; }
  __device__ __forceinline__ const float4* tex1() const { return RENORM ? grad : nullptr; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int, const TgtView& tv) {
    b.s = &s;
    if (RENORM) {
      const float4 g = tv.e1[tv.k];
      const float gs[3] = {g.x, g.y, g.z};
#pragma unroll
      for (int k = 0; k < D; ++k) b.gi[k] = 0.5f * gs[k];
    }
    b.invH = s.invH;
    b.Kg = s.Kg;
    b.Cv = s.Cv;
    b.eH2 = s.eH2;
    const PD<D> me = load_pd_plain<D>(tv.a, tv.k);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      b.xi[k] = me.x[k];
      b.vi[k] = me.v[k];
      b.acc[k] = 0.f;
    }
    b.rho_i = me.rho;
    b.p_i = me.p;
    b.c1 = b.c2 = 0.f;
    return me.m > 0.f;  // fluid
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    PD<D> me = load_pd_plain<D>(tv.a, tv.k);
    const uint2 m = tv.a.meta[tv.k];
    const bool fluid = me.m > 0.f;
    float acc_a[D];
    const float inv_rho = 1.f / me.rho;
#pragma unroll
    for (int k = 0; k < D; ++k) acc_a[k] = fmaf(b.acc[k], inv_rho, s.g[k]);
    const float drho = fmaf(me.rho, b.c1, -2.f * s.Cdel * b.c2);
    if (!INTEGRATE) {
      if (fluid) {
        const int o = (int)(m.x & ~kWallBit) + ro.orig_base[m.y];
#pragma unroll
        for (int k = 0; k < D; ++k) ro.a[(size_t)o * D + k] = acc_a[k];
        ro.drho[o] = drho;
        ro.rho[o] = me.rho;
      }
      return;
    }
    Cold c = load_cold<D>(tv.a, tv.k);
    if (fluid) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        me.v[k] = fmaf(s.dt, acc_a[k], me.v[k]);
        ds_add(c.hi[k], c.lo[k], __fmul_rn(s.dt, me.v[k]));
        me.x[k] = __fadd_rn(__fsub_rn(c.hi[k], c.off[k]), c.lo[k]);
      }
      if (s.density_mode == 0) {
        float rh = me.rho;
        ds_add(rh, c.rlo, __fmul_rn(s.dt, drho));
        me.rho = rh;
        const float e = __fadd_rn(__fsub_rn(rh, s.rho0), c.rlo) / s.rho0;
        me.p = s.B * expm1f(s.gamma * log1pf(e));
        me.V = me.m / me.rho;
      }
      if (disp.xb) {  // displacement since the last build, in units of (skin/2 - margin)
        const float4 xb = tv.e0[tv.k];
        float d2 = 0.f;
        if (D == 2) {
          const float e0 = me.x[0] - xb.x, e1 = me.x[1] - xb.y;
          d2 = fmaf(e0, e0, e1 * e1);
        } else {
          const float e0 = me.x[0] - xb.x, e1 = me.x[1] - xb.y, e2 = me.x[D - 1] - xb.z;
          d2 = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
        }
        dmax = fmaxf(dmax, d2 * s.inv_half2);
      }
      bool bad = !(me.rho > 0.5f * s.rho0 && me.rho < 2.f * s.rho0);
#pragma unroll
      for (int k = 0; k < D; ++k) bad |= !isfinite(c.hi[k]) || !isfinite(me.v[k]);
      if (bad) {
        atomicOr(status, 1);
        atomicOr(status + 4 + (int)m.y, 1);  // which scene of the batch
      }
    } else if (FUSED) {
      return;  // a wall: written by its wall task
    }
    store_pd<D>(out, i, me);
    store_cold<D>(out, i, c);
    out.meta[i] = m;
  }
};

// ================================================================== particle shifting
// Explicit shifting at the end of a step (the paper's post-processing step; the delta+-SPH form
// of Sun et al.), on the post-sweep state of every fluid particle:
//   a_i = sum_j V_j [1 + R (W_ij / W(dp_i))^4] grad_i W_ij,  dx_i = -C H^2 a_i,  R = 0.2,
//   dp_i = (m_i / rho0)^(1/d);
// the smallest eigenvalue lambda_i of M_i = sum_j V_j (x_j - x_i) (x) grad_i W_ij selects bulk
// (>= 0.75: dx_i), free-surface band (>= 0.4: the part of dx_i orthogonal to the outward normal
// n_i = -c_i / |c_i|, c_i = sum_j V_j grad_i W_ij) or isolated (no shift).  The pass writes the
// whole state into the other buffer (walls and velocities unchanged) and measures the
// displacement since the last cell build, like the sweep.
constexpr float kShiftR = 0.2f, kLambdaBulk = 0.75f, kLambdaSplash = 0.4f;

template <int D, int KERN>
struct ShiftPass {
  static constexpr int NM = D * (D + 1) / 2;
  struct Body {
    const DevSeg* s;
    float invW0;
    float a[D], c[D], m[NM];
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4, float, int) {
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      const float q = safe_q(r2, s->invH);
      const float Vg = pj.V * (s->Kg * kern_gt<KERN>(q));
      const float wr = s->Kw * kern_w<KERN>(q) * invW0;
      const float w2 = wr * wr;
      const float Vgf = Vg * fmaf(kShiftR, w2 * w2, 1.f);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a[k] = fmaf(Vgf, r[k], a[k]);
        c[k] = fmaf(Vg, r[k], c[k]);
      }
      int e = 0;
#pragma unroll
      for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q2 = p; q2 < D; ++q2, ++e) m[e] = fmaf(-Vg * r[p], r[q2], m[e]);
    }
    template <int L>
    __device__ __forceinline__ void reduce() {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a[k] = group_sum<L>(a[k]);
        c[k] = group_sum<L>(c[k]);
      }
#pragma unroll
      for (int e = 0; e < NM; ++e) m[e] = group_sum<L>(m[e]);
    }
  };
  Arrays a, out;
  Displace disp;
  float dmax = 0.f;
  // the rebuild decision of the next step, now from the shifted positions (the sweep has
  // counted this step already)
  __device__ __forceinline__ void last_cta() {
    if (!disp.ctl) return;
    RebuildCtl* c = disp.ctl;
    const bool r = c->since >= disp.interval || __uint_as_float(*(volatile unsigned*)&c->maxr) > 1.f;
    c->flag = r ? 1 : 0;
    if (r) c->since = 0;
    c->maxr = 0u;
  }
  __device__ __forceinline__ void flush() {
    if (!disp.maxr) return;
    const unsigned v = __reduce_max_sync(kFull, __float_as_uint(dmax));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(disp.maxr, v);
  }
  __device__ static __forceinline__ bool wants(uint32_t m) { return (m & kWallBit) == 0; }
  __device__ __forceinline__ void skip(int i, const TgtView& tv) {
    store_pd<D>(out, i, load_pd_plain<D>(tv.a, tv.k));
    store_cold<D>(out, i, load_cold<D>(tv.a, tv.k));
    out.meta[i] = tv.a.meta[tv.k];
  }
  __device__ __forceinline__ const float4* tex0() const { return disp.xb; }
  __device__ __forceinline__ const float4* tex1() const { return nullptr; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int, const TgtView& tv) {
    b.s = &s;
    const PD<D> me = load_pd_plain<D>(tv.a, tv.k);
    const float vol = fabsf(me.m) / s.rho0;
    const float dp = D == 2 ? sqrtf(vol) : cbrtf(vol);
    b.invW0 = 1.f / (s.Kw * kern_w<KERN>(dp * s.invH));
#pragma unroll
    for (int k = 0; k < D; ++k) b.a[k] = b.c[k] = 0.f;
#pragma unroll
    for (int e = 0; e < NM; ++e) b.m[e] = 0.f;
    return me.m > 0.f;  // fluid
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    PD<D> me = load_pd_plain<D>(tv.a, tv.k);
    Cold c = load_cold<D>(tv.a, tv.k);
    const uint2 m = tv.a.meta[tv.k];
    if (me.m > 0.f && s.shiftC > 0.f) {
      float lam;
      if constexpr (D == 2) {
        const float half = 0.5f * (b.m[0] - b.m[2]);
        lam = 0.5f * (b.m[0] + b.m[2]) - sqrtf(fmaf(half, half, b.m[1] * b.m[1]));
      } else {
        float A[3][3], Q[3][3];
        jacobi_sym3<false>(b.m, A, Q);
        lam = fminf(A[0][0], fminf(A[1][1], A[2][2]));
      }
      float dx[D];
#pragma unroll
      for (int k = 0; k < D; ++k) dx[k] = lam >= kLambdaSplash ? -s.shiftC * b.a[k] : 0.f;
      if (lam >= kLambdaSplash && lam < kLambdaBulk) {
        float c2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) c2 = fmaf(b.c[k], b.c[k], c2);
        if (c2 > 0.f) {
          const float inv = rsqrtf(c2);
          float n[D], sn = 0.f;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            n[k] = -b.c[k] * inv;
            sn = fmaf(dx[k], n[k], sn);
          }
#pragma unroll
          for (int k = 0; k < D; ++k) dx[k] = fmaf(-sn, n[k], dx[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        ds_add(c.hi[k], c.lo[k], dx[k]);
        me.x[k] = __fadd_rn(__fsub_rn(c.hi[k], c.off[k]), c.lo[k]);
      }
    }
    if (me.m > 0.f && disp.xb) {
      const float4 xb = tv.e0[tv.k];
      float d2;
      if (D == 2) {
        const float e0 = me.x[0] - xb.x, e1 = me.x[1] - xb.y;
        d2 = fmaf(e0, e0, e1 * e1);
      } else {
        const float e0 = me.x[0] - xb.x, e1 = me.x[1] - xb.y, e2 = me.x[D - 1] - xb.z;
        d2 = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
      }
      dmax = fmaxf(dmax, d2 * s.inv_half2);
    }
    store_pd<D>(out, i, me);
    store_cold<D>(out, i, c);
    out.meta[i] = m;
  }
};

// ================================================================== pair export
// VAR: per-particle support radii (the records' H_i): a pair needs |x_ij| < max(H_i, H_j), decided
// in FP64 like the scene's cut-off.
template <int D, bool VAR = false>
struct PairPass {
  struct Body {
    uint32_t id_i;
    const uint2* meta;
    int32_t *pi, *pj;
    unsigned long long* count;
    long long cap;
    const DevSeg* s;
    const Arrays* a;
    int i;
    float Hi;
    __device__ __forceinline__ void pair_at(const float*, const PD<D>&, float4, float, int j) {
      if (VAR) {
        const float hj = __ldg(&a->O[j].w);
        const double Hm = (double)fmaxf(Hi, hj > 0.f ? hj : s->H);
        if (!(exact_d2<D>(*s, *a, i, j) < Hm * Hm)) return;
      }
      const unsigned long long k = atomicAdd(count, 1ull);
      if ((long long)k < cap) {
        pi[k] = (int32_t)id_i;
        pj[k] = (int32_t)(meta[j].x & ~kWallBit);
      }
    }
    template <int L>
    __device__ __forceinline__ void reduce() {}
  };
  Arrays a;
  int32_t *pi, *pj;
  unsigned long long* count;
  long long cap;
  __device__ static __forceinline__ bool wants(uint32_t) { return true; }
  __device__ __forceinline__ void skip(int, const TgtView&) {}
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return nullptr; }
  __device__ __forceinline__ const float4* tex1() const { return nullptr; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    b.id_i = tv.a.meta[tv.k].x & ~kWallBit;
    b.meta = a.meta;
    b.s = &s;
    b.a = &a;
    b.i = i;
    const float h = tv.a.O[tv.k].w;
    b.Hi = h > 0.f ? h : s.H;
    b.pi = pi;
    b.pj = pj;
    b.count = count;
    b.cap = cap;
    return true;
  }
  __device__ __forceinline__ void finish(Body&, const DevSeg&, int, const TgtView&) {}
};

// ================================================================== adjoint sweep (Sec. 2.2)
// Threads per target of the adjoint sweep: SPH_ADJ_LANES_X times the tile shape's (the same tiles
// as the forward passes; more lanes split a target's candidates further, for the small scenes of
// adjoint workloads where the launch has few targets per SM), and the CTAs per SM its registers
// are budgeted for.
#ifndef SPH_ADJ_LANES_X
#define SPH_ADJ_LANES_X 1
#endif
template <int D>
constexpr int adj_lanes() {
  constexpr int l = TileCfg<D>::LANES * SPH_ADJ_LANES_X;
  return (l > 32 || TileCfg<D>::TP * l > 1024) ? TileCfg<D>::LANES : l;
}
template <int D>
constexpr int adj_threads() { return TileCfg<D>::TP * adj_lanes<D>(); }
#ifndef SPH_ADJ_MINB
#define SPH_ADJ_MINB 0
#endif
template <int D>
constexpr int adj_minb() { return SPH_ADJ_MINB > 0 ? SPH_ADJ_MINB : (512 / adj_threads<D>() > 0 ? 512 / adj_threads<D>() : 1); }
// For pair (i, j) the step's pair terms add alpha_ab r_ab to a_a and beta_ab to drho_a
// (a = self, b = other).  With seeds abar = dt vtilde, bbar = dt rhobar' of the self particle,
// Phi_ab = alpha_ab (abar_a . r_ab) + bbar_a beta_ab; the gather at i adds the derivatives of
// its own Phi_ij and of the neighbours' Phi_ji with respect to x_i, v_i, rho_i (atomic-free).
template <int D, int KERN>
struct AdjPass {
  struct Body {
    const DevSeg* s;
    float xi[D], vi[D], rho_i, p_i, V_i, P_i;
    float ab_i[D], bb_i;
    float gx[D], gv[D], grho, gnu;
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4 Sj, float ppj, int) {
      const DevSeg& c = *s;
      float ab_j[3], bb_j, P_j;
      if (D == 2) {
        ab_j[0] = Sj.x; ab_j[1] = Sj.y; ab_j[2] = 0.f; bb_j = Sj.z; P_j = Sj.w;
      } else {
        ab_j[0] = Sj.x; ab_j[1] = Sj.y; ab_j[2] = Sj.z; bb_j = Sj.w; P_j = ppj;
      }
      (void)P_j;
      float r[D], u[D];
      const float r2 = diff<D>(xs, pj.x, r);
      const float q = safe_q(r2, c.invH);
      const float gK = c.Kg * kern_gt<KERN>(q);
      const float hK = c.Kh * kern_ht<KERN>(q);
      const float sd = __fdividef(1.f, r2 + c.eH2);
      float w = 0.f, e_i = 0.f, e_j = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        u[k] = vi[k] - pj.v[k];
        w = fmaf(u[k], r[k], w);
        e_i = fmaf(ab_i[k], r[k], e_i);
        e_j = fmaf(ab_j[k], r[k], e_j);
      }
      e_j = -e_j;
      const float ws = w * sd;
      const float X = fmaf(c.Cv, ws, -(p_i + pj.p));
      const float r2s = r2 * sd;
      const float S1 = hK * r2s + 2.f * gK * sd * (c.eH2 * sd);
      const float CvsgK = c.Cv * sd * gK;
      const float XhR = fmaf(X, hK, -2.f * gK * c.Cv * w * sd * sd);
      float cR, cU, alpha;
      {  // own term: a = i, b = j
        const float Vb_ra = pj.V / rho_i;
        alpha = Vb_ra * gK * X;
        const float cRb = rho_i * pj.V * hK * w - 2.f * c.Cdel * pj.V * (pj.rho - rho_i) * S1;
        const float cUb = rho_i * pj.V * gK;
        cR = e_i * (Vb_ra * XhR) + bb_i * cRb;
        cU = e_i * (Vb_ra * CvsgK) + bb_i * cUb;
        grho += e_i * (-pj.V * gK * P_i / rho_i - alpha / rho_i) +
                bb_i * (pj.V * gK * w + 2.f * c.Cdel * pj.V * gK * r2s);
        gnu += e_i * Vb_ra * gK * c.dCv_dnu * ws;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        gx[k] += alpha * ab_i[k] + cR * r[k] + cU * u[k];
        gv[k] += cU * r[k];
      }
      {  // transposed term: a = j, b = i
        const float Va_rb = V_i / pj.rho;
        alpha = Va_rb * gK * X;
        const float beta = pj.rho * V_i * gK * w - 2.f * c.Cdel * V_i * (rho_i - pj.rho) * gK * r2s;
        const float cRb = pj.rho * V_i * hK * w - 2.f * c.Cdel * V_i * (rho_i - pj.rho) * S1;
        const float cUb = pj.rho * V_i * gK;
        cR = e_j * (Va_rb * XhR) + bb_j * cRb;
        cU = e_j * (Va_rb * CvsgK) + bb_j * cUb;
        grho += e_j * (-alpha / rho_i - V_i * gK * P_i / pj.rho) + bb_j * (-beta / rho_i - 2.f * c.Cdel * V_i * gK * r2s);
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        gx[k] += -alpha * ab_j[k] + cR * r[k] + cU * u[k];
        gv[k] += cU * r[k];
      }
    }
    template <int L>
    __device__ __forceinline__ void reduce() {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        gx[k] = group_sum<L>(gx[k]);
        gv[k] = group_sum<L>(gv[k]);
      }
      grho = group_sum<L>(grho);
      gnu = group_sum<L>(gnu);
    }
  };
  Arrays a;
  const float4 *S, *XBin, *VBin;
  const float* Pp;
  float4 *XBout, *VBout;
  double* nu_acc;  // per storage slot: the viscosity adjoint of every step so far (summed at the end)
  __device__ static __forceinline__ bool wants(uint32_t) { return true; }
  __device__ __forceinline__ void skip(int, const TgtView&) {}
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return XBin; }
  __device__ __forceinline__ const float4* tex1() const { return VBin; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    b.s = &s;
    const PD<D> me = load_pd_plain<D>(tv.a, tv.k);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      b.xi[k] = me.x[k];
      b.vi[k] = me.v[k];
      b.gx[k] = b.gv[k] = 0.f;
    }
    b.rho_i = me.rho;
    b.p_i = me.p;
    b.V_i = me.V;
    const float4 Si = S[i];
    if (D == 2) {
      b.ab_i[0] = Si.x; b.ab_i[1] = Si.y; b.bb_i = Si.z; b.P_i = Si.w;
    } else {
      b.ab_i[0] = Si.x; b.ab_i[1] = Si.y; b.ab_i[2] = Si.z; b.bb_i = Si.w; b.P_i = Pp[i];
    }
    b.grho = b.gnu = 0.f;
    return me.m > 0.f;
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    const float4 xb = tv.e0[tv.k], vb = tv.e1[tv.k];
    const float xbs[3] = {xb.x, xb.y, xb.z}, vbs[3] = {vb.x, vb.y, vb.z};
    float ox[3] = {0.f, 0.f, 0.f}, ov[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float vt = fmaf(s.dt, xbs[k], vbs[k]);
      ox[k] = xbs[k] + b.gx[k];
      ov[k] = vt + b.gv[k];
    }
    XBout[i] = make_float4(ox[0], ox[1], ox[2], xb.w + b.grho);
    VBout[i] = make_float4(ov[0], ov[1], ov[2], 0.f);
    nu_acc[i] += (double)b.gnu;  // the slot's own running sum: no atomics, a fixed order
  }
};

// Summation mode: the step's density rho^_i = sum_j m_j W_ij (self term included) feeds the rates
// and is the stored density after the step (it is not integrated), so its adjoint, which the
// adjoint sweep leaves in XB.w (the seed's rhobar' plus the rates' density terms), passes on to
// the positions,
//   x_bar_i += sum_j grad_i W_ij (rhobar_i m_j + rhobar_j m_i),
// and the density before the step, which the step overwrites, gets a zero adjoint.  A second
// gathered pass after the adjoint sweep (it needs the neighbours' complete rhobar_j).
template <int D, int KERN>
struct AdjDensityPass {
  struct Body {
    const DevSeg* s;
    float xi[D], rb_i, m_i;
    float gx[D];
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4 XBj, float, int) {
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      const float gK = s->Kg * kern_gt<KERN>(safe_q(r2, s->invH));
      const float c = gK * fmaf(rb_i, fabsf(pj.m), XBj.w * m_i);
#pragma unroll
      for (int k = 0; k < D; ++k) gx[k] = fmaf(c, r[k], gx[k]);
    }
    template <int L>
    __device__ __forceinline__ void reduce() {
#pragma unroll
      for (int k = 0; k < D; ++k) gx[k] = group_sum<L>(gx[k]);
    }
  };
  const float4 *XBin, *VBin;
  float4 *XBout, *VBout;
  __device__ static __forceinline__ bool wants(uint32_t) { return true; }
  __device__ __forceinline__ void skip(int, const TgtView&) {}
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return XBin; }
  __device__ __forceinline__ const float4* tex1() const { return VBin; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int, const TgtView& tv) {
    b.s = &s;
    const float4 A = tv.a.A[tv.k];
    b.xi[0] = A.x; b.xi[1] = A.y;
    if (D == 3) b.xi[2] = A.z;
    b.rb_i = tv.e0[tv.k].w;
    b.m_i = fabsf(D == 3 ? tv.a.C[tv.k].y : tv.a.B[tv.k].w);
#pragma unroll
    for (int k = 0; k < D; ++k) b.gx[k] = 0.f;
    return true;
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg&, int i, const TgtView& tv) {
    const float4 xb = tv.e0[tv.k];
    const float gz = D == 3 ? b.gx[D - 1] : 0.f;
    XBout[i] = make_float4(xb.x + b.gx[0], xb.y + b.gx[1], D == 3 ? xb.z + gz : xb.z, 0.f);
    VBout[i] = tv.e1[tv.k];
  }
};

// ================================================================== shifting by optimisation
// The paper's differentiable particle shifting / density-target sampling: the objective
//   L = (1/n) sum_i [ w_c (1 - c_i)^2 + w_g |g_i|^2 + w_r (rho_i - t(x_i))^2 + w_p sum_{|x_ij| < a dp_i} (a dp_i - |x_ij|)^2 ]
// over the fluid (walls are fixed neighbours), rho_i = sum_j m_j W_ij (self included, every
// particle), c_i = sum_j V_j W_ij (self included), g_i = sum_j V_j grad_i W_ij, V_j = m_j / rho_j,
// and its gradient with respect to the fluid positions, hand-derived and gathered per particle
// in four passes (atomic-free):
//   P1  rho_i, V_i                                             (every particle)
//   P2  c_i, g_i, the penalty; loss l_i; seeds cb_i = -2 w_c (1 - c_i)/n, gb_i = 2 w_g g_i / n
//   P3  Vb_i = cb_i W(0) + sum_j [cb_j W_ij - gK (gb_j . r_ij)],  rhob_i = 2 w_r e_i / n - Vb_i V_i / rho_i
//       (every particle), and for the fluid xb_i = sum_j [(cb_i V_j + cb_j V_i) gK r_ij
//       + Hess W_ij (V_j gb_i - V_i gb_j) + penalty terms] - 2 w_r e_i grad t(x_i) / n
//   P4  xb_i += sum_j (rhob_i m_j + rhob_j m_i) gK r_ij; the gradient out, or a descent step
// (r_ij = x_i - x_j, grad_i W_ij = gK r_ij, Hess W_ij = gK I + hK r r^T, e_i = rho_i - t(x_i)).
template <int D>
__device__ __forceinline__ float target_density(const ShiftObjective& o, const float* x, float* grad) {
  if (o.target_kind == 0) {
    float a = o.t_phase;
#pragma unroll
    for (int k = 0; k < D; ++k) a = fmaf(o.t_k[k], x[k], a);
    float sn, cs;
    sincosf(a, &sn, &cs);
#pragma unroll
    for (int k = 0; k < D; ++k) grad[k] = o.t_amp * cs * o.t_k[k];
    return fmaf(o.t_amp, sn, o.t_base);
  }
  float sg = -o.t_c;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    sg = fmaf(o.t_n[k], x[k], sg);
    grad[k] = 0.f;
  }
  return sg < 0.f ? o.t_lo : o.t_hi;
}

template <int D, int KERN>
struct OptDensityPass {
  struct Body {
    const DevSeg* s;
    float rho;
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4, float, int) {
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      rho = fmaf(fabsf(pj.m), s->Kw * kern_w<KERN>(safe_q(r2, s->invH)), rho);
    }
    template <int L>
    __device__ __forceinline__ void reduce() { rho = group_sum<L>(rho); }
  };
  float4* S1;  // (V, rho, 0, 0)
  __device__ static __forceinline__ bool wants(uint32_t) { return true; }
  __device__ __forceinline__ void skip(int, const TgtView&) {}
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return nullptr; }
  __device__ __forceinline__ const float4* tex1() const { return nullptr; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int, const TgtView&) {
    b.s = &s;
    b.rho = 0.f;
    return true;
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    const float m = fabsf(load_pd_plain<D>(tv.a, tv.k).m);
    const float rho = fmaf(m, s.Kw, b.rho);  // self term, w(0) = 1
    S1[i] = make_float4(m / rho, rho, 0.f, 0.f);
  }
};

template <int D, int KERN>
struct OptColorPass {
  struct Body {
    const DevSeg* s;
    float delta, c, reg, g[D];
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4 e, float, int) {
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      const float q = safe_q(r2, s->invH);
      const float Vj = e.x;
      c = fmaf(Vj, s->Kw * kern_w<KERN>(q), c);
      const float VgK = Vj * (s->Kg * kern_gt<KERN>(q));
#pragma unroll
      for (int k = 0; k < D; ++k) g[k] = fmaf(VgK, r[k], g[k]);
      const float rl = sqrtf(r2);
      if (rl < delta) reg = fmaf(delta - rl, delta - rl, reg);
    }
    template <int L>
    __device__ __forceinline__ void reduce() {
      c = group_sum<L>(c);
      reg = group_sum<L>(reg);
#pragma unroll
      for (int k = 0; k < D; ++k) g[k] = group_sum<L>(g[k]);
    }
  };
  const float4* S1;
  float4* S2;  // (cb, gb)
  float* Lp;   // loss contribution of each particle (0 for walls)
  ShiftObjective o;
  __device__ static __forceinline__ bool wants(uint32_t m) { return (m & kWallBit) == 0; }
  __device__ __forceinline__ void skip(int i, const TgtView&) {
    S2[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    Lp[i] = 0.f;
  }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return S1; }
  __device__ __forceinline__ const float4* tex1() const { return nullptr; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int, const TgtView& tv) {
    b.s = &s;
    const float m = load_pd_plain<D>(tv.a, tv.k).m;
    const float vol = fabsf(m) / s.rho0;
    b.delta = o.reg_fraction * (D == 2 ? sqrtf(vol) : cbrtf(vol));
    b.c = b.reg = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) b.g[k] = 0.f;
    return m > 0.f;
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    const PD<D> me = load_pd_plain<D>(tv.a, tv.k);
    if (!(me.m > 0.f)) {
      skip(i, tv);
      return;
    }
    const float4 s1 = tv.e0[tv.k];
    const float inv_n = 1.f / (float)s.nf;
    const float c = fmaf(s1.x, s.Kw, b.c);  // self term
    float gt[3];
    const float e = s1.y - target_density<D>(o, me.x, gt);
    float g2 = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) g2 = fmaf(b.g[k], b.g[k], g2);
    const float l = o.w_color * (1.f - c) * (1.f - c) + o.w_grad * g2 + o.w_density * e * e + o.w_reg * b.reg;
    Lp[i] = l * inv_n;
    const float gb = 2.f * o.w_grad * inv_n;
    S2[i] = make_float4(-2.f * o.w_color * (1.f - c) * inv_n, gb * b.g[0], gb * b.g[1], D == 3 ? gb * b.g[D - 1] : 0.f);
  }
};

template <int D, int KERN>
struct OptAdjPass {
  struct Body {
    const DevSeg* s;
    float cb, gb[D], V, delta, wr;  // the target's seeds, volume, penalty reach, 2 w_p / n
    bool fluid;
    float Vb, xb[D];
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4 e, float Vj, int) {
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      const float q = safe_q(r2, s->invH);
      const float W = s->Kw * kern_w<KERN>(q);
      const float gK = s->Kg * kern_gt<KERN>(q);
      const float gbj[3] = {e.y, e.z, e.w};
      float gr = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) gr = fmaf(gbj[k], r[k], gr);
      Vb = fmaf(e.x, W, fmaf(-gK, gr, Vb));
      if (!fluid) return;
      const float hK = s->Kh * kern_ht<KERN>(q);
      const float coef = fmaf(cb, Vj, e.x * V) * gK;
      float v[D], rv = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        v[k] = fmaf(Vj, gb[k], -V * gbj[k]);
        rv = fmaf(r[k], v[k], rv);
      }
      float pen = 0.f;  // pair penalty: d/dx_i of (a dp - |r|)^2 from both ends' terms
      const float rl = sqrtf(r2);
      if (rl < delta) pen += delta - rl;
      if (pj.m > 0.f) {
        const float volj = pj.m / s->rho0;
        const float dj = delta_frac * (D == 2 ? sqrtf(volj) : cbrtf(volj));
        if (rl < dj) pen += dj - rl;
      }
      const float pc = rl > 0.f ? -wr * pen / rl : 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) xb[k] += fmaf(coef + hK * rv + pc, r[k], gK * v[k]);
    }
    float delta_frac;
    template <int L>
    __device__ __forceinline__ void reduce() {
      Vb = group_sum<L>(Vb);
#pragma unroll
      for (int k = 0; k < D; ++k) xb[k] = group_sum<L>(xb[k]);
    }
  };
  const float4* S1;
  const float4* S2;
  float4* XB;  // (xb partial, rhob)
  ShiftObjective o;
  __device__ static __forceinline__ bool wants(uint32_t) { return true; }
  __device__ __forceinline__ void skip(int, const TgtView&) {}
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return S2; }
  __device__ __forceinline__ const float4* tex1() const { return S1; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int, const TgtView& tv) {
    b.s = &s;
    const float m = load_pd_plain<D>(tv.a, tv.k).m;
    const float4 s2 = tv.e0[tv.k], s1 = tv.e1[tv.k];
    const float inv_n = 1.f / (float)s.nf;
    b.cb = s2.x;
    b.gb[0] = s2.y;
    b.gb[1] = s2.z;
    if (D == 3) b.gb[D - 1] = s2.w;
    b.V = s1.x;
    b.fluid = m > 0.f;
    const float vol = fabsf(m) / s.rho0;
    b.delta_frac = o.reg_fraction;
    b.delta = b.fluid ? o.reg_fraction * (D == 2 ? sqrtf(vol) : cbrtf(vol)) : 0.f;
    b.wr = 2.f * o.w_reg * inv_n;
    b.Vb = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) b.xb[k] = 0.f;
    return true;
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    const PD<D> me = load_pd_plain<D>(tv.a, tv.k);
    const float4 s1 = tv.e1[tv.k];
    const float inv_n = 1.f / (float)s.nf;
    const float Vb = fmaf(b.cb, s.Kw, b.Vb);  // self term of the colour field
    float rhob = -Vb * s1.x / s1.y;
    float xb[3] = {0.f, 0.f, 0.f};
    if (b.fluid) {
      float gt[3];
      const float e = s1.y - target_density<D>(o, me.x, gt);
      const float se = 2.f * o.w_density * e * inv_n;
      rhob += se;
#pragma unroll
      for (int k = 0; k < D; ++k) xb[k] = fmaf(-se, gt[k], b.xb[k]);
    }
    XB[i] = make_float4(xb[0], xb[1], xb[2], rhob);
  }
};

template <int D, int KERN, bool UPDATE>
struct OptAdj2Pass {
  struct Body {
    const DevSeg* s;
    float rb, m;
    float xb[D];
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4 e, float, int) {
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      const float gK = s->Kg * kern_gt<KERN>(safe_q(r2, s->invH));
      const float coef = fmaf(rb, fabsf(pj.m), e.w * m) * gK;
#pragma unroll
      for (int k = 0; k < D; ++k) xb[k] = fmaf(coef, r[k], xb[k]);
    }
    template <int L>
    __device__ __forceinline__ void reduce() {
#pragma unroll
      for (int k = 0; k < D; ++k) xb[k] = group_sum<L>(xb[k]);
    }
  };
  const float4* XB;
  float4* G;     // the gradient dL/dx (0 for walls)
  Arrays out;    // UPDATE: the state after the descent step x <- x - step dL/dx
  float step;
  __device__ static __forceinline__ bool wants(uint32_t m) { return (m & kWallBit) == 0; }
  __device__ __forceinline__ void skip(int i, const TgtView& tv) {
    G[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (UPDATE) {
      store_pd<D>(out, i, load_pd_plain<D>(tv.a, tv.k));
      store_cold<D>(out, i, load_cold<D>(tv.a, tv.k));
      out.meta[i] = tv.a.meta[tv.k];
    }
  }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return XB; }
  __device__ __forceinline__ const float4* tex1() const { return nullptr; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int, const TgtView& tv) {
    b.s = &s;
    b.rb = tv.e0[tv.k].w;
    b.m = load_pd_plain<D>(tv.a, tv.k).m;
#pragma unroll
    for (int k = 0; k < D; ++k) b.xb[k] = 0.f;
    return b.m > 0.f;
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    PD<D> me = load_pd_plain<D>(tv.a, tv.k);
    if (!(me.m > 0.f)) {
      skip(i, tv);
      return;
    }
    const float4 p = tv.e0[tv.k];
    const float ps[3] = {p.x, p.y, p.z};
    float gx[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < D; ++k) gx[k] = ps[k] + b.xb[k];
    G[i] = make_float4(gx[0], gx[1], gx[2], 0.f);
    if (UPDATE) {
      Cold c = load_cold<D>(tv.a, tv.k);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        ds_add(c.hi[k], c.lo[k], -step * gx[k]);
        me.x[k] = __fadd_rn(__fsub_rn(c.hi[k], c.off[k]), c.lo[k]);
      }
      store_pd<D>(out, i, me);
      store_cold<D>(out, i, c);
      out.meta[i] = tv.a.meta[tv.k];
    }
  }
};

template <int D, int KERN>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, TileCfg<D>::MINB) k_opt_density(TravArgs t, const Tile* tiles, const int* ntiles, float4* S1) {
  OptDensityPass<D, KERN> pass;
  pass.S1 = S1;
  run_tiles<D, 0, 0>(t, tiles, ntiles, nullptr, nullptr, pass);
}
template <int D, int KERN>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, TileCfg<D>::MINB) k_opt_color(TravArgs t, const Tile* tiles, const int* ntiles, const float4* S1, float4* S2,
                                                 float* Lp, ShiftObjective o) {
  OptColorPass<D, KERN> pass;
  pass.S1 = S1;
  pass.S2 = S2;
  pass.Lp = Lp;
  pass.o = o;
  run_tiles<D, 1, 0>(t, tiles, ntiles, S1, nullptr, pass);
}
template <int D, int KERN>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, 512 / TileCfg<D>::THREADS) k_opt_adj(TravArgs t, const Tile* tiles, const int* ntiles, const float4* S1, const float4* S2,
                                               const float* Vs, float4* XB, ShiftObjective o) {
  OptAdjPass<D, KERN> pass;
  pass.S1 = S1;
  pass.S2 = S2;
  pass.XB = XB;
  pass.o = o;
  run_tiles<D, 2, 0>(t, tiles, ntiles, S2, Vs, pass);
}
template <int D, int KERN, bool UPDATE>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, TileCfg<D>::MINB) k_opt_adj2(TravArgs t, const Tile* tiles, const int* ntiles, const float4* XB, float4* G,
                                                Arrays out, float step) {
  OptAdj2Pass<D, KERN, UPDATE> pass;
  pass.XB = XB;
  pass.G = G;
  pass.out = out;
  pass.step = step;
  run_tiles<D, 1, 0>(t, tiles, ntiles, XB, nullptr, pass);
}
// the volumes of P1 as a plain float array (the second staged payload of P3)
__global__ void k_opt_volumes(int N, const float4* __restrict__ S1, float* __restrict__ V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) V[i] = S1[i].x;
}

// ================================================================== variable support radius
// Per-particle support radii H_i <= H (the scene's H sizes the cells; H_i = 0 stands for H).  For
// every particle (the paper's symmetric search radius and super-symmetric neighbourhood):
//   s_i    = max(H_i, max{H_k : |x_ik| < H_k})                                the search radius
//   rhoS_i = sum_j m_j (W(|x_ij|, H_i) + W(|x_ij|, H_j)) / 2 over |x_ij| < max(H_i, H_j)
//   rhoG_i = sum_j m_j W(|x_ij|, H_i) over |x_ij| < H_i                       (gather)
// self terms included, W(r, h) = C_d / h^d w(r / h).  The comparisons |x_ij|^2 < H_k^2 are taken
// in FP64 from the double-single positions when the FP32 distance lies within a guard band of
// H_k^2, so s_i (a maximum of given radii) is exact; the sum gathers what the paper computes with
// an atomic maximum in scatter form.
template <int D, int KERN>
struct VarSupportPass {
  struct Body {
    const DevSeg* s;
    const Arrays* a;
    int i;
    float Hi, band, smax, rs, rg;  // band: FP32 error bound of a squared distance (absolute)
    __device__ __forceinline__ bool inside(float r2, float h, int j) const {
      const float h2 = h * h;
      if (fabsf(r2 - h2) > band) return r2 < h2;
      return exact_d2<D>(*s, *a, i, j) < (double)h * (double)h;
    }
    __device__ __forceinline__ float Wh(float r2, float h) const {
      const float sc = s->H / h;
      float f = sc * sc;
      if (D == 3) f *= sc;
      const float q = sqrtf(r2) / h;
      return q < 1.f ? s->Kw * f * kern_w<KERN>(q) : 0.f;
    }
    __device__ __forceinline__ void pair_at(const float* xs, const PD<D>& pj, float4 e, float, int j) {
      float r[D];
      const float r2 = diff<D>(xs, pj.x, r);
      const float Hj = e.x;
      const bool inj = inside(r2, Hj, j), ini = inside(r2, Hi, j);
      if (inj) smax = fmaxf(smax, Hj);
      if (!(ini || inj)) return;
      const float wi = ini ? Wh(r2, Hi) : 0.f, wj = inj ? Wh(r2, Hj) : 0.f;
      const float m = fabsf(pj.m);
      rs = fmaf(m, 0.5f * (wi + wj), rs);
      rg = fmaf(m, wi, rg);
    }
    template <int L>
    __device__ __forceinline__ void reduce() {
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(kFull, smax, o));
      rs = group_sum<L>(rs);
      rg = group_sum<L>(rg);
    }
  };
  Arrays a;
  float4* out;  // (s, rhoS, rhoG, 0)
  float band;
  __device__ static __forceinline__ bool wants(uint32_t) { return true; }
  __device__ __forceinline__ void skip(int, const TgtView&) {}
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void last_cta() {}
  __device__ __forceinline__ const float4* tex0() const { return nullptr; }
  __device__ __forceinline__ const float4* tex1() const { return nullptr; }
  __device__ __forceinline__ bool init(Body& b, const DevSeg& s, int i, const TgtView& tv) {
    b.s = &s;
    b.a = &a;
    b.i = i;
    const float h = tv.a.O[tv.k].w;
    b.Hi = h > 0.f ? h : s.H;
    b.band = band;
    b.smax = b.Hi;
    b.rs = b.rg = 0.f;
    return true;
  }
  __device__ __forceinline__ void finish(Body& b, const DevSeg&, int i, const TgtView& tv) {
    const float m = fabsf(load_pd_plain<D>(tv.a, tv.k).m);
    const float w0 = b.Wh(0.f, b.Hi);
    out[i] = make_float4(b.smax, fmaf(m, w0, b.rs), fmaf(m, w0, b.rg), 0.f);
  }
};

template <int D, int KERN>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, TileCfg<D>::MINB) k_varsupport(TravArgs t, const Tile* tiles, const int* ntiles, const float4* Hs,
                                                    float4* out, float band) {
  VarSupportPass<D, KERN> pass;
  pass.a = t.a;
  pass.out = out;
  pass.band = band;
  run_tiles<D, 1, 2>(t, tiles, ntiles, Hs, nullptr, pass);
}
// the support radius of every particle as a staged payload (H_i, 0, 0, 0)
__global__ void k_support_payload(int N, const float4* __restrict__ O, const DevSeg* __restrict__ segs,
                                  const uint2* __restrict__ meta, float4* __restrict__ Hs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const float h = O[k].w;
  Hs[k] = make_float4(h > 0.f ? h : segs[meta[k].y].H, 0.f, 0.f, 0.f);
}
// per-particle support radii by original row into the records
__global__ void k_set_support(int N, const uint2* __restrict__ meta, const int* __restrict__ orig_base,
                              const float* __restrict__ H, float4* __restrict__ O) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const uint2 m = meta[k];
  O[k].w = H[orig_base[m.y] + (int)(m.x & ~kWallBit)];
}
// a float4 array (x, y, z) in sorted order into three arrays by original row
__global__ void k_unpermute3(int N, const uint2* __restrict__ meta, const int* __restrict__ orig_base,
                             const float4* __restrict__ src, float* __restrict__ a, float* __restrict__ b,
                             float* __restrict__ c) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const uint2 m = meta[k];
  const int o = orig_base[m.y] + (int)(m.x & ~kWallBit);
  const float4 v = src[k];
  if (a) a[o] = v.x;
  if (b) b[o] = v.y;
  if (c) c[o] = v.z;
}

// ================================================================== kernels
// The wall pass visits only the tiles that hold a wall particle (listed at each rebuild).
template <int D, int KERN>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, TileCfg<D>::MINB) k_walls_t(TravArgs t, const Tile* tiles, const int* wall_tiles,
                                                 const int* n_wall_tiles) {
  WallPass<D, KERN> pass;
  pass.a = t.a;
  run_tiles<D, 0, 0>(t, tiles, n_wall_tiles, nullptr, nullptr, pass, wall_tiles);
}

// List of the tiles holding at least one wall particle: one warp per tile.
template <int D>
__global__ void k_wall_tiles(const Tile* __restrict__ tiles, const int* __restrict__ ntiles,
                             const uint2* __restrict__ meta, int* __restrict__ list, uint4* __restrict__ wall_p,
                             uint4* __restrict__ fluid_p, int* __restrict__ count) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= *ntiles) return;  // warp-uniform
  list_tile<D>(tiles[w], w, lane, meta, list, wall_p, fluid_p, count);
}
template <int D, int KERN>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, TileCfg<D>::MINB) k_density_t(TravArgs t, const Tile* tiles, const int* ntiles) {
  wait_prior_grid();
  DensityPass<D, KERN> pass;
  pass.a = t.a;
  run_tiles<D, 0, 1>(t, tiles, ntiles, nullptr, nullptr, pass);
}
// Wall pass and sweep in one launch: the tiles holding walls are the first tasks of the shared
// task counter (so every wall task is held by a running CTA before any sweep task waits on it),
// the tiles holding fluid follow (both lists hold copies of the tiles); a sweep tile whose staged
// region holds no wall particle runs at once, the others wait for the wall tasks to finish
// (tile_task's gate).  Same results as the two launches.
template <int D, int KERN>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, TileCfg<D>::MINB) k_walls_sweep_t(TravArgs t, uint4* wall_p,
                                                 uint4* fluid_p, const int* n_lists, Arrays out, Displace disp) {
  wait_prior_grid();
  extern __shared__ __align__(16) unsigned char smraw[];
  TileSmem<D, 0>& sm = *reinterpret_cast<TileSmem<D, 0>*>(smraw);
  __shared__ int s_task;
  WallPass<D, KERN> wp;
  wp.a = t.a;
  wp.out = out;
  SweepPass<D, KERN, true, false, true> sp;
  sp.a = t.a;
  sp.out = out;
  sp.ro = RateOut{};
  sp.status = t.status;
  sp.disp = disp;
  sp.grad = nullptr;
  const int nw = n_lists[0], nt = n_lists[1];
  unsigned* gate = reinterpret_cast<unsigned*>(t.tile_ctr + 2);
  __shared__ int s_gate;
  long long pairs_cta = 0;
  while (true) {
    if (threadIdx.x == 0) {
      s_task = atomicAdd(t.tile_ctr, 1);
      s_gate = ld_acquire(gate) >= (unsigned)nw;  // before every load of the task (two barriers on)
    }
    __syncthreads();
    const int task = s_task;
    if (task >= nw + nt) break;
    uint4* plan = task < nw ? wall_p + (size_t)task * TilePlan<D>::U4 : fluid_p + (size_t)(task - nw) * TilePlan<D>::U4;
    load_plan(sm, plan);
    __syncthreads();
    const Tile T = sm.ptile;
    if (task < nw) {
      tile_task<D, 0, 0, false>(t, T, sm, nullptr, nullptr, wp, nullptr, 0, plan);
      __syncthreads();  // every wall record of the tile is written
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(gate, 1u);
      }
    } else {
      pairs_cta += tile_task<D, 0, 0, true>(t, T, sm, nullptr, nullptr, sp, gate, (unsigned)nw, plan, s_gate);
      __syncthreads();
    }
  }
  end_tiles(t, sp, pairs_cta);
}
template <int D, int KERN>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, TileCfg<D>::MINB) k_grad_t(TravArgs t, const Tile* tiles, const int* ntiles, float4* grad) {
  wait_prior_grid();
  GradPass<D, KERN> pass;
  pass.grad = grad;
  run_tiles<D, 0, 0>(t, tiles, ntiles, nullptr, nullptr, pass);
}
// (3D with the renormalised diffusion: three CTAs per SM, so that its registers do not spill)
template <int D, int KERN, bool INTEGRATE, bool RENORM>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, (D == 3 && RENORM ? 768 : 1024) / TileCfg<D>::THREADS) k_sweep_t(TravArgs t, const Tile* tiles, const int* ntiles, Arrays out,
                                                 RateOut ro, Displace disp, const float4* grad) {
  wait_prior_grid();
  SweepPass<D, KERN, INTEGRATE, RENORM> pass;
  pass.a = t.a;
  pass.out = out;
  pass.ro = ro;
  pass.status = t.status;
  pass.disp = disp;
  pass.grad = grad;
  run_tiles<D, RENORM ? 1 : 0, 0>(t, tiles, ntiles, RENORM ? grad : nullptr, nullptr, pass);
}
// The positions of the sweep's input as pairs (x_2p, x_2p+1, y_2p, y_2p+1) and (z_2p, z_2p+1) for
// the warp-per-tile sweep's paired tests; a missing last partner and the padding pairs lie far
// away.  One thread per pair of the padded arrays (warp_pairs_stride(N) pairs each).
__global__ void k_pack_pairs3(int N, int stride, const float4* __restrict__ A, float4* __restrict__ PXY,
                              float2* __restrict__ PZ) {
  wait_prior_grid();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // the sweep may launch
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= stride) return;
  const float4 far = make_float4(1e30f, 1e30f, 1e30f, 0.f);
  const float4 a = 2 * p < N ? __ldg(A + 2 * p) : far;
  const float4 b = 2 * p + 1 < N ? __ldg(A + 2 * p + 1) : far;
  PXY[p] = make_float4(a.x, b.x, a.y, b.y);
  PZ[p] = make_float2(a.z, b.z);
}

// The same sweep on the warp-per-tile traversal (one thread per target).
template <int D, int KERN, bool INTEGRATE, bool RENORM>
__global__ void __launch_bounds__(WCfg::THREADS, SPH_W_MINB) k_sweep_w(TravArgs t, const Tile* tiles,
                                                                            const int* ntiles, Arrays out,
                                                                            RateOut ro, Displace disp,
                                                                            const float4* grad) {
  wait_prior_grid();
  SweepPass<D, KERN, INTEGRATE, RENORM> pass;
  pass.a = t.a;
  pass.out = out;
  pass.ro = ro;
  pass.status = t.status;
  pass.disp = disp;
  pass.grad = grad;
  run_warp_tiles<D, true, RENORM, false>(t, tiles, ntiles, RENORM ? grad : nullptr, nullptr, pass,
                                         [&](long long pairs) { end_tiles(t, pass, pairs); });
}
template <int D, int KERN>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, (D == 3 ? 768 : 1024) / TileCfg<D>::THREADS) k_shift_t(TravArgs t, const Tile* tiles, const int* ntiles, Arrays out,
                                                 Displace disp) {
  wait_prior_grid();
  ShiftPass<D, KERN> pass;
  pass.a = t.a;
  pass.out = out;
  pass.disp = disp;
  run_tiles<D, 0, 0>(t, tiles, ntiles, nullptr, nullptr, pass);
}
template <int D, bool VAR>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, TileCfg<D>::MINB) k_pairs_t(TravArgs t, const Tile* tiles, const int* ntiles, int32_t* pi,
                                                 int32_t* pj, unsigned long long* count, long long cap) {
  PairPass<D, VAR> pass;
  pass.a = t.a;
  pass.pi = pi;
  pass.pj = pj;
  pass.count = count;
  pass.cap = cap;
  run_tiles<D, 0, 2>(t, tiles, ntiles, nullptr, nullptr, pass);
}
template <int D, int KERN>
__global__ void __launch_bounds__(adj_threads<D>(), adj_minb<D>()) k_adj_t(TravArgs t, const Tile* tiles, const int* ntiles, const float4* S,
                                               const float* Pp, const float4* XBin, const float4* VBin, float4* XBout,
                                               float4* VBout, double* nu_acc) {
  wait_prior_grid();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // the next kernel of the adjoint step may launch
  AdjPass<D, KERN> pass;
  pass.a = t.a;
  pass.S = S;
  pass.Pp = Pp;
  pass.XBin = XBin;
  pass.VBin = VBin;
  pass.XBout = XBout;
  pass.VBout = VBout;
  pass.nu_acc = nu_acc;
  run_tiles<D, (D == 2 ? 1 : 2), 0, AdjPass<D, KERN>, adj_lanes<D>()>(t, tiles, ntiles, S, D == 2 ? nullptr : Pp, pass);
}

template <int D, int KERN>
__global__ void __launch_bounds__(TileCfg<D>::THREADS, TileCfg<D>::MINB) k_adj_dens_t(TravArgs t, const Tile* tiles, const int* ntiles,
                                                                     const float4* XBin, const float4* VBin,
                                                                     float4* XBout, float4* VBout) {
  wait_prior_grid();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // the next kernel of the adjoint step may launch
  AdjDensityPass<D, KERN> pass;
  pass.XBin = XBin;
  pass.VBin = VBin;
  pass.XBout = XBout;
  pass.VBout = VBout;
  run_tiles<D, 1, 0>(t, tiles, ntiles, XBin, nullptr, pass);
}

// Per-scene sums of per-particle float partials into FP64 accumulators (acc[s] += sum over the
// scene's particles), in a fixed order: CTA (c, s) sums chunk c (kSumChunk particles) of scene s,
// and the CTA that finishes a scene's last chunk adds the chunk sums in chunk order.  B300's FP64
// rate is low per SM, so the chunks spread the FP64 additions over many SMs (one CTA summing a
// 16K-particle scene took about as long as half an adjoint sweep).  chunk: S x gridDim.x doubles;
// ctr: S counters, zero between launches (the last CTA resets its scene's).
constexpr int kSumChunk = 2048;
template <class T>
__global__ void k_sum_segments(const T* __restrict__ part, const DevSeg* __restrict__ segs, double* __restrict__ chunk,
                               int* __restrict__ ctr, double* __restrict__ acc) {
  wait_prior_grid();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // the next kernel of the adjoint step may launch
  __shared__ double sh[32];
  __shared__ int last;
  const int sg = blockIdx.y, nc = gridDim.x;
  const DevSeg& s = segs[sg];
  const int b = s.p0 + blockIdx.x * kSumChunk, e = min(s.p1, b + kSumChunk);
  double v = 0.0;
  for (int k = b + (int)threadIdx.x; k < e; k += blockDim.x) v += (double)__ldg(part + k);
  const double tot = block_sum(v, sh);
  if (threadIdx.x == 0) {
    chunk[(size_t)sg * nc + blockIdx.x] = tot;
    __threadfence();
    last = atomicAdd(ctr + sg, 1) == nc - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const volatile double* cv = chunk + (size_t)sg * nc;
    double sum = 0.0;
    for (int c = 0; c < nc; ++c) sum += cv[c];
    acc[sg] += sum;
    ctr[sg] = 0;
  }
}

// Deterministic sum of per-particle float partials into an FP64 accumulator (fixed order).
__global__ void k_sum_float_partials(const float* __restrict__ part, int n, double* __restrict__ acc) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += (double)part[k];
  double tot = block_sum(v, sh);
  if (threadIdx.x == 0) *acc += tot;
}

// ================================================================== launchers
template <int D>
size_t pass_smem(int extra) {
  if (extra == 0) return tile_smem_bytes<D, 0>();
  if (extra == 1) return tile_smem_bytes<D, 1>();
  return tile_smem_bytes<D, 2>();
}

static int g_num_sms = 148;
// Resident CTAs per SM of each pass kernel (queried once), so the grid is exactly one wave.
static std::map<const void*, int> g_occ;
static int pass_grid(const void* fn, int tiles_upper) {
  auto it = g_occ.find(fn);
  const int occ = it == g_occ.end() ? 1 : std::max(1, it->second);
  long long g = (long long)g_num_sms * occ;
  return (int)std::max<long long>(1, std::min<long long>(g, tiles_upper));
}
static void set_occ(const void* fn, size_t smem, int threads) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) == cudaSuccess) g_occ[fn] = n;
}

template <int D>
void launch_tiles(const DevSeg* segs, int S, const int* line_base, int n_lines, const int* cell_off, Tile* tiles,
                  int* ntiles, cudaStream_t st) {
  cudaMemsetAsync(ntiles, 0, sizeof(int), st);
  if (n_lines > 0) k_tiles<D><<<(n_lines + 7) / 8, 256, 0, st>>>(segs, S, line_base, n_lines, cell_off, tiles, ntiles);
}
template <int D>
void launch_wall_tiles(const Tile* tiles, const int* ntiles, int tiles_upper, const uint2* meta, int* list,
                       uint4* wall_p, uint4* fluid_p, int* count, cudaStream_t st) {
  cudaMemsetAsync(count, 0, 2 * sizeof(int), st);
  k_wall_tiles<D><<<(tiles_upper + 7) / 8, 256, 0, st>>>(tiles, ntiles, meta, list, wall_p, fluid_p, count);
}
template void launch_wall_tiles<2>(const Tile*, const int*, int, const uint2*, int*, uint4*, uint4*, int*, cudaStream_t);
template void launch_wall_tiles<3>(const Tile*, const int*, int, const uint2*, int*, uint4*, uint4*, int*, cudaStream_t);

template <int D, int KERN>
void launch_walls_t(const TravArgs& t, const Tile* tiles, const int* wall_tiles, const int* n_wall_tiles,
                    int tiles_upper, cudaStream_t st) {
  k_walls_t<D, KERN><<<pass_grid((const void*)k_walls_t<D, KERN>, tiles_upper), TileCfg<D>::THREADS, pass_smem<D>(0), st>>>(
      t, tiles, wall_tiles, n_wall_tiles);
}
template <int D, int KERN>
void launch_density_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, cudaStream_t st) {
  PdlLaunch L(pass_grid((const void*)k_density_t<D, KERN>, tiles_upper), TileCfg<D>::THREADS, pass_smem<D>(0), st);
  cudaLaunchKernelEx(&L.cfg, k_density_t<D, KERN>, t, tiles, ntiles);
}
template <int D, int KERN>
void launch_mdbc(const TravArgs& t, const Tile* tiles, const int* wall_tiles, const int* n_wall_tiles, int tiles_upper,
                 const float4* ghost, const int* orig_base, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((long long)tiles_upper * (TileCfg<D>::TP / 8),
                                                                   16LL * g_num_sms));
  k_mdbc<D, KERN><<<grid, 256, 0, st>>>(t, tiles, wall_tiles, n_wall_tiles, ghost, orig_base);
}
template <int D, int KERN>
void launch_walls_sweep_t(const TravArgs& t, uint4* wall_p, uint4* fluid_p, const int* n_lists,
                          int tiles_upper, const Arrays& out, const Displace& disp, cudaStream_t st) {
  PdlLaunch L(pass_grid((const void*)k_walls_sweep_t<D, KERN>, tiles_upper), TileCfg<D>::THREADS, pass_smem<D>(0), st);
  cudaLaunchKernelEx(&L.cfg, k_walls_sweep_t<D, KERN>, t, wall_p, fluid_p, n_lists, out, disp);
}
template <int D, int KERN>
void launch_grad_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, float4* grad,
                   cudaStream_t st) {
  PdlLaunch L(pass_grid((const void*)k_grad_t<D, KERN>, tiles_upper), TileCfg<D>::THREADS, pass_smem<D>(0), st);
  cudaLaunchKernelEx(&L.cfg, k_grad_t<D, KERN>, t, tiles, ntiles, grad);
}
template <int D, int KERN, bool INTEGRATE, bool RENORM>
static void launch_sweep_any(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const Arrays& out,
                             const RateOut& ro, const Displace& disp, const float4* grad, cudaStream_t st) {
  if constexpr (D == 3 && SPH_W3) {
    if (t.N <= kWMaxParticles && t.packed) {
      const int stride = (int)warp_pairs_stride(t.N);
      PdlLaunch P((stride + 255) / 256, 256, 0, st);
      cudaLaunchKernelEx(&P.cfg, k_pack_pairs3, t.N, stride, (const float4*)t.a.A, reinterpret_cast<float4*>(t.packed),
                         reinterpret_cast<float2*>(t.packed + 4 * (size_t)stride));
      auto fw = k_sweep_w<D, KERN, INTEGRATE, RENORM>;
      PdlLaunch L(pass_grid((const void*)fw, (tiles_upper + WCfg::WARPS - 1) / WCfg::WARPS), WCfg::THREADS,
                  warp_tiles_smem(), st);
      cudaLaunchKernelEx(&L.cfg, fw, t, tiles, ntiles, out, ro, disp, grad);
      return;
    }
  }
  auto fn = k_sweep_t<D, KERN, INTEGRATE, RENORM>;
  PdlLaunch L(pass_grid((const void*)fn, tiles_upper), TileCfg<D>::THREADS, pass_smem<D>(RENORM ? 1 : 0), st);
  cudaLaunchKernelEx(&L.cfg, fn, t, tiles, ntiles, out, ro, disp, grad);
}
template <int D, int KERN>
void launch_sweep_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const Arrays& out,
                    const Displace& disp, const float4* grad, cudaStream_t st) {
  if (grad) launch_sweep_any<D, KERN, true, true>(t, tiles, ntiles, tiles_upper, out, RateOut{}, disp, grad, st);
  else launch_sweep_any<D, KERN, true, false>(t, tiles, ntiles, tiles_upper, out, RateOut{}, disp, nullptr, st);
}
template <int D, int KERN>
void launch_rates_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const RateOut& ro,
                    const float4* grad, cudaStream_t st) {
  if (grad) launch_sweep_any<D, KERN, false, true>(t, tiles, ntiles, tiles_upper, Arrays{}, ro, Displace{}, grad, st);
  else launch_sweep_any<D, KERN, false, false>(t, tiles, ntiles, tiles_upper, Arrays{}, ro, Displace{}, nullptr, st);
}
template <int D, int KERN>
void launch_shift_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const Arrays& out,
                    const Displace& disp, cudaStream_t st) {
  PdlLaunch L(pass_grid((const void*)k_shift_t<D, KERN>, tiles_upper), TileCfg<D>::THREADS, pass_smem<D>(0), st);
  cudaLaunchKernelEx(&L.cfg, k_shift_t<D, KERN>, t, tiles, ntiles, out, disp);
}
template <int D>
void launch_pairs_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, int32_t* pi, int32_t* pj,
                    unsigned long long* count, long long cap, bool var, cudaStream_t st) {
  if (var)
    k_pairs_t<D, true><<<pass_grid((const void*)k_pairs_t<D, true>, tiles_upper), TileCfg<D>::THREADS, pass_smem<D>(0), st>>>(t, tiles, ntiles, pi, pj, count, cap);
  else
    k_pairs_t<D, false><<<pass_grid((const void*)k_pairs_t<D, false>, tiles_upper), TileCfg<D>::THREADS, pass_smem<D>(0), st>>>(t, tiles, ntiles, pi, pj, count, cap);
}
template <int D, int KERN>
void launch_adj_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const float4* S,
                  const float* Pp, const float4* XBin, const float4* VBin, float4* XBout, float4* VBout,
                  double* nu_acc, cudaStream_t st) {
  PdlLaunch L(pass_grid((const void*)k_adj_t<D, KERN>, tiles_upper), adj_threads<D>(),
              tile_smem_bytes<D, (D == 2 ? 1 : 2), adj_lanes<D>()>(), st);
  cudaLaunchKernelEx(&L.cfg, k_adj_t<D, KERN>, t, tiles, ntiles, S, Pp, XBin, VBin, XBout, VBout, nu_acc);
}
template <int D, int KERN>
void launch_adj_dens_t(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, const float4* XBin,
                       const float4* VBin, float4* XBout, float4* VBout, cudaStream_t st) {
  PdlLaunch L(pass_grid((const void*)k_adj_dens_t<D, KERN>, tiles_upper), TileCfg<D>::THREADS, pass_smem<D>(1), st);
  cudaLaunchKernelEx(&L.cfg, k_adj_dens_t<D, KERN>, t, tiles, ntiles, XBin, VBin, XBout, VBout);
}
// Shifting-by-optimisation passes: the objective (P1, P2) and its gradient (P3, P4; with `out`, the
// descent step).  Buffers: S1, S2, XB, G (float4 x N), V, Lp (N).
template <int D, int KERN>
void launch_opt_forward(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper,
                        const ShiftObjective& o, float4* S1, float4* S2, float* V, float* Lp, cudaStream_t st) {
  const int TH = TileCfg<D>::THREADS;
  k_opt_density<D, KERN><<<pass_grid((const void*)k_opt_density<D, KERN>, tiles_upper), TH, pass_smem<D>(0), st>>>(t, tiles, ntiles, S1);
  k_opt_color<D, KERN><<<pass_grid((const void*)k_opt_color<D, KERN>, tiles_upper), TH, pass_smem<D>(1), st>>>(t, tiles, ntiles, S1, S2, Lp, o);
  if (t.N > 0) k_opt_volumes<<<(t.N + 255) / 256, 256, 0, st>>>(t.N, S1, V);
}
template <int D, int KERN>
void launch_opt_backward(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper,
                         const ShiftObjective& o, const float4* S1, const float4* S2, const float* V, float4* XB,
                         float4* G, const Arrays* out, float step, cudaStream_t st) {
  const int TH = TileCfg<D>::THREADS;
  k_opt_adj<D, KERN><<<pass_grid((const void*)k_opt_adj<D, KERN>, tiles_upper), TH, pass_smem<D>(2), st>>>(t, tiles, ntiles, S1, S2, V, XB, o);
  if (out)
    k_opt_adj2<D, KERN, true><<<pass_grid((const void*)k_opt_adj2<D, KERN, true>, tiles_upper), TH, pass_smem<D>(1), st>>>(t, tiles, ntiles, XB, G, *out, step);
  else
    k_opt_adj2<D, KERN, false><<<pass_grid((const void*)k_opt_adj2<D, KERN, false>, tiles_upper), TH, pass_smem<D>(1), st>>>(t, tiles, ntiles, XB, G, Arrays{}, 0.f);
}
template <int D, int KERN>
void launch_varsupport(const TravArgs& t, const Tile* tiles, const int* ntiles, int tiles_upper, float4* Hs,
                       float4* out, float band, cudaStream_t st) {
  if (t.N > 0) k_support_payload<<<(t.N + 255) / 256, 256, 0, st>>>(t.N, t.a.O, t.segs, t.a.meta, Hs);
  k_varsupport<D, KERN><<<pass_grid((const void*)k_varsupport<D, KERN>, tiles_upper), TileCfg<D>::THREADS, pass_smem<D>(1), st>>>(
      t, tiles, ntiles, Hs, out, band);
}
void launch_set_support(int N, const uint2* meta, const int* orig_base, const float* H, float4* O, cudaStream_t st) {
  if (N > 0) k_set_support<<<(N + 255) / 256, 256, 0, st>>>(N, meta, orig_base, H, O);
}
void launch_unpermute3(int N, const uint2* meta, const int* orig_base, const float4* src, float* a, float* b, float* c,
                       cudaStream_t st) {
  if (N > 0) k_unpermute3<<<(N + 255) / 256, 256, 0, st>>>(N, meta, orig_base, src, a, b, c);
}
int sum_segments_chunks(long long max_seg_n) { return (int)std::max(1LL, (max_seg_n + kSumChunk - 1) / kSumChunk); }
void launch_sum_segments(const float* part, const DevSeg* segs, int S, int nchunks, double* chunk, int* ctr,
                         double* acc, cudaStream_t st) {
  PdlLaunch L(dim3(nchunks, S), 256, 0, st);
  cudaLaunchKernelEx(&L.cfg, k_sum_segments<float>, part, segs, chunk, ctr, acc);
}
void launch_sum_segments(const double* part, const DevSeg* segs, int S, int nchunks, double* chunk, int* ctr,
                         double* acc, cudaStream_t st) {
  PdlLaunch L(dim3(nchunks, S), 256, 0, st);
  cudaLaunchKernelEx(&L.cfg, k_sum_segments<double>, part, segs, chunk, ctr, acc);
}
void launch_sum_float_partials(const float* part, int n, double* acc, cudaStream_t st) {
  k_sum_float_partials<<<1, 1024, 0, st>>>(part, n, acc);
}

size_t packed_pairs_floats(long long N) { return 6 * warp_pairs_stride(N); }
bool warp_sweep(int dim, long long N) { return dim == 3 && SPH_W3 && N <= kWMaxParticles; }
int sweep_kernels(int dim, long long N, const float* packed) {
  return (dim == 3 && SPH_W3 && packed && N <= kWMaxParticles) ? 2 : 1;
}

cudaError_t configure_passes() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
#define SPH_ATTR(DIM, fn, bytes)                                                                                  \
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes)); \
  if (e == cudaSuccess) set_occ((const void*)fn, (bytes), TileCfg<DIM>::THREADS);
  SPH_ATTR(2, (k_walls_t<2, 0>), pass_smem<2>(0)) SPH_ATTR(2, (k_walls_t<2, 1>), pass_smem<2>(0))
  SPH_ATTR(3, (k_walls_t<3, 0>), pass_smem<3>(0)) SPH_ATTR(3, (k_walls_t<3, 1>), pass_smem<3>(0))
  SPH_ATTR(2, (k_density_t<2, 0>), pass_smem<2>(0)) SPH_ATTR(2, (k_density_t<2, 1>), pass_smem<2>(0))
  SPH_ATTR(3, (k_density_t<3, 0>), pass_smem<3>(0)) SPH_ATTR(3, (k_density_t<3, 1>), pass_smem<3>(0))
  SPH_ATTR(2, (k_sweep_t<2, 0, true, false>), pass_smem<2>(0)) SPH_ATTR(2, (k_sweep_t<2, 1, true, false>), pass_smem<2>(0))
  SPH_ATTR(3, (k_sweep_t<3, 0, true, false>), pass_smem<3>(0)) SPH_ATTR(3, (k_sweep_t<3, 1, true, false>), pass_smem<3>(0))
  SPH_ATTR(2, (k_sweep_t<2, 0, false, false>), pass_smem<2>(0)) SPH_ATTR(2, (k_sweep_t<2, 1, false, false>), pass_smem<2>(0))
  SPH_ATTR(3, (k_sweep_t<3, 0, false, false>), pass_smem<3>(0)) SPH_ATTR(3, (k_sweep_t<3, 1, false, false>), pass_smem<3>(0))
  SPH_ATTR(2, (k_sweep_t<2, 0, true, true>), pass_smem<2>(1)) SPH_ATTR(2, (k_sweep_t<2, 1, true, true>), pass_smem<2>(1))
  SPH_ATTR(3, (k_sweep_t<3, 0, true, true>), pass_smem<3>(1)) SPH_ATTR(3, (k_sweep_t<3, 1, true, true>), pass_smem<3>(1))
  SPH_ATTR(2, (k_sweep_t<2, 0, false, true>), pass_smem<2>(1)) SPH_ATTR(2, (k_sweep_t<2, 1, false, true>), pass_smem<2>(1))
  SPH_ATTR(3, (k_sweep_t<3, 0, false, true>), pass_smem<3>(1)) SPH_ATTR(3, (k_sweep_t<3, 1, false, true>), pass_smem<3>(1))
  SPH_ATTR(2, (k_opt_density<2, 0>), pass_smem<2>(0)) SPH_ATTR(2, (k_opt_density<2, 1>), pass_smem<2>(0))
  SPH_ATTR(3, (k_opt_density<3, 0>), pass_smem<3>(0)) SPH_ATTR(3, (k_opt_density<3, 1>), pass_smem<3>(0))
  SPH_ATTR(2, (k_opt_color<2, 0>), pass_smem<2>(1)) SPH_ATTR(2, (k_opt_color<2, 1>), pass_smem<2>(1))
  SPH_ATTR(3, (k_opt_color<3, 0>), pass_smem<3>(1)) SPH_ATTR(3, (k_opt_color<3, 1>), pass_smem<3>(1))
  SPH_ATTR(2, (k_opt_adj<2, 0>), pass_smem<2>(2)) SPH_ATTR(2, (k_opt_adj<2, 1>), pass_smem<2>(2))
  SPH_ATTR(3, (k_opt_adj<3, 0>), pass_smem<3>(2)) SPH_ATTR(3, (k_opt_adj<3, 1>), pass_smem<3>(2))
  SPH_ATTR(2, (k_opt_adj2<2, 0, true>), pass_smem<2>(1)) SPH_ATTR(2, (k_opt_adj2<2, 1, true>), pass_smem<2>(1))
  SPH_ATTR(3, (k_opt_adj2<3, 0, true>), pass_smem<3>(1)) SPH_ATTR(3, (k_opt_adj2<3, 1, true>), pass_smem<3>(1))
  SPH_ATTR(2, (k_opt_adj2<2, 0, false>), pass_smem<2>(1)) SPH_ATTR(2, (k_opt_adj2<2, 1, false>), pass_smem<2>(1))
  SPH_ATTR(3, (k_opt_adj2<3, 0, false>), pass_smem<3>(1)) SPH_ATTR(3, (k_opt_adj2<3, 1, false>), pass_smem<3>(1))
  SPH_ATTR(2, (k_walls_sweep_t<2, 0>), pass_smem<2>(0)) SPH_ATTR(2, (k_walls_sweep_t<2, 1>), pass_smem<2>(0))
  SPH_ATTR(3, (k_walls_sweep_t<3, 0>), pass_smem<3>(0)) SPH_ATTR(3, (k_walls_sweep_t<3, 1>), pass_smem<3>(0))
  SPH_ATTR(2, (k_shift_t<2, 0>), pass_smem<2>(0)) SPH_ATTR(2, (k_shift_t<2, 1>), pass_smem<2>(0))
  SPH_ATTR(3, (k_shift_t<3, 0>), pass_smem<3>(0)) SPH_ATTR(3, (k_shift_t<3, 1>), pass_smem<3>(0))
  SPH_ATTR(2, (k_grad_t<2, 0>), pass_smem<2>(0)) SPH_ATTR(2, (k_grad_t<2, 1>), pass_smem<2>(0))
  SPH_ATTR(3, (k_grad_t<3, 0>), pass_smem<3>(0)) SPH_ATTR(3, (k_grad_t<3, 1>), pass_smem<3>(0))
  SPH_ATTR(2, (k_pairs_t<2, false>), pass_smem<2>(0)) SPH_ATTR(3, (k_pairs_t<3, false>), pass_smem<3>(0))
  SPH_ATTR(2, (k_pairs_t<2, true>), pass_smem<2>(0)) SPH_ATTR(3, (k_pairs_t<3, true>), pass_smem<3>(0))
  SPH_ATTR(2, (k_varsupport<2, 0>), pass_smem<2>(1)) SPH_ATTR(2, (k_varsupport<2, 1>), pass_smem<2>(1))
  SPH_ATTR(3, (k_varsupport<3, 0>), pass_smem<3>(1)) SPH_ATTR(3, (k_varsupport<3, 1>), pass_smem<3>(1))
#define SPH_AATTR(DIM, fn, bytes)                                                                                 \
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes)); \
  if (e == cudaSuccess) set_occ((const void*)fn, (bytes), adj_threads<DIM>());
  SPH_AATTR(2, (k_adj_t<2, 0>), (tile_smem_bytes<2, 1, adj_lanes<2>()>()))
  SPH_AATTR(2, (k_adj_t<2, 1>), (tile_smem_bytes<2, 1, adj_lanes<2>()>()))
  SPH_AATTR(3, (k_adj_t<3, 0>), (tile_smem_bytes<3, 2, adj_lanes<3>()>()))
  SPH_AATTR(3, (k_adj_t<3, 1>), (tile_smem_bytes<3, 2, adj_lanes<3>()>()))
#undef SPH_AATTR
  SPH_ATTR(2, (k_adj_dens_t<2, 0>), pass_smem<2>(1)) SPH_ATTR(2, (k_adj_dens_t<2, 1>), pass_smem<2>(1))
  SPH_ATTR(3, (k_adj_dens_t<3, 0>), pass_smem<3>(1)) SPH_ATTR(3, (k_adj_dens_t<3, 1>), pass_smem<3>(1))
#define SPH_WATTR(fn)                                                                                            \
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                                 (int)warp_tiles_smem());                                           \
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributePreferredSharedMemoryCarveout,   \
                                                 warp_tiles_carveout());                                            \
  if (e == cudaSuccess) set_occ((const void*)fn, warp_tiles_smem(), WCfg::THREADS);
  SPH_WATTR((k_sweep_w<3, 0, true, false>)) SPH_WATTR((k_sweep_w<3, 1, true, false>))
  SPH_WATTR((k_sweep_w<3, 0, false, false>)) SPH_WATTR((k_sweep_w<3, 1, false, false>))
  SPH_WATTR((k_sweep_w<3, 0, true, true>)) SPH_WATTR((k_sweep_w<3, 1, true, true>))
  SPH_WATTR((k_sweep_w<3, 0, false, true>)) SPH_WATTR((k_sweep_w<3, 1, false, true>))
#undef SPH_WATTR
#undef SPH_ATTR
  return e;
}

#define SPH_INST_PD(D)                                                                                       \
  template void launch_tiles<D>(const DevSeg*, int, const int*, int, const int*, Tile*, int*, cudaStream_t);    \
  template void launch_pairs_t<D>(const TravArgs&, const Tile*, const int*, int, int32_t*, int32_t*,          \
                                  unsigned long long*, long long, bool, cudaStream_t);
SPH_INST_PD(2)
SPH_INST_PD(3)
#define SPH_INST_PDK(D, K)                                                                                   \
  template void launch_walls_t<D, K>(const TravArgs&, const Tile*, const int*, const int*, int, cudaStream_t); \
  template void launch_density_t<D, K>(const TravArgs&, const Tile*, const int*, int, cudaStream_t);        \
  template void launch_grad_t<D, K>(const TravArgs&, const Tile*, const int*, int, float4*, cudaStream_t);   \
  template void launch_varsupport<D, K>(const TravArgs&, const Tile*, const int*, int, float4*, float4*, float, \
                                        cudaStream_t);                                                       \
  template void launch_opt_forward<D, K>(const TravArgs&, const Tile*, const int*, int, const ShiftObjective&, \
                                         float4*, float4*, float*, float*, cudaStream_t);                     \
  template void launch_opt_backward<D, K>(const TravArgs&, const Tile*, const int*, int, const ShiftObjective&, \
                                          const float4*, const float4*, const float*, float4*, float4*,       \
                                          const Arrays*, float, cudaStream_t);                                \
  template void launch_mdbc<D, K>(const TravArgs&, const Tile*, const int*, const int*, int, const float4*,  \
                                  const int*, cudaStream_t);                                                 \
  template void launch_walls_sweep_t<D, K>(const TravArgs&, uint4*, uint4*, const int*, int,                     \
                                           const Arrays&, const Displace&, cudaStream_t);                    \
  template void launch_shift_t<D, K>(const TravArgs&, const Tile*, const int*, int, const Arrays&,          \
                                     const Displace&, cudaStream_t);                                         \
  template void launch_sweep_t<D, K>(const TravArgs&, const Tile*, const int*, int, const Arrays&, const Displace&, \
                                     const float4*, cudaStream_t);                                           \
  template void launch_rates_t<D, K>(const TravArgs&, const Tile*, const int*, int, const RateOut&, const float4*, \
                                     cudaStream_t);                                                          \
  template void launch_adj_t<D, K>(const TravArgs&, const Tile*, const int*, int, const float4*, const float*,  \
                                   const float4*, const float4*, float4*, float4*, double*, cudaStream_t);     \
  template void launch_adj_dens_t<D, K>(const TravArgs&, const Tile*, const int*, int, const float4*,          \
                                        const float4*, float4*, float4*, cudaStream_t);
SPH_INST_PDK(2, 0)
SPH_INST_PDK(2, 1)
SPH_INST_PDK(3, 0)
SPH_INST_PDK(3, 1)

}  // namespace sph
