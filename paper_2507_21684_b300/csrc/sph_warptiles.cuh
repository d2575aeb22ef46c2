// Warp-per-tile traversal of the tiled neighbour passes (one thread per target).
//
// A warp owns one tile (at most 32 consecutive sorted particles of one cell line) at a time and
// walks, in lockstep, the union of its targets' stencil runs: for each of the 3^(d-1) neighbour
// lines, the columns that some target of the tile can reach (the same reach test as the staged
// traversal, reduced over the warp with redux.sync), split into the in-box range and the two
// periodic image cells.  Every candidate record is therefore read once per warp at one address
// (a broadcast through L1), tested by every lane against its own target and, on a hit, appended
// to the lane's list in shared memory; the lists are evaluated (Body::pair_at) from the neighbour
// records in global memory when a lane's list may overflow and at the end of the tile.
//
// Against the staged traversal (sph_tiles.cuh: a CTA stages the 3^(d-1) lines into shared memory
// and LANES threads split one target's candidates) this needs no staging, no CTA barrier per tile,
// no reduction over lanes and no tile-size fallback, and its loop control is warp-uniform; it
// tests more candidates per target (the union of 32 targets' stencils instead of each target's
// own) but each test is a broadcast load and six FP32 operations.  Each warp takes its own tiles
// from the launch's tile counter.
//
// Periodic images follow the staged traversal's convention, so that every coordinate difference
// is formed from exactly shifted operands: a lower image (the line or column wraps below the box)
// takes the box length off the neighbour's coordinate, which lies in the upper half of the box; an
// upper image takes it off the target's.
#pragma once
#include "sph_tiles.cuh"

namespace sph {

#ifndef SPH_W_WARPS
#define SPH_W_WARPS 4
#endif
#ifndef SPH_W_LIST
#define SPH_W_LIST 64
#endif
// entries of every lane's ring evaluated at a time when one may overflow
#ifndef SPH_W_EVAL
#define SPH_W_EVAL (SPH_W_LIST / 2)
#endif
// candidates per step of the test loop (two per paired load; loads in flight per lane)
#ifndef SPH_W_UNROLL
#define SPH_W_UNROLL 8
#endif
// CTAs per SM the warp-traversal kernels are compiled for (register budget 64K / (MINB x THREADS))
#ifndef SPH_W_MINB
#define SPH_W_MINB 5
#endif

struct WCfg {
  static constexpr int WARPS = SPH_W_WARPS;    // warps per CTA
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int LIST = SPH_W_LIST;      // hit-ring entries per thread
  static constexpr int EVAL = SPH_W_EVAL;      // entries per lane evaluated at a time
  static constexpr int UNROLL = SPH_W_UNROLL;  // candidates per step of the test loop
};
static_assert(WCfg::LIST > WCfg::UNROLL, "a step of the test loop must fit into a list with room");
static_assert(WCfg::EVAL >= WCfg::UNROLL && WCfg::EVAL <= WCfg::LIST, "an evaluation frees a step's room");
static_assert(TileCfg<3>::TP <= 32, "a warp holds one tile's targets");

// Hit-list entry: neighbour index in the packed arrays (26 bits) and the shifts of the pair:
// bit 26 + q: the neighbour's coordinate q takes off L_q; bit 29 + q: the target's does.
constexpr int kWIdxBits = 26;
constexpr uint32_t kWIdxMask = (1u << kWIdxBits) - 1u;
constexpr long long kWMaxParticles = 1LL << kWIdxBits;

__host__ __device__ constexpr size_t warp_tiles_smem() { return sizeof(uint32_t) * WCfg::LIST * WCfg::THREADS; }
// Shared-memory carveout (percent of the SM's maximum) that holds MINB CTAs' lists and no more:
// the rest of the unified L1 caches the neighbour records the traversal reads from global memory.
constexpr int warp_tiles_carveout() {
  return (int)((100 * (size_t)SPH_W_MINB * (warp_tiles_smem() + 1024) + 228 * 1024 - 1) / (228 * 1024));
}

// A lane's hit list is a ring of LIST entries (free-running counters head and tail): the tests
// append at head, the evaluation takes entries from tail.  When some lane's ring may overflow, the
// warp evaluates up to EVAL entries of every lane (the oldest ones) and goes on testing: the lanes
// keep about half a ring each, so an evaluation keeps most lanes busy (evaluating every list to
// the end whenever the fullest one is full leaves the others idle for the difference; a ring of
// 64 with 32 per evaluation needs a third fewer evaluation steps than emptying lists of 48 on the
// 128^3 vortex, counted on its cell lists).
static_assert((WCfg::LIST & (WCfg::LIST - 1)) == 0, "the hit ring's length is a power of two");

// Evaluation of up to `most` entries of every lane's ring: the warp iterates up to the longest
// batch (lanes with fewer entries idle), each lane loads its neighbour's records and calls
// body.pair_at with both ends in the pair's periodic image.  Returns the entries evaluated by this
// lane.  EX0 / EX1: the pass stages a float4 / float payload with the neighbours.
template <int D, bool EX0, bool EX1, class Body>
__device__ __forceinline__ int warp_drain(const float* L, const Arrays& a, const float4* __restrict__ extra0,
                                          const float* __restrict__ extra1, const uint32_t* list, unsigned head,
                                          unsigned& tail, int most, const float* xt, Body& body) {
  constexpr unsigned MASK = WCfg::LIST - 1;
  const int lane = threadIdx.x & 31;
  const int mine = min((int)(head - tail), most);
  const int m = (int)__reduce_max_sync(kFull, (unsigned)mine);
  for (int e = 0; e < m; ++e) {
    if (e < mine) {
      const uint32_t code = list[((tail + (unsigned)e) & MASK) * 32u + lane];
      const int j = (int)(code & kWIdxMask);
      PD<D> pj = load_pd<D>(a, j);
      float xs[D];
#pragma unroll
      for (int q = 0; q < D; ++q) xs[q] = xt[q];
      if (code >> kWIdxBits) {  // a periodic image (particles near the box faces only)
#pragma unroll
        for (int q = 0; q < D; ++q) {
          if ((code >> (29 + q)) & 1u) xs[q] -= L[q];
          if ((code >> (26 + q)) & 1u) pj.x[q] -= L[q];
        }
      }
      const float4 ex = EX0 ? __ldg(extra0 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float pp = EX1 ? __ldg(extra1 + j) : 0.f;
      body.pair_at(xs, pj, ex, pp, j);
    }
  }
  tail += (unsigned)mine;
  return mine;
}

// Test the candidates [g0, g1) of one run (per lane: the run of the lane's group) against this
// lane's target, two at a time: the positions come as pairs (PXY[p] = (x_2p, x_2p+1, y_2p, y_2p+1),
// PZ[p] = (z_2p, z_2p+1), packed before the launch) and the squared distances of a pair are formed
// with the paired FP32 instructions.  nt: minus the target's coordinates in the run's image plus
// the shift taken off the candidates (the test's rounding near |r| = H does not matter: W and
// grad W vanish there; the evaluation forms the pair's separation from exactly shifted operands).
// Hits are appended to the lane's ring with the entry tag.  The loop is warp-uniform (up to the
// longest run of the warp); a lane whose run is shorter tests clamped pairs and keeps none.
// ZERO_OK: a pair at zero distance (the target itself) is harmless to the pass, so only
// r^2 < H^2 is tested; the caller discounts the target from the pair count.
template <int D, bool ZERO_OK, class Drain>
__device__ __forceinline__ void warp_scan_run(const float4* __restrict__ PXY, const float2* __restrict__ PZ, int g0,
                                              int g1, float2 ntx, float2 nty, float2 ntz, uint32_t tag, float H2,
                                              uint32_t* list, unsigned& head, const unsigned& tail, Drain& drain) {
  constexpr int U = WCfg::UNROLL / 2;  // pairs per step
  constexpr unsigned MASK = WCfg::LIST - 1;
  const int lane = threadIdx.x & 31;
  const int pa = g0 >> 1;
  const int np = g1 > g0 ? ((g1 + 1) >> 1) - pa : 0;
  const int mlen = (int)__reduce_max_sync(kFull, (unsigned)np);
  const int plast = max(pa + np - 1, 0);  // a valid pair for the clamped tests of a short run
  auto test = [&](int it, float4 Q, float2 Z) {
    const int k0 = 2 * (pa + it);
    const float2 dx = __fadd2_rn(make_float2(Q.x, Q.y), ntx);
    const float2 dy = __fadd2_rn(make_float2(Q.z, Q.w), nty);
    float2 r2 = __ffma2_rn(dy, dy, __fmul2_rn(dx, dx));
    if (D == 3) {
      const float2 dz = __fadd2_rn(Z, ntz);
      r2 = __ffma2_rn(dz, dz, r2);
    }
    const bool in = it < np;
    list[(head & MASK) * 32u + lane] = (uint32_t)k0 | tag;
    head += (in && k0 >= g0 && r2.x < H2 && (ZERO_OK || r2.x > 0.f)) ? 1u : 0u;
    list[(head & MASK) * 32u + lane] = (uint32_t)(k0 + 1) | tag;
    head += (in && k0 + 1 < g1 && r2.y < H2 && (ZERO_OK || r2.y > 0.f)) ? 1u : 0u;
  };
  auto ldq = [&](int it) { return __ldg(PXY + min(pa + it, plast)); };
  auto ldz = [&](int it) { return D == 3 ? __ldg(PZ + min(pa + it, plast)) : make_float2(0.f, 0.f); };
  int it = 0;
  for (; it + U <= mlen; it += U) {
    if (__any_sync(kFull, (int)(head - tail) > WCfg::LIST - 2 * U)) drain();
    float4 Q[U];
    float2 Z[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      Q[u] = ldq(it + u);
      Z[u] = ldz(it + u);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) test(it + u, Q[u], Z[u]);
  }
  if (it < mlen) {
    if (__any_sync(kFull, (int)(head - tail) > WCfg::LIST - 2 * U)) drain();
    for (; it < mlen; ++it) test(it, ldq(it), ldz(it));
  }
}

// One tile on one warp: per-lane target set-up, the union runs of every neighbour line, the
// tests, the evaluation of the lists and the pass's epilogue.  The lanes are grouped by their
// target's cell (match_any): each group walks the union of its own targets' reach, so a tile
// whose targets span two or three cells does not test every target against all of them.
// Returns the pairs this lane evaluated (the target itself not counted).
template <int D, bool ZERO_OK, bool EX0, bool EX1, class Pass>
__device__ __forceinline__ int warp_tile_task(const TravArgs& t, const Tile& T, uint32_t* list,
                                              const float4* __restrict__ extra0, const float* __restrict__ extra1,
                                              Pass& pass) {
  constexpr int NL = TileCfg<D>::NL;
  const DevSeg& s = t.segs[T.seg];
  const int lane = threadIdx.x & 31;
  const int i = T.p0 + lane;
  const bool valid = i < T.p1;
  const TgtView tv{t.a, pass.tex0(), pass.tex1(), i};
  const bool want = valid && Pass::wants(t.a.meta[i].x);
  if (!__any_sync(kFull, want)) {  // no target of this pass in the tile
    if (valid) pass.skip(i, tv);
    return 0;
  }
  typename Pass::Body body;
  bool active = false;
  float xt[3] = {0.f, 0.f, 0.f}, fl[3] = {0.f, 0.f, 0.f}, fh[3] = {0.f, 0.f, 0.f};
  int cx = -1;  // invalid lanes form a group of their own and walk nothing
  if (valid) {
    active = pass.init(body, s, i, tv);
    const float4 A = __ldg(t.a.A + i);
    xt[0] = A.x; xt[1] = A.y; xt[2] = D == 3 ? A.z : 0.f;
    const int c[3] = {(int)t.keys[i] - (s.cell_base + (T.cz * s.n[1] + T.cy) * s.n[0]), T.cy, T.cz};
    cx = c[0];
#pragma unroll
    for (int q = 0; q < D; ++q) {  // squared distances to the own cell's faces (0 past a face)
      const float lo = s.lo[q] + s.cs[q] * (float)c[q];
      const float a0 = fmaxf(xt[q] - lo, 0.f), a1 = fmaxf(lo + s.cs[q] - xt[q], 0.f);
      fl[q] = a0 * a0;
      fh[q] = a1 * a1;
    }
  }
  // the lanes of one cell form a group (contiguous lanes: the targets are in cell order); the
  // groups' lowest lanes
  const unsigned gmask = __match_any_sync(kFull, cx);
  const unsigned leaders = __ballot_sync(kFull, (gmask & ((1u << lane) - 1u)) == 0u);
  const float L[3] = {s.L[0], s.L[1], D == 3 ? s.L[2] : 0.f};
  const float H2 = s.H2, R2 = s.trimR2;
  const int nx = s.n[0];
  const bool px = s.periodic_mask & 1;
  unsigned head = 0u, tail = 0u;
  int np = 0;
  auto drain = [&]() { np += warp_drain<D, EX0, EX1>(L, t.a, extra0, extra1, list, head, tail, WCfg::EVAL, xt, body); };
  for (int l = 0; l < NL; ++l) {
    float tsh[2], csh[2];
    const int lc = tile_line<D>(s, T, l, tsh, csh);  // uniform over the warp
    if (lc < 0) continue;
    const int dy = (D == 2) ? l - 1 : l % 3 - 1;
    const int dz = (D == 2) ? 0 : l / 3 - 1;
    int clo = 0x7fffffff, chi = -0x7fffffff;
    if (active) {
      const float dyz = (dy < 0 ? fl[1] : dy > 0 ? fh[1] : 0.f) + (dz < 0 ? fl[2] : dz > 0 ? fh[2] : 0.f);
      if (dyz < R2) {
        clo = cx - (fl[0] + dyz < R2 ? 1 : 0);
        chi = cx + 1 + (fh[0] + dyz < R2 ? 1 : 0);
      }
    }
    {  // the union over the lane's group: full-warp reductions, one group at a time
      int glo = clo, ghi = chi;
      for (unsigned m = leaders; m; m &= m - 1u) {
        const unsigned gm = __shfl_sync(kFull, gmask, __ffs(m) - 1);
        const bool in = (gm >> lane) & 1u;
        const int a = __reduce_min_sync(kFull, in ? clo : 0x7fffffff);
        const int b = __reduce_max_sync(kFull, in ? chi : -0x7fffffff);
        if (in) { glo = a; ghi = b; }
      }
      clo = glo;
      chi = ghi;
    }
    if (!px) {
      clo = max(clo, 0);
      chi = min(chi, nx);
    }
    if (!__any_sync(kFull, active && clo < chi)) continue;  // (lanes of wall targets walk nothing)
    // the line's image on y and z: the target takes off L (upper) or the records do (lower)
    const float tl[3] = {xt[0], tsh[0] != 0.f ? xt[1] - L[1] : xt[1], (D == 3 && tsh[1] != 0.f) ? xt[2] - L[2] : xt[2]};
    const float sh[3] = {0.f, -csh[0], D == 3 ? -csh[1] : 0.f};
    const uint32_t tag = (tsh[0] != 0.f ? 1u << 30 : 0u) | (D == 3 && tsh[1] != 0.f ? 1u << 31 : 0u) |
                         (csh[0] != 0.f ? 1u << 27 : 0u) | (D == 3 && csh[1] != 0.f ? 1u << 28 : 0u);
    const float4* PXY = reinterpret_cast<const float4*>(t.packed);
    const float2* PZ = reinterpret_cast<const float2*>(t.packed + 4 * (size_t)((t.N + 1) / 2));
    // left periodic image (groups whose union starts left of column 0): the last column of the
    // line, shifted down by L
    if (__any_sync(kFull, active && clo < 0)) {
      int g0 = 0, g1 = 0;
      if (active && clo < 0) { g0 = t.cell_off[lc + nx - 1]; g1 = t.cell_off[lc + nx]; }
      warp_scan_run<D, ZERO_OK>(PXY, PZ, g0, g1, make_float2(-(tl[0] + L[0]), -(tl[0] + L[0])),
                                make_float2(-(tl[1] + sh[1]), -(tl[1] + sh[1])),
                                make_float2(-(tl[2] + sh[2]), -(tl[2] + sh[2])), tag | (1u << 26), H2, list, head,
                                tail, drain);
    }
    // in-box columns
    {
      const int c0 = max(clo, 0), c1 = min(chi, nx);
      int g0 = 0, g1 = 0;
      if (active && c0 < c1) { g0 = t.cell_off[lc + c0]; g1 = t.cell_off[lc + c1]; }
      warp_scan_run<D, ZERO_OK>(PXY, PZ, g0, g1, make_float2(-tl[0], -tl[0]),
                                make_float2(-(tl[1] + sh[1]), -(tl[1] + sh[1])),
                                make_float2(-(tl[2] + sh[2]), -(tl[2] + sh[2])), tag, H2, list, head, tail, drain);
    }
    // right periodic image (groups whose union ends right of the last column): the first column
    // of the line; the target takes off L
    if (__any_sync(kFull, active && chi > nx)) {
      int g0 = 0, g1 = 0;
      if (active && chi > nx) { g0 = t.cell_off[lc]; g1 = t.cell_off[lc + 1]; }
      const float txr = xt[0] - L[0];
      warp_scan_run<D, ZERO_OK>(PXY, PZ, g0, g1, make_float2(-txr, -txr),
                                make_float2(-(tl[1] + sh[1]), -(tl[1] + sh[1])),
                                make_float2(-(tl[2] + sh[2]), -(tl[2] + sh[2])), tag | (1u << 29), H2, list, head,
                                tail, drain);
    }
  }
  while (__any_sync(kFull, head != tail)) drain();
  if (ZERO_OK && active) --np;  // the target found itself
  body.template reduce<1>();
  if (valid) pass.finish(body, s, i, tv);
  return np;
}

// Skeleton of a warp-traversal launch: each warp takes its first tile by its index in the grid,
// then further ones from the launch's tile counter; the CTA ends as the staged launches do
// (end_tiles in sph_passes.cu: partial results, pair count, counters reset by the last CTA).
template <int D, bool ZERO_OK, bool EX0, bool EX1, class Pass, class End>
__device__ __forceinline__ void run_warp_tiles(const TravArgs& t, const Tile* __restrict__ tiles,
                                               const int* __restrict__ ntiles, const float4* __restrict__ extra0,
                                               const float* __restrict__ extra1, Pass& pass, End end) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5;
  uint32_t* list = reinterpret_cast<uint32_t*>(smraw) + (size_t)warp * WCfg::LIST * 32;
  const int nt = *ntiles;
  long long pairs = 0;
  int ti = blockIdx.x * WCfg::WARPS + warp;
  while (ti < nt) {
    const Tile T = tiles[ti];
    pairs += warp_tile_task<D, ZERO_OK, EX0, EX1>(t, T, list, extra0, extra1, pass);
    int nxt = 0;
    if ((threadIdx.x & 31) == 0) nxt = (int)gridDim.x * WCfg::WARPS + atomicAdd(t.tile_ctr, 1);
    ti = __shfl_sync(kFull, nxt, 0);
  }
  end(pairs);
}

}  // namespace sph
