// Warp-per-tile traversal of the tiled neighbour passes (one thread per target).
//
// A warp owns one tile (at most 32 consecutive sorted particles of one cell line) at a time.  Each
// lane walks its own target's stencil: for each of the 3^(d-1) neighbour lines, the columns its
// target can reach (the same face-distance test as the staged traversal), split into the in-box
// range and the two periodic image cells.  The walks run in lockstep over the warp (up to the
// longest run of the warp; shorter runs are masked), so their loop control is warp-uniform, and
// lanes of one cell, whose runs mostly coincide, read the same candidate records (a broadcast
// through L1).  The candidates' positions come packed as pairs and are tested two at a time with
// paired FP32 instructions; each step of the test loop records the step's hits as one entry of a
// per-lane ring in shared memory (the step's first pair and a bit mask of its hits), so that a
// candidate costs a bit, not a list append.  The rings are evaluated (Body::pair_at) from the
// neighbour records in global memory when one may overflow and at the end of the tile.
//
// Against the staged traversal (sph_tiles.cuh: a CTA stages the 3^(d-1) lines into shared memory
// and LANES threads split one target's candidates) this needs no staging, no CTA barrier per tile,
// no reduction over lanes and no tile-size fallback.  A CTA (one per SM) claims chunks of
// consecutive tiles from the launch's tile counter and its warps take the chunk's tiles as they
// free up.
//
// Periodic images follow the staged traversal's convention, so that every coordinate difference
// is formed from exactly shifted operands: a lower image (the line or column wraps below the box)
// takes the box length off the neighbour's coordinate, which lies in the upper half of the box; an
// upper image takes it off the target's.
#pragma once
#include "sph_tiles.cuh"

namespace sph {

// warps per CTA: one CTA of 24 warps per SM (80 registers a thread), so that every warp of an SM
// takes its tiles from the same chunks and shares the SM's L1
#ifndef SPH_W_WARPS
#define SPH_W_WARPS 24
#endif
// hit-ring entries per lane (one entry per step of the test loop that found a hit); 16 entries
// (96 KB of rings per CTA) leave the rest of the SM's unified memory to L1
#ifndef SPH_W_LIST
#define SPH_W_LIST 16
#endif
// hits of every lane evaluated at a time when some lane's ring is full
#ifndef SPH_W_EVAL
#define SPH_W_EVAL 32
#endif
// candidates per step of the test loop (two per paired load; loads in flight per lane)
#ifndef SPH_W_UNROLL
#define SPH_W_UNROLL 16
#endif
// evaluate two hits per iteration of the evaluation loop (their loads in flight together)
#ifndef SPH_W_DRAIN2
#define SPH_W_DRAIN2 1
#endif
// the two hits of an iteration evaluated together with the paired FP32 operations (passes whose
// body provides pair_at2; the 128^3 vortex 1.195 -> 1.170 ms per step)
#ifndef SPH_W_PAIR2
#define SPH_W_PAIR2 1
#endif
// CTAs per SM the warp-traversal kernels are compiled for (register budget 64K / (MINB x THREADS))
#ifndef SPH_W_MINB
#define SPH_W_MINB 1
#endif
// consecutive tiles a CTA claims from the launch's counter at a time, shared out to its warps as
// they free up (0: every warp claims its own tiles)
#ifndef SPH_W_CHUNK
#define SPH_W_CHUNK 8
#endif

struct WCfg {
  static constexpr int WARPS = SPH_W_WARPS;    // warps per CTA
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int LIST = SPH_W_LIST;      // hit-ring entries per thread
  static constexpr int EVAL = SPH_W_EVAL;      // hits per lane evaluated at a time
  static constexpr int UNROLL = SPH_W_UNROLL;  // candidates per step of the test loop
};
static_assert(WCfg::UNROLL % 2 == 0 && WCfg::UNROLL <= 16, "a step's hit mask holds up to 16 candidates");
// an evaluation of EVAL hits finishes the entry in registers (up to UNROLL hits) and frees a slot
static_assert(WCfg::EVAL > WCfg::UNROLL, "an evaluation frees a ring slot");
static_assert((WCfg::LIST & (WCfg::LIST - 1)) == 0, "the hit ring's length is a power of two");
static_assert(TileCfg<3>::TP <= 32, "a warp holds one tile's targets");

// Hit-ring entry: x = index of the first candidate pair of the step, y = the step's hit mask (bit
// k: candidate 2x + k) in bits 0-15 and the shifts of the run's periodic image in bits 16-21
// (bit 16 + q: the neighbour's coordinate q takes off L_q; bit 19 + q: the target's does).
constexpr uint32_t kWHitBits = 0xffffu;
constexpr int kWShift = 16;
constexpr long long kWMaxParticles = 1LL << 30;
// The packed pair arrays are padded by this many pairs: the last step of a run reads up to
// UNROLL/2 - 1 pairs past the run's end (masked out of the hits).
constexpr int kWPadPairs = 16;
static_assert(WCfg::UNROLL / 2 <= kWPadPairs, "the pair arrays' padding covers a step");
// Pairs per packed array (positions as pairs (x_2p, x_2p+1, y_2p, y_2p+1) and (z_2p, z_2p+1));
// the z array starts 4 x this many floats into the buffer, which holds 6 x this many floats.
__host__ __device__ inline size_t warp_pairs_stride(long long N) { return (size_t)((N + 1) / 2) + kWPadPairs; }

__host__ __device__ constexpr size_t warp_tiles_smem() { return sizeof(uint2) * WCfg::LIST * WCfg::THREADS; }
// Shared-memory carveout (percent of the SM's maximum) that holds MINB CTAs' rings and no more:
// the rest of the unified L1 caches the neighbour records the traversal reads from global memory.
constexpr int warp_tiles_carveout() {
  return (int)((100 * (size_t)SPH_W_MINB * (warp_tiles_smem() + 1024) + 228 * 1024 - 1) / (228 * 1024));
}

// A lane's hits: the ring (free-running counters head and tail, in entries), the entry being
// evaluated (its first pair and its remaining mask and shifts) and the hits not yet evaluated.
// When some lane's ring is full, the warp evaluates up to EVAL hits of every lane (the oldest
// ones) and goes on testing, so the lanes keep part of their rings and an evaluation keeps most
// lanes busy.
struct WHits {
  unsigned head = 0u, tail = 0u;
  uint32_t base = 0u, bits = 0u;
  int pend = 0;
};

// One hit's evaluation: body.pair_at with both ends in the pair's periodic image.  EX0 / EX1: the
// pass reads a float4 / float payload of the neighbours.
template <int D, bool EX0, bool EX1, class Body>
__device__ __forceinline__ void warp_eval_hit(const float* L, const Arrays& a, const float4* __restrict__ extra0,
                                              const float* __restrict__ extra1, int j, uint32_t sh, PD<D> pj,
                                              const float* xt, Body& body) {
  float xs[D];
#pragma unroll
  for (int q = 0; q < D; ++q) xs[q] = xt[q];
  if (sh) {  // a periodic image (particles near the box faces only)
#pragma unroll
    for (int q = 0; q < D; ++q) {
      if ((sh >> (3 + q)) & 1u) xs[q] -= L[q];
      if ((sh >> q) & 1u) pj.x[q] -= L[q];
    }
  }
  const float4 ex = EX0 ? __ldg(extra0 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float pp = EX1 ? __ldg(extra1 + j) : 0.f;
  body.pair_at(xs, pj, ex, pp, j);
}

// The next hit of a lane: the lowest bit of its current entry, or of the next entry of its ring
// when that one is spent.  j: the neighbour's index; sh: the pair's shifts.
__device__ __forceinline__ void warp_pop_hit(const uint2* ring, WHits& h, int& j, uint32_t& sh) {
  constexpr unsigned MASK = WCfg::LIST - 1;
  if ((h.bits & kWHitBits) == 0u) {
    const uint2 en = ring[(h.tail & MASK) * 32u + (threadIdx.x & 31)];
    ++h.tail;
    h.base = en.x;
    h.bits = en.y;
  }
  const int b = __ffs(h.bits) - 1;  // the lowest set bit lies in the (non-empty) mask
  h.bits &= h.bits - 1u;
  j = 2 * (int)h.base + b;
  sh = h.bits >> kWShift;
}

// Evaluation of up to `most` hits of every lane: the warp iterates up to the largest count (lanes
// with fewer idle), each lane takes its next hit (the lowest bit of its current entry, the next
// entry of its ring when that one is spent), loads the neighbour's records and calls
// body.pair_at with both ends in the pair's periodic image.  Returns the hits this lane
// evaluated.
template <int D, bool EX0, bool EX1, class Body>
__device__ __forceinline__ int warp_drain(const float* L, const Arrays& a, const float4* __restrict__ extra0,
                                          const float* __restrict__ extra1, const uint2* ring, WHits& h, int most,
                                          const float* xt, Body& body) {
  const int mine = min(h.pend, most);
  const int m = (int)__reduce_max_sync(kFull, (unsigned)mine);
#if SPH_W_DRAIN2
  // two hits per iteration: both neighbours' records are requested before either is evaluated
  for (int e = 0; e < m; e += 2) {
    const bool oa = e < mine, ob = e + 1 < mine;
    int ja = 0, jb = 0;
    uint32_t sa = 0u, sb = 0u;
    if (oa) warp_pop_hit(ring, h, ja, sa);
    if (ob) warp_pop_hit(ring, h, jb, sb);
    const PD<D> pa = load_pd<D>(a, ja), pb = load_pd<D>(a, jb);  // index 0 for a lane without the hit
#if SPH_W_PAIR2
    if constexpr (Body::kPaired) {
      if (oa) {  // b rides along (dropped when this lane has no second hit)
        float xa[D], xb[D];
        PD<D> qa = pa, qb = pb;
#pragma unroll
        for (int q = 0; q < D; ++q) xa[q] = xb[q] = xt[q];
        if (sa | sb) {  // periodic images (particles near the box faces only)
#pragma unroll
          for (int q = 0; q < D; ++q) {
            if ((sa >> (3 + q)) & 1u) xa[q] -= L[q];
            if ((sa >> q) & 1u) qa.x[q] -= L[q];
            if ((sb >> (3 + q)) & 1u) xb[q] -= L[q];
            if ((sb >> q) & 1u) qb.x[q] -= L[q];
          }
        }
        body.pair_at2(xa, qa, xb, qb, ob);
      }
      continue;
    }
#endif
    if (oa) warp_eval_hit<D, EX0, EX1>(L, a, extra0, extra1, ja, sa, pa, xt, body);
    if (ob) warp_eval_hit<D, EX0, EX1>(L, a, extra0, extra1, jb, sb, pb, xt, body);
  }
#else
  for (int e = 0; e < m; ++e) {
    if (e < mine) {
      int j;
      uint32_t sh;
      warp_pop_hit(ring, h, j, sh);
      warp_eval_hit<D, EX0, EX1>(L, a, extra0, extra1, j, sh, load_pd<D>(a, j), xt, body);
    }
  }
#endif
  h.pend -= mine;
  return mine;
}

// Test the candidates [g0, g1) of one run (per lane: its own run) against this lane's target,
// UNROLL at a time: the positions come as pairs (PXY[p] = (x_2p, x_2p+1, y_2p, y_2p+1), PZ[p] =
// (z_2p, z_2p+1), packed before the launch) and the squared distances of a pair are formed with
// the paired FP32 instructions.  nt: minus the target's coordinates in the run's image plus the
// shift taken off the candidates (the test's rounding near |r| = H does not matter: W and grad W
// vanish there; the evaluation forms the pair's separation from exactly shifted operands).  A
// step with hits appends one ring entry (its first pair, its hit mask and the run's shifts
// `tag`).  The loop is warp-uniform (up to the longest run of the warp); the candidates of a
// step that lie outside the lane's run (the one before g0 when g0 is odd, those past g1, and
// every one of a lane past its run, which re-reads its last pairs) are masked out.  ZERO_OK: a
// pair at zero distance (the target itself) is harmless to the pass, so only r^2 < H^2 is
// tested; the caller discounts the target from the pair count.
template <int D, bool ZERO_OK, class Drain>
__device__ __forceinline__ void warp_scan_run(const float4* __restrict__ PXY, const float2* __restrict__ PZ, int g0,
                                              int g1, float2 ntx, float2 nty, float2 ntz, uint32_t tag, float H2,
                                              uint2* ring, WHits& h, Drain& drain) {
  constexpr int U = WCfg::UNROLL / 2;  // pairs per step
  constexpr unsigned FULLM = (1u << (2 * U)) - 1u;
  constexpr unsigned MASK = WCfg::LIST - 1;
  const int lane = threadIdx.x & 31;
  const int len = max(g1 - g0, 0);
  const int pa = g0 >> 1;
  const int odd = g0 & 1;
  const int np = len > 0 ? ((g1 + 1) >> 1) - pa : 0;
  const int mlen = (int)__reduce_max_sync(kFull, (unsigned)np);
  const int last = max(np - 1, 0);
  unsigned fm = odd ? FULLM - 1u : FULLM;  // the first step's candidate 2 pa = g0 - 1 is not in the run
  for (int it = 0; it < mlen; it += U) {
    if (__any_sync(kFull, h.head - h.tail >= (unsigned)WCfg::LIST)) drain();
    const int q0 = pa + min(it, last);
    float4 Q[U];
    float2 Z[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      Q[u] = __ldg(PXY + q0 + u);
      Z[u] = D == 3 ? __ldg(PZ + q0 + u) : make_float2(0.f, 0.f);
    }
    unsigned hm = 0u;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float2 dx = __fadd2_rn(make_float2(Q[u].x, Q[u].y), ntx);
      const float2 dy = __fadd2_rn(make_float2(Q[u].z, Q[u].w), nty);
      float2 r2 = __ffma2_rn(dy, dy, __fmul2_rn(dx, dx));
      if (D == 3) {
        const float2 dz = __fadd2_rn(Z[u], ntz);
        r2 = __ffma2_rn(dz, dz, r2);
      }
      hm |= ((r2.x < H2 && (ZERO_OK || r2.x > 0.f)) ? 1u : 0u) << (2 * u);
      hm |= ((r2.y < H2 && (ZERO_OK || r2.y > 0.f)) ? 1u : 0u) << (2 * u + 1);
    }
    // candidates of the step still in the run: 2 (pa + it) + k < g1
    const int rem = len + odd - 2 * it;
    const unsigned vm = rem >= 2 * U ? FULLM : (rem > 0 ? (1u << rem) - 1u : 0u);
    const unsigned msk = hm & vm & fm;
    fm = FULLM;
    if (msk) {
      ring[(h.head & MASK) * 32u + lane] = make_uint2((uint32_t)(pa + it), msk | tag);
      ++h.head;
      h.pend += __popc(msk);
    }
  }
}

// One tile on one warp: per-lane target set-up, the runs of every neighbour line, the tests, the
// evaluation of the rings and the pass's epilogue.  Returns the pairs this lane evaluated (the
// target itself not counted).
template <int D, bool ZERO_OK, bool EX0, bool EX1, class Pass>
__device__ __forceinline__ int warp_tile_task(const TravArgs& t, const Tile& T, uint2* ring,
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
  int cx = 0;
  if (valid) {
    active = pass.init(body, s, i, tv);
    const float4 A = __ldg(t.a.A + i);
    xt[0] = A.x; xt[1] = A.y; xt[2] = D == 3 ? A.z : 0.f;
    const int c[3] = {(int)(t.keys[i] >> t.kshift) - (s.cell_base + (T.cz * s.n[1] + T.cy) * s.n[0]), T.cy, T.cz};
    cx = c[0];
#pragma unroll
    for (int q = 0; q < D; ++q) {  // squared distances to the own cell's faces (0 past a face)
      const float lo = s.lo[q] + s.cs[q] * (float)c[q];
      const float a0 = fmaxf(xt[q] - lo, 0.f), a1 = fmaxf(lo + s.cs[q] - xt[q], 0.f);
      fl[q] = a0 * a0;
      fh[q] = a1 * a1;
    }
  }
  const float L[3] = {s.L[0], s.L[1], D == 3 ? s.L[2] : 0.f};
  const float H2 = s.H2, R2 = s.trimR2;
  const int nx = s.n[0];
  const bool px = s.periodic_mask & 1;
  const float4* PXY = reinterpret_cast<const float4*>(t.packed);
  const float2* PZ = reinterpret_cast<const float2*>(t.packed + 4 * warp_pairs_stride(t.N));
  WHits h;
  int np = 0;
  auto drain = [&]() { np += warp_drain<D, EX0, EX1>(L, t.a, extra0, extra1, ring, h, WCfg::EVAL, xt, body); };
  for (int l = 0; l < NL; ++l) {
    float tsh[2], csh[2];
    const int lc = tile_line<D>(s, T, l, tsh, csh);  // uniform over the warp
    if (lc < 0) continue;
    const int dy = (D == 2) ? l - 1 : l % 3 - 1;
    const int dz = (D == 2) ? 0 : l / 3 - 1;
    // the lane's runs of this line: the left image (the line's upper end, shifted down by L), the
    // in-box range and the right image (the line's lower end; the target takes off L)
    int lg0 = 0, lg1 = 0, mg0 = 0, mg1 = 0, rg0 = 0, rg1 = 0;
    const float dyz = (dy < 0 ? fl[1] : dy > 0 ? fh[1] : 0.f) + (dz < 0 ? fl[2] : dz > 0 ? fh[2] : 0.f);
    if (active && dyz < R2) {
      if (t.bin_off) {
        // cells ordered by x sub-bin: the window of the reach's chord, [x - c, x + c] with c^2 =
        // R^2 - dyz, in sub-bins of the line (the same monotone function the keys used)
        constexpr int B = kXBins;
        const int nb = nx * B;
        const float c = sqrtf(R2 - dyz);
        int bl = line_xbin<B>(s, xt[0] - c), bh = line_xbin<B>(s, xt[0] + c);
        bl = px ? max(bl, -nb) : max(bl, 0);
        bh = px ? min(bh, 2 * nb - 1) : min(bh, nb - 1);
        const int* bo = t.bin_off + (size_t)lc * B;
        if (bl < 0) { lg0 = bo[bl + nb]; lg1 = bo[nb]; }
        const int b0 = max(bl, 0), b1 = min(bh, nb - 1);
        if (b0 <= b1) { mg0 = bo[b0]; mg1 = bo[b1 + 1]; }
        if (bh >= nb) { rg0 = bo[0]; rg1 = bo[bh - nb + 1]; }
      } else {
        // whole cells: the columns [clo, chi) the face-distance test keeps
        int clo = cx - (fl[0] + dyz < R2 ? 1 : 0);
        int chi = cx + 1 + (fh[0] + dyz < R2 ? 1 : 0);
        if (!px) {
          clo = max(clo, 0);
          chi = min(chi, nx);
        }
        if (clo < 0) { lg0 = t.cell_off[lc + nx - 1]; lg1 = t.cell_off[lc + nx]; }
        const int c0 = max(clo, 0), c1 = min(chi, nx);
        if (c0 < c1) { mg0 = t.cell_off[lc + c0]; mg1 = t.cell_off[lc + c1]; }
        if (chi > nx) { rg0 = t.cell_off[lc]; rg1 = t.cell_off[lc + 1]; }
      }
    }
    const bool lft = __any_sync(kFull, lg0 < lg1), mid = __any_sync(kFull, mg0 < mg1),
               rgt = __any_sync(kFull, rg0 < rg1);
    if (!(lft || mid || rgt)) continue;  // (lanes of wall targets walk nothing)
    // the line's image on y and z: the target takes off L (upper) or the records do (lower)
    const float tl[3] = {xt[0], tsh[0] != 0.f ? xt[1] - L[1] : xt[1], (D == 3 && tsh[1] != 0.f) ? xt[2] - L[2] : xt[2]};
    const float sh[3] = {0.f, -csh[0], D == 3 ? -csh[1] : 0.f};
    const uint32_t tag = (tsh[0] != 0.f ? 1u << (kWShift + 4) : 0u) | (D == 3 && tsh[1] != 0.f ? 1u << (kWShift + 5) : 0u) |
                         (csh[0] != 0.f ? 1u << (kWShift + 1) : 0u) | (D == 3 && csh[1] != 0.f ? 1u << (kWShift + 2) : 0u);
    const float2 nty = make_float2(-(tl[1] + sh[1]), -(tl[1] + sh[1]));
    const float2 ntz = make_float2(-(tl[2] + sh[2]), -(tl[2] + sh[2]));
    if (lft) {
      const float nx0 = -(tl[0] + L[0]);
      warp_scan_run<D, ZERO_OK>(PXY, PZ, lg0, lg1, make_float2(nx0, nx0), nty, ntz, tag | (1u << kWShift), H2, ring,
                                h, drain);
    }
    if (mid) warp_scan_run<D, ZERO_OK>(PXY, PZ, mg0, mg1, make_float2(-tl[0], -tl[0]), nty, ntz, tag, H2, ring, h, drain);
    if (rgt) {
      const float txr = -(xt[0] - L[0]);
      warp_scan_run<D, ZERO_OK>(PXY, PZ, rg0, rg1, make_float2(txr, txr), nty, ntz, tag | (1u << (kWShift + 3)), H2,
                                ring, h, drain);
    }
  }
  while (__any_sync(kFull, h.pend > 0)) drain();
  if (ZERO_OK && active) --np;  // the target found itself
  body.template reduce<1>();
  if (valid) pass.finish(body, s, i, tv);
  return np;
}

// Skeleton of a warp-traversal launch: tiles are handed out in launch order from the launch's tile
// counter, so the warps in flight walk a narrow front of consecutive tiles (a few planes of cell
// lines), whose neighbour lines stay in L2 (splitting the tiles into one contiguous range per CTA,
// which spreads the warps over the whole domain, made the 128^3 sweep 5 % slower).  The CTA ends
// as the staged launches do (end_tiles in sph_passes.cu: partial results, pair count, counters
// reset by the last CTA).
//
// With SPH_W_CHUNK > 0 (the default) the counter hands out chunks of CHUNK consecutive tiles to a
// CTA, and the CTA's warps take the chunk's tiles one at a time as they free up, so the warps that
// share an SM's L1 work on neighbouring tiles of one cell line, whose neighbour lines largely
// coincide (with one warp per claim the warps of an SM held tiles about 148 apart).  A warp that
// takes the first tile of a chunk claims the chunk and publishes its index in a small ring of
// slots in shared memory; one that takes a later tile waits (bounded) for that slot.  A slot is
// reused by the chunk SLOTS chunks later, which needs SLOTS x CHUNK further claims by the other
// warps of the CTA, each after a whole tile, while the waiting warp polls a flag that the
// claimant sets right after one global atomic; a wait that runs out sets status bit 1.
constexpr long long kChunkSpins = 1LL << 20;

template <int D, bool ZERO_OK, bool EX0, bool EX1, class Pass, class End>
__device__ __forceinline__ void run_warp_tiles(const TravArgs& t, const Tile* __restrict__ tiles,
                                               const int* __restrict__ ntiles, const float4* __restrict__ extra0,
                                               const float* __restrict__ extra1, Pass& pass, End end) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5;
  uint2* ring = reinterpret_cast<uint2*>(smraw) + (size_t)warp * WCfg::LIST * 32;
  const int nt = *ntiles;
  long long pairs = 0;
#if SPH_W_CHUNK > 0
  constexpr int CH = SPH_W_CHUNK, SLOTS = 8;
  __shared__ int s_claim;         // tiles this CTA has taken so far
  __shared__ int s_chunk[SLOTS];  // the launch's index of the CTA's c-th chunk, in slot c % SLOTS
  __shared__ int s_ready[SLOTS];  // c + 1 once slot c % SLOTS holds the c-th chunk
  if (threadIdx.x == 0) s_claim = 0;
  if (threadIdx.x < SLOTS) s_ready[threadIdx.x] = 0;
  __syncthreads();
#endif
  for (;;) {
    int nxt = 0;
    if ((threadIdx.x & 31) == 0) {
#if SPH_W_CHUNK > 0
      const int k = atomicAdd(&s_claim, 1);
      const int c = k / CH, pos = k - c * CH, slot = c % SLOTS;
      int g;
      if (pos == 0) {
        g = atomicAdd(t.tile_ctr, 1);
        s_chunk[slot] = g;
        __threadfence_block();
        atomicExch(&s_ready[slot], c + 1);
      } else {
        long long it = 0;
        while (*(volatile int*)&s_ready[slot] != c + 1 && ++it <= kChunkSpins) __nanosleep(16);
        __threadfence_block();
        if (it > kChunkSpins) {
          atomicOr(t.status, 2);
          g = nt;  // gives up: no further tile for this warp
        } else {
          g = *(volatile int*)&s_chunk[slot];
        }
      }
      nxt = g >= nt ? nt : g * CH + pos;
#else
      nxt = atomicAdd(t.tile_ctr, 1);
#endif
    }
    const int ti = __shfl_sync(kFull, nxt, 0);
    if (ti >= nt) break;
    const Tile T = tiles[ti];
    pairs += warp_tile_task<D, ZERO_OK, EX0, EX1>(t, T, ring, extra0, extra1, pass);
  }
  end(pairs);
}

}  // namespace sph
