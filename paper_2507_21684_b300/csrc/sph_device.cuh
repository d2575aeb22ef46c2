// Device-side building blocks of the B300 WCSPH library: per-scene parameters, particle
// record layouts, the Wendland kernels, and the warp-cooperative cell traversal that every
// neighbour pass (walls, density, fused sweep, adjoint sweep, pair export) shares.
//
// Data layout (HBM, all arrays in sorted cell order, one contiguous range per scene):
//   hot records, read for every neighbour pair:
//     2D  A = (x_h, y_h, vx, vy)      B = (rho, p, V = m/rho, +-m)         (float4 each)
//     3D  A = (x_h, y_h, z_h, V)      B = (vx, vy, vz, p)   C = (rho, +-m)  (float4, float4, float2)
//   cold records, read once per particle and step (the integrated state in double-single form,
//   value = hi + lo with |lo| <= ulp(hi)/2, so rounding of the per-step increment does not
//   accumulate over long rollouts):
//     2D  X = (x_hi, y_hi, x_lo, y_lo)   O = (o_x, o_y, rho_lo, -)
//     3D  X = (x_hi, y_hi, z_hi, rho_lo) XL = (x_lo, y_lo, z_lo, -)  O = (o_x, o_y, o_z, -)
//   meta = (original index | wall bit, scene index)
// x_h = x - o is the position folded into the primary box at the last rebuild (o = L k for an
// integer k per periodic axis), so a candidate range that crosses a periodic edge needs one
// uniform shift instead of a per-pair minimum image (Sec. 3.2, App. B).
// The sign of the mass field marks wall particles (negative = wall).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sph {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kWallBit = 0x80000000u;
constexpr int kListCap = 48;  // neighbour-list entries per lane between drains

// Per-scene parameters as the kernels read them (one entry per packed scene).
struct DevSeg {
  int dim, kernel, density_mode, periodic_mask;
  int n[3];          // cells per axis
  int cell_base;     // first global cell id of this scene
  int p0, p1;        // particle range in the packed arrays
  int nf;            // fluid particles (original indices < nf are fluid)
  int pad0;
  float L[3], lo[3], invL[3];
  double lo_d[3], L_d[3], cs_d[3];
  float H, H2, invH, dt, rho0, c0, gamma, B;
  float Cv, dCv_dnu, Cdel, eH2;
  float Kg;          // grad W = Kg * g~(q) * r   (g~ = poly part of w'(q)/q)
  float Kw;          // W = Kw * w(q)
  float Kh;          // Hessian radial factor constant: d(g)/dr = Kh * h~(q) * r
  float g[3];
  float band_lo, band_hi;  // FP32 r^2 guard band for the exact pair predicate
  double H2_d;
  float nu, pad1;
};

// ---------------------------------------------------------------- Wendland kernels
// Written as W = Kw * w(q), grad_i W_ij = Kg * gt(q) * r_ij, with gt = w'(q)/q divided by its
// leading constant, so no division by |r| is needed (App. A.1 definition of grad W).
//   C4: w = (1-q)^6 (1 + 6q + 35/3 q^2),  w'/q = -(56/3)(1-q)^5 (1+5q),  (w'/q)'/q = 560 (1-q)^4
//   C2: w = (1-q)^4 (1 + 4q),             w'/q = -20 (1-q)^3,           (w'/q)'/q = 60 (1-q)^2 / q
template <int KERN>
__device__ __forceinline__ float kern_w(float q) {
  float om = 1.f - q, om2 = om * om;
  if (KERN == 0) return om2 * om2 * om2 * fmaf(q, fmaf(q, 35.f / 3.f, 6.f), 1.f);
  return om2 * om2 * fmaf(4.f, q, 1.f);
}
template <int KERN>
__device__ __forceinline__ float kern_gt(float q) {  // Kg carries -(56/3) or -20
  float om = 1.f - q, om2 = om * om;
  if (KERN == 0) return om2 * om2 * om * fmaf(5.f, q, 1.f);
  return om2 * om;
}
template <int KERN>
__device__ __forceinline__ float kern_ht(float q) {  // Kh carries 560/H^2 or 60/H^2
  float om = 1.f - q, om2 = om * om;
  if (KERN == 0) return om2 * om2;
  return q > 0.f ? om2 / q : 0.f;
}

// Tait equation of state p = B[(rho/rho0)^gamma - 1], evaluated as B expm1(gamma log1p(e))
// with e = (rho - rho0)/rho0 so that small compressions keep full relative accuracy.
__device__ __forceinline__ float tait_p(const DevSeg& s, float rho) {
  float e = (rho - s.rho0) / s.rho0;
  return s.B * expm1f(s.gamma * log1pf(e));
}
// dp/drho = gamma (p + B) / rho
__device__ __forceinline__ float tait_slope(const DevSeg& s, float rho, float p) {
  return s.gamma * (p + s.B) / rho;
}
__device__ __forceinline__ float tait_rho(const DevSeg& s, float p) {
  return s.rho0 * expf(log1pf(p / s.B) / s.gamma);
}

// ---------------------------------------------------------------- particle arrays
struct Arrays {
  float4* A;
  float4* B;
  float2* C;      // 3D only
  float4* X;      // unwrapped position, high parts (+ low parts in 2D, rho_lo in 3D)
  float4* XL;     // 3D only: low parts of the position
  float4* O;      // wrap offset (+ rho_lo in 2D)
  uint2* meta;
};

// Cold (integrated) state of one particle: position and density in double-single form.
struct Cold {
  float hi[3], lo[3], off[3];
  float rlo;
};

template <int D>
__device__ __forceinline__ Cold load_cold(const Arrays& a, int i) {
  Cold c;
  float4 X = a.X[i], O = a.O[i];
  c.off[0] = O.x; c.off[1] = O.y; c.off[2] = O.z;
  if (D == 2) {
    c.hi[0] = X.x; c.hi[1] = X.y; c.hi[2] = 0.f;
    c.lo[0] = X.z; c.lo[1] = X.w; c.lo[2] = 0.f;
    c.rlo = O.z;
    c.off[2] = 0.f;
  } else {
    float4 L = a.XL[i];
    c.hi[0] = X.x; c.hi[1] = X.y; c.hi[2] = X.z;
    c.lo[0] = L.x; c.lo[1] = L.y; c.lo[2] = L.z;
    c.rlo = X.w;
  }
  return c;
}

template <int D>
__device__ __forceinline__ void store_cold(const Arrays& a, int i, const Cold& c) {
  if (D == 2) {
    a.X[i] = make_float4(c.hi[0], c.hi[1], c.lo[0], c.lo[1]);
    a.O[i] = make_float4(c.off[0], c.off[1], c.rlo, 0.f);
  } else {
    a.X[i] = make_float4(c.hi[0], c.hi[1], c.hi[2], c.rlo);
    a.XL[i] = make_float4(c.lo[0], c.lo[1], c.lo[2], 0.f);
    a.O[i] = make_float4(c.off[0], c.off[1], c.off[2], 0.f);
  }
}

// hi + lo <- hi + lo + d  (TwoSum, then renormalise; explicit roundings, never contracted)
__device__ __forceinline__ void ds_add(float& hi, float& lo, float d) {
  float s = __fadd_rn(hi, d);
  float bp = __fsub_rn(s, hi);
  float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(d, bp));
  float l = __fadd_rn(lo, e);
  float h = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(h, s));
  hi = h;
}

template <int D>
struct PosT;
template <>
struct PosT<2> {
  float x[2];
};
template <>
struct PosT<3> {
  float x[3];
};

template <int D>
__device__ __forceinline__ void load_pos(const float4* __restrict__ A, int j, float* p) {
  if (D == 2) {
    float2 t = __ldg(reinterpret_cast<const float2*>(A) + 2 * j);
    p[0] = t.x;
    p[1] = t.y;
  } else {
    float4 t = __ldg(A + j);
    p[0] = t.x;
    p[1] = t.y;
    p[2] = t.z;
  }
}

// Exact neighbour predicate on the unwrapped float32 positions: |mimg(x_i - x_j)|^2 < H^2
// with every operation in FP64 and rounded as written (no contraction).
template <int D>
__device__ bool exact_pair(const DevSeg& s, const Arrays& arr, int i, int j) {
  Cold a = load_cold<D>(arr, i), b = load_cold<D>(arr, j);
  double d2 = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double xi = __dadd_rn((double)a.hi[k], (double)a.lo[k]);
    double xj = __dadd_rn((double)b.hi[k], (double)b.lo[k]);
    double dx = __dsub_rn(xi, xj);
    if ((s.periodic_mask >> k) & 1) {
      double n = rint(__ddiv_rn(dx, s.L_d[k]));
      dx = __dsub_rn(dx, __dmul_rn(s.L_d[k], n));
    }
    d2 = __dadd_rn(d2, __dmul_rn(dx, dx));
  }
  return d2 < s.H2_d;
}

// ---------------------------------------------------------------- traversal
// Cell coordinates of a global key inside its scene.
__device__ __forceinline__ void key_coords(const DevSeg& s, uint32_t key, int* c) {
  int local = (int)key - s.cell_base;
  c[0] = local % s.n[0];
  int rest = local / s.n[0];
  c[1] = rest % s.n[1];
  c[2] = rest / s.n[1];
}

// Warp-cooperative traversal.  A warp owns 32 consecutive sorted particles.  Lanes that sit
// in the same cell line (same scene, same y[,z] cell row) form a group; for each group the
// warp walks the union of the neighbouring lines' column ranges [cx_min-1, cx_max+1] once,
// every lane testing the same candidate (broadcast loads).  In-radius candidates go to a
// per-lane list in shared memory; when any list fills up, each lane evaluates its own list
// (Body::pair).  Candidates outside a lane's own 3^d cells fail the cut-off test, so the
// union is exact.  With EXACT the FP32 test is confirmed in FP64 inside a guard band
// (bit-exact pair sets); otherwise r^2 < H^2 in FP32 decides (pairs that differ lie within
// a relative 1e-4 of the cut-off, where W and its derivatives vanish to O(1e-13) or less).
template <int D, bool EXACT, class Body>
__device__ __forceinline__ void traverse(const DevSeg* __restrict__ segs, const float4* __restrict__ A,
                                         const Arrays& arr, const uint32_t* __restrict__ keys,
                                         const int* __restrict__ cell_off, int i, bool active, int seg,
                                         uint32_t* __restrict__ list, Body& body) {
  const int lane = threadIdx.x & 31;
  float xi[3] = {0.f, 0.f, 0.f};
  int ci[3] = {0, 0, 0};
  uint32_t line_id = 0xffffffffu;
  if (active) {
    load_pos<D>(A, i, xi);
    key_coords(segs[seg], keys[i], ci);
    line_id = ((uint32_t)seg << 20) | (uint32_t)(ci[1] + ci[2] * segs[seg].n[1]);
  }
  uint32_t pending = __ballot_sync(kFull, active);
  int cnt = 0;
  auto drain = [&]() {
    for (int t = 0; t < cnt; ++t) body.pair(list[t * 32]);
    cnt = 0;
  };
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const uint32_t gl = __shfl_sync(kFull, line_id, leader);
    const bool mine = active && line_id == gl;
    pending &= ~__ballot_sync(kFull, mine);
    const int gseg = __shfl_sync(kFull, seg, leader);
    const DevSeg& s = segs[gseg];
    const int cxmin = __reduce_min_sync(kFull, mine ? ci[0] : 0x7fffffff);
    const int cxmax = __reduce_max_sync(kFull, mine ? ci[0] : -1);
    const int gy = __shfl_sync(kFull, ci[1], leader);
    const int gz = __shfl_sync(kFull, ci[2], leader);
    const float H2 = s.H2;
    const int nx = s.n[0], ny = s.n[1], nz = s.n[2];
    const bool perx = s.periodic_mask & 1, pery = (s.periodic_mask >> 1) & 1, perz = (s.periodic_mask >> 2) & 1;
    const int zlo = (D == 3) ? -1 : 0, zhi = (D == 3) ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
      int cz = gz + dz;
      float sz = 0.f;
      if (D == 3) {
        if (cz < 0) { if (!perz) continue; cz += nz; sz = -s.L[2]; }
        else if (cz >= nz) { if (!perz) continue; cz -= nz; sz = s.L[2]; }
      }
      for (int dy = -1; dy <= 1; ++dy) {
        int cy = gy + dy;
        float sy = 0.f;
        if (cy < 0) { if (!pery) continue; cy += ny; sy = -s.L[1]; }
        else if (cy >= ny) { if (!pery) continue; cy -= ny; sy = s.L[1]; }
        const int row = s.cell_base + (cz * ny + cy) * nx;
        // up to three column ranges: left wrap, main, right wrap
        for (int part = 0; part < 3; ++part) {
          int c0, c1;
          float sx = 0.f;
          if (part == 0) {
            if (!(perx && cxmin - 1 < 0)) continue;
            c0 = c1 = nx - 1;
            sx = -s.L[0];
          } else if (part == 1) {
            c0 = max(cxmin - 1, 0);
            c1 = min(cxmax + 1, nx - 1);
          } else {
            if (!(perx && cxmax + 1 > nx - 1)) continue;
            c0 = c1 = 0;
            sx = s.L[0];
          }
          // cell offsets are monotone by construction; the clamp keeps every read in bounds
          const int jb = max(cell_off[row + c0], s.p0), je = min(cell_off[row + c1 + 1], s.p1);
          const float px = xi[0] - sx, py = xi[1] - sy, pz = xi[2] - sz;
          for (int j0 = jb; j0 < je; j0 += 8) {
            if (__any_sync(kFull, cnt > kListCap - 8)) drain();
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int j = j0 + u;
              if (j < je) {
                float pj[3];
                load_pos<D>(A, j, pj);
                float dx = px - pj[0], dy2 = py - pj[1];
                float r2 = fmaf(dy2, dy2, dx * dx);
                if (D == 3) {
                  float dz2 = pz - pj[2];
                  r2 = fmaf(dz2, dz2, r2);
                }
                bool in;
                if (EXACT) {
                  in = mine && j != i && r2 < s.band_hi;
                  if (in && r2 >= s.band_lo) in = exact_pair<D>(s, arr, i, j);
                } else {
                  in = mine && j != i && r2 < H2;
                }
                if (in) {
                  list[cnt * 32] = (uint32_t)j;
                  ++cnt;
                }
              }
            }
          }
        }
      }
    }
  }
  drain();
  (void)lane;
}

// Deterministic block reduction of a double (fixed shuffle tree, then warps in order).
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  }
  __syncthreads();
  return t;
}

}  // namespace sph
