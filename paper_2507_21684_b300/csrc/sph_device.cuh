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
//     2D  X = (x_hi, y_hi, x_lo, y_lo)   O = (o_x, o_y, rho_lo, H_i)
//     3D  X = (x_hi, y_hi, z_hi, rho_lo) XL = (x_lo, y_lo, z_lo, -)  O = (o_x, o_y, o_z, H_i)
//     (H_i: per-particle support radius of the variable-support queries, 0 = the scene's H)
//   meta = (original index | wall bit, scene index)
// x_h = x - o is the position folded into the primary box at the last rebuild (o = L k for an
// integer k per periodic axis), so a candidate range that crosses a periodic edge needs one
// uniform shift instead of a per-pair minimum image (Sec. 3.2, App. B).
// The sign of the mass field marks wall particles (negative = wall).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sph {

// Programmatic dependent launch: a kernel launched with PdlLaunch may start while the kernel
// before it in its stream still runs (the step's first neighbour pass after the cell rebuild
// launch, which allows it at its start; the kernels of an adjoint step after one another); it
// waits here, before its first memory access, until that kernel has completed and its writes are
// visible.  Without the launch attribute it returns at once.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch configuration of a kernel that may start before the previous kernel in its stream has
// finished (it calls wait_prior_grid first).
struct PdlLaunch {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  PdlLaunch(dim3 grid, int threads, size_t smem, cudaStream_t st) {
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
};


constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kWallBit = 0x80000000u;

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
  float nu, shiftC;         // shiftC = C H^2 of the particle shifting (0: off)
  float cs[3];             // cell edge (FP32) of the folded frame
  float trimR2;            // squared reach used to skip neighbour cells (H + skin/2 + margins)
  float invcs[3];          // FP32 reciprocal cell edge (fast path of the cell key)
  float inv_half2;         // 1 / (skin/2 - margin)^2: displacement scale of the rebuild check (0: no skin)
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
  float aux;  // per-particle support radius of the variable-support queries (0: the scene's H)
};

template <int D>
__device__ __forceinline__ Cold load_cold(const Arrays& a, int i) {
  Cold c;
  float4 X = a.X[i], O = a.O[i];
  c.off[0] = O.x; c.off[1] = O.y; c.off[2] = O.z;
  c.aux = O.w;
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
    a.O[i] = make_float4(c.off[0], c.off[1], c.rlo, c.aux);
  } else {
    a.X[i] = make_float4(c.hi[0], c.hi[1], c.hi[2], c.rlo);
    a.XL[i] = make_float4(c.lo[0], c.lo[1], c.lo[2], 0.f);
    a.O[i] = make_float4(c.off[0], c.off[1], c.off[2], c.aux);
  }
}

// Compensated accumulation: hi + lo gathers the terms d with hi the rounded running sum and lo
// the sum of the exact rounding errors (TwoSum; explicit roundings, never contracted).  For the
// sums of non-negative kernel terms this is as accurate as an FP64 sum, in FP32 arithmetic.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float d) {
  const float s = __fadd_rn(hi, d);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(d, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}
// (hi, lo) += (oh, ol): the same for a partial sum of another lane (exact error of the hi parts;
// symmetric in its two operands, so a butterfly gives every lane the same result)
__device__ __forceinline__ void two_sum_merge(float& hi, float& lo, float oh, float ol) {
  const float s = __fadd_rn(hi, oh);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(oh, bp));
  hi = s;
  lo = __fadd_rn(__fadd_rn(lo, ol), e);
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

// The same FP64 squared distance, returned (for per-pair radii).
template <int D>
__device__ double exact_d2(const DevSeg& s, const Arrays& arr, int i, int j) {
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
  return d2;
}

// ---------------------------------------------------------------- particle records
template <int D>
struct PD {
  float x[D], v[D], rho, p, V, m;
};

// (COH: through L2 only, for records another CTA of the same launch may have rewritten)
template <int D, bool COH = false>
__device__ __forceinline__ PD<D> load_pd(const Arrays& a, int j) {
  PD<D> r;
  float4 A = COH ? __ldcg(a.A + j) : __ldg(a.A + j), B = COH ? __ldcg(a.B + j) : __ldg(a.B + j);
  if (D == 2) {
    r.x[0] = A.x; r.x[1] = A.y; r.v[0] = A.z; r.v[1] = A.w;
    r.rho = B.x; r.p = B.y; r.V = B.z; r.m = B.w;
  } else {
    float2 C = COH ? __ldcg(a.C + j) : __ldg(a.C + j);
    r.x[0] = A.x; r.x[1] = A.y; r.x[2] = A.z; r.V = A.w;
    r.v[0] = B.x; r.v[1] = B.y; r.v[2] = B.z; r.p = B.w;
    r.rho = C.x; r.m = C.y;
  }
  return r;
}

// Same as load_pd through plain loads (for Arrays views of shared memory).
template <int D>
__device__ __forceinline__ PD<D> load_pd_plain(const Arrays& a, int j) {
  PD<D> r;
  const float4 A = a.A[j], B = a.B[j];
  if (D == 2) {
    r.x[0] = A.x; r.x[1] = A.y; r.v[0] = A.z; r.v[1] = A.w;
    r.rho = B.x; r.p = B.y; r.V = B.z; r.m = B.w;
  } else {
    const float2 C = a.C[j];
    r.x[0] = A.x; r.x[1] = A.y; r.x[2] = A.z; r.V = A.w;
    r.v[0] = B.x; r.v[1] = B.y; r.v[2] = B.z; r.p = B.w;
    r.rho = C.x; r.m = C.y;
  }
  return r;
}

template <int D>
__device__ __forceinline__ void store_pd(const Arrays& a, int j, const PD<D>& r) {
  if (D == 2) {
    a.A[j] = make_float4(r.x[0], r.x[1], r.v[0], r.v[1]);
    a.B[j] = make_float4(r.rho, r.p, r.V, r.m);
  } else {
    a.A[j] = make_float4(r.x[0], r.x[1], r.x[2], r.V);
    a.B[j] = make_float4(r.v[0], r.v[1], r.v[2], r.p);
    a.C[j] = make_float2(r.rho, r.m);
  }
}

// separation r = mimg(x_i - x_j) on folded positions.  Across a periodic edge the box length
// is taken off the coordinate near the upper edge first (x - L is exact there), so the image
// separation carries one rounding, as an interior one does.
template <int D>
__device__ __forceinline__ float separation(const DevSeg& s, const float* xi, const float* xj, float* r) {
  float r2 = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    float d = xi[k] - xj[k];
    if ((s.periodic_mask >> k) & 1) {
      const float hL = 0.5f * s.L[k];
      if (d > hL) d = (xi[k] - s.L[k]) - xj[k];
      else if (d < -hL) d = xi[k] - (xj[k] - s.L[k]);
    }
    r[k] = d;
    r2 = fmaf(d, d, r2);
  }
  return r2;
}

// r = x_i - x_j for positions already in the same periodic image
template <int D>
__device__ __forceinline__ float diff(const float* xi, const float* xj, float* r) {
  float r2 = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    r[k] = xi[k] - xj[k];
    r2 = fmaf(r[k], r[k], r2);
  }
  return r2;
}

__device__ __forceinline__ float safe_q(float r2, float invH) { return r2 * rsqrtf(fmaxf(r2, 1e-30f)) * invH; }

// ---------------------------------------------------------------- traversal
// Cell coordinates of a global key inside its scene.
__device__ __forceinline__ void key_coords(const DevSeg& s, uint32_t key, int* c) {
  int local = (int)key - s.cell_base;
  c[0] = local % s.n[0];
  int rest = local / s.n[0];
  c[1] = rest % s.n[1];
  c[2] = rest / s.n[1];
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

// Sub-bins of a cell along x (3D warp-per-tile sweep): the cell keys of such scenes carry the
// particle's sub-bin in their low kXShift bits (cell * kXBins + bin; 8 sub-bins), so the sort orders every
// cell by sub-bin and the sweep can walk x windows of a line instead of whole cells.
#ifndef SPH_W_XSHIFT
#define SPH_W_XSHIFT 3
#endif
constexpr int kXShift = SPH_W_XSHIFT;
constexpr int kXBins = 1 << kXShift;

// Sub-bin of a folded x coordinate along its cell line: floor((x - lo_box) / cell edge * B), the
// function the cell keys (sph_sort.cuh) and the warp-per-tile sweep's x windows share (monotone
// in x).
template <int B>
__device__ __forceinline__ int line_xbin(const DevSeg& s, float x) {
  return (int)floorf((x - s.lo[0]) * s.invcs[0] * (float)B);
}

// True when the FP32 estimate (hi - lo) / L of periodic axis q lies farther than a safety
// margin inside (0, 1), so that the FP64 fold floor((x - lo) / L) of x = hi + lo is 0 (the
// particle is in the primary box).  The margin 2^-18 (|hi| + |lo|) / L + 2^-18 exceeds the
// estimate's error (a few FP32 roundings and |lo part| <= 2^-24 |hi|) more than ten times.
__device__ __forceinline__ bool in_primary_box(const DevSeg& s, int q, float hi) {
  const float w = (hi - s.lo[q]) * s.invL[q];
  const float m = 0x1p-18f * fmaf(fabsf(hi) + fabsf(s.lo[q]), s.invL[q], 1.f);
  return w >= m && w <= 1.f - m;
}

}  // namespace sph
