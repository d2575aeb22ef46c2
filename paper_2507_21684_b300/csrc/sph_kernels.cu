// CUDA kernels of the WCSPH step (sm_103a).  One pass of the method is
//   cell keys -> stable LSD radix sort -> cell ranges -> permute  (neighbour search, App. B)
//   -> wall extrapolation -> density summation                     (Sec. 2.3, App. A.6)
//   -> fused sweep: continuity + delta diffusion, Tait pressure, viscosity, gravity,
//      kick-drift epilogue                                          (Sec. 2.3, Sec. 3.4)
// and the mirrored adjoint sweep of a step (Sec. 2.2, 3.3).
#include "sph_kernels.cuh"

namespace sph {

// ================================================================== neighbour search
// Cell key of every particle in the current storage order (P2: floor-modulo wrap on
// periodic axes, clamp on open axes; all in FP64 from the float32 unwrapped position).
template <int D>
__global__ void k_keys(const DevSeg* __restrict__ segs, int N, Arrays a, uint32_t* __restrict__ keys,
                       uint32_t* __restrict__ vals) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const DevSeg& s = segs[a.meta[i].y];
  Cold c = load_cold<D>(a, i);
  int cc3[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double x = __dadd_rn((double)c.hi[k], (double)c.lo[k]);
    double xw = x;
    if ((s.periodic_mask >> k) & 1) {
      double f = floor(__ddiv_rn(__dsub_rn(x, s.lo_d[k]), s.L_d[k]));
      xw = __dsub_rn(x, __dmul_rn(s.L_d[k], f));
    }
    double cc = floor(__ddiv_rn(__dsub_rn(xw, s.lo_d[k]), s.cs_d[k]));
    cc = fmin(fmax(cc, 0.0), (double)(s.n[k] - 1));
    cc3[k] = (int)cc;
  }
  keys[i] = (uint32_t)(s.cell_base + (cc3[2] * s.n[1] + cc3[1]) * s.n[0] + cc3[0]);
  vals[i] = (uint32_t)i;
}

// ---- stable LSD radix sort, 8-bit digits, 2048-key tiles ---------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortIPT = 8;
constexpr int kSortTile = kSortThreads * kSortIPT;

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys, int N, int shift,
                                                            uint32_t* __restrict__ hist, int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * kSortTile;
#pragma unroll
  for (int k = 0; k < kSortIPT; ++k) {
    int i = base + k * kSortThreads + threadIdx.x;
    if (i < N) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of n uint32 in place, 2048 per block; block totals to sums.
__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t* __restrict__ a, int n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t sh[2048];
  const int base = blockIdx.x * 2048;
  for (int k = threadIdx.x; k < 2048; k += 1024) sh[k] = (base + k < n) ? a[base + k] : 0u;
  __syncthreads();
  // Blelloch up-sweep / down-sweep
  for (int d = 1; d < 2048; d <<= 1) {
    int idx = (threadIdx.x + 1) * (d << 1) - 1;
    if (idx < 2048) sh[idx] += sh[idx - d];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (sums) sums[blockIdx.x] = sh[2047];
    sh[2047] = 0;
  }
  __syncthreads();
  for (int d = 1024; d >= 1; d >>= 1) {
    int idx = (threadIdx.x + 1) * (d << 1) - 1;
    if (idx < 2048) {
      uint32_t t = sh[idx - d];
      sh[idx - d] = sh[idx];
      sh[idx] += t;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < 2048; k += 1024)
    if (base + k < n) a[base + k] = sh[k];
}

__global__ void k_scan_add(uint32_t* __restrict__ a, int n, const uint32_t* __restrict__ sums) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += sums[i / 2048];
}

// Scatter with stable ranks: warp w owns the contiguous sub-tile [w*256, w*256+256) and walks
// it in 8 rounds of 32; within a round, equal digits are ranked by lane via match_any.
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint32_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                               int N, int shift, const uint32_t* __restrict__ hist,
                                                               int nblocks) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t cnt[W][257];
  __shared__ uint32_t goff[256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < W * 257; k += kSortThreads) (&cnt[0][0])[k] = 0;
  goff[threadIdx.x] = hist[threadIdx.x * nblocks + blockIdx.x];
  __syncthreads();
  uint32_t kk[kSortIPT], vv[kSortIPT], rk[kSortIPT];
  const int base = blockIdx.x * kSortTile + w * 32 * kSortIPT;
#pragma unroll
  for (int r = 0; r < kSortIPT; ++r) {
    int i = base + r * 32 + lane;
    bool ok = i < N;
    kk[r] = ok ? kin[i] : 0u;
    vv[r] = ok ? vin[i] : 0u;
    uint32_t dg = ok ? ((kk[r] >> shift) & 255u) : 256u;
    uint32_t peers = __match_any_sync(kFull, dg);
    uint32_t before = __popc(peers & ((1u << lane) - 1u));
    rk[r] = cnt[w][dg] + before;
    __syncwarp();
    if (before == 0) cnt[w][dg] += __popc(peers);
    __syncwarp();
    rk[r] |= dg << 20;  // keep the digit beside the warp-local rank (rank < 256 per warp)
  }
  __syncthreads();
  // exclusive prefix over warps for each digit (thread t handles digit t)
  {
    uint32_t run = 0;
    for (int q = 0; q < W; ++q) {
      uint32_t c = cnt[q][threadIdx.x];
      cnt[q][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortIPT; ++r) {
    uint32_t dg = rk[r] >> 20;
    if (dg < 256u) {
      uint32_t pos = goff[dg] + cnt[w][dg] + (rk[r] & 0xfffffu);
      kout[pos] = kk[r];
      vout[pos] = vv[r];
    }
  }
}

// CSR cell offsets: off[c] = first sorted index whose key >= c, for c in [0, C].
__global__ void k_cell_offsets(const uint32_t* __restrict__ keys, int N, int C, int* __restrict__ off) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > N) return;
  int lo = (k == 0) ? 0 : (int)keys[k - 1] + 1;
  int hi = (k < N) ? (int)keys[k] : C;
  for (int c = lo; c <= hi; ++c) off[c] = k;
}

// Gather the state into sorted order; re-fold positions into the primary box.
template <int D>
__global__ void k_permute(const DevSeg* __restrict__ segs, int N, const uint32_t* __restrict__ perm, Arrays in,
                          Arrays out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int src = (int)perm[k];
  uint2 m = in.meta[src];
  const DevSeg& s = segs[m.y];
  float4 a = in.A[src], b = in.B[src];
  Cold c = load_cold<D>(in, src);
  float xh[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < D; ++q) {
    double x = __dadd_rn((double)c.hi[q], (double)c.lo[q]);
    double f = 0.0;
    if ((s.periodic_mask >> q) & 1) f = floor(__ddiv_rn(__dsub_rn(x, s.lo_d[q]), s.L_d[q]));
    double o = __dmul_rn(s.L_d[q], f);
    c.off[q] = (float)o;
    xh[q] = (float)__dsub_rn(x, o);
  }
  if (D == 2) {
    out.A[k] = make_float4(xh[0], xh[1], a.z, a.w);
  } else {
    out.A[k] = make_float4(xh[0], xh[1], xh[2], a.w);
    out.C[k] = in.C[src];
  }
  store_cold<D>(out, k, c);
  out.B[k] = b;
  out.meta[k] = m;
}

// ================================================================== particle records
template <int D>
struct PD {
  float x[D], v[D], rho, p, V, m;
};

template <int D>
__device__ __forceinline__ PD<D> load_pd(const Arrays& a, int j) {
  PD<D> r;
  float4 A = __ldg(a.A + j), B = __ldg(a.B + j);
  if (D == 2) {
    r.x[0] = A.x; r.x[1] = A.y; r.v[0] = A.z; r.v[1] = A.w;
    r.rho = B.x; r.p = B.y; r.V = B.z; r.m = B.w;
  } else {
    float2 C = __ldg(a.C + j);
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

__device__ __forceinline__ float safe_q(float r2, float invH) { return r2 * rsqrtf(fmaxf(r2, 1e-30f)) * invH; }

// ================================================================== walls (config: dam break)
// p_w = [sum_f p_f W_wf + g . sum_f rho_f r_wf W_wf] / sum_f W_wf over fluid f, r_wf = x_w - x_f;
// rho_w = rho0 (1 + p_w / B)^(1/gamma); p_w = 0 when no fluid is in range.
template <int D, int KERN>
struct WallBody {
  const DevSeg* s;
  Arrays a;
  float xi[D];
  float sW, sp, sh;
  __device__ void pair(uint32_t j) {
    PD<D> pj = load_pd<D>(a, (int)j);
    if (pj.m < 0.f) return;  // wall neighbour
    float r[D];
    float r2 = separation<D>(*s, xi, pj.x, r);
    float W = s->Kw * kern_w<KERN>(safe_q(r2, s->invH));
    float gr = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) gr = fmaf(s->g[k], r[k], gr);
    sW += W;
    sp = fmaf(pj.p, W, sp);
    sh = fmaf(pj.rho * gr, W, sh);
  }
};

template <int D, int KERN>
__global__ void __launch_bounds__(256) k_walls(TravArgs t) {
  extern __shared__ uint32_t s_list[];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < t.N;
  uint2 m = valid ? t.a.meta[i] : make_uint2(0u, 0u);
  const bool wall = valid && (m.x & kWallBit);
  if (!__any_sync(kFull, wall)) return;
  const int seg = (int)m.y;
  WallBody<D, KERN> body;
  body.s = t.segs + seg;
  body.a = t.a;
  body.sW = body.sp = body.sh = 0.f;
  if (wall) load_pos<D>(t.a.A, i, body.xi);
  uint32_t* list = s_list + (threadIdx.x >> 5) * (kListCap * 32) + (threadIdx.x & 31);
  traverse<D, false>(t.segs, t.a.A, t.a, t.keys, t.cell_off, i, wall, seg, list, body);
  if (wall) {
    const DevSeg& s = *body.s;
    float pw = body.sW > 0.f ? (body.sp + body.sh) / body.sW : 0.f;
    float rw = tait_rho(s, pw);
    PD<D> me = load_pd<D>(t.a, i);
    me.rho = rw;
    me.p = pw;
    me.V = fabsf(me.m) / rw;
    store_pd<D>(t.a, i, me);
  }
}

// ================================================================== density summation
// Summation density rho_i = sum_j m_j W_ij (self term included).  The sum is accumulated in
// FP64 and the pressure is taken from the FP64 value: p = B[(rho/rho0)^gamma - 1] amplifies
// a relative density error by gamma (p + B)/p, which a float32 sum would not survive.
template <int D, int KERN>
struct DensityBody {
  const DevSeg* s;
  Arrays a;
  float xi[D];
  double rho;
  __device__ void pair(uint32_t j) {
    PD<D> pj = load_pd<D>(a, (int)j);
    float r[D];
    float r2 = separation<D>(*s, xi, pj.x, r);
    rho += (double)(fabsf(pj.m) * (s->Kw * kern_w<KERN>(safe_q(r2, s->invH))));
  }
};

template <int D, int KERN>
__global__ void __launch_bounds__(256) k_density(TravArgs t) {
  extern __shared__ uint32_t s_list[];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < t.N;
  uint2 m = valid ? t.a.meta[i] : make_uint2(0u, 0u);
  const bool fluid = valid && !(m.x & kWallBit);
  if (!__any_sync(kFull, fluid)) return;
  const int seg = (int)m.y;
  DensityBody<D, KERN> body;
  body.s = t.segs + seg;
  body.a = t.a;
  PD<D> me;
  if (fluid) {
    me = load_pd<D>(t.a, i);
    for (int k = 0; k < D; ++k) body.xi[k] = me.x[k];
    body.rho = (double)(me.m * body.s->Kw);  // self term, w(0) = 1
  }
  uint32_t* list = s_list + (threadIdx.x >> 5) * (kListCap * 32) + (threadIdx.x & 31);
  traverse<D, false>(t.segs, t.a.A, t.a, t.keys, t.cell_off, i, fluid, seg, list, body);
  if (fluid) {
    const DevSeg& s = *body.s;
    const double rho = body.rho;
    const float e = (float)((rho - (double)s.rho0) / (double)s.rho0);
    me.rho = (float)rho;
    me.p = s.B * expm1f(s.gamma * log1pf(e));
    me.V = me.m / me.rho;
    store_pd<D>(t.a, i, me);
    Cold c = load_cold<D>(t.a, i);
    c.rlo = (float)(rho - (double)me.rho);
    store_cold<D>(t.a, i, c);
  }
}

// ================================================================== fused sweep
// Rates of fluid particle i (Sec. 2.3):
//   a_i    = (1/rho_i) sum_j V_j gK (Cv w s - (p_i + p_j)) r  + g
//   drho_i = rho_i sum_j V_j gK w  - 2 Cdel sum_j V_j gK (rho_j - rho_i) r^2 s
// with r = x_i - x_j, gK r = grad_i W_ij, w = (v_i - v_j).r, s = 1/(r^2 + eps H^2),
// Cv = 2(d+2) nu rho0, Cdel = delta H c0.  These are the paper's terms regrouped per pair.
template <int D, int KERN>
struct SweepBody {
  const DevSeg* s;
  Arrays a;
  float xi[D], vi[D], rho_i, p_i;
  float acc[D], c1, c2;
  int npair;
  __device__ void pair(uint32_t j) {
    PD<D> pj = load_pd<D>(a, (int)j);
    float r[D];
    float r2 = separation<D>(*s, xi, pj.x, r);
    float q = safe_q(r2, s->invH);
    float gK = s->Kg * kern_gt<KERN>(q);
    float w = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) w = fmaf(vi[k] - pj.v[k], r[k], w);
    float sd = __frcp_rn(r2 + s->eH2);
    float VgK = pj.V * gK;
    float t = VgK * fmaf(s->Cv * w, sd, -(p_i + pj.p));
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = fmaf(t, r[k], acc[k]);
    c1 = fmaf(VgK, w, c1);
    c2 = fmaf(VgK * (pj.rho - rho_i), r2 * sd, c2);
    ++npair;
  }
};

template <int D, int KERN, bool INTEGRATE>
__global__ void __launch_bounds__(256) k_sweep(TravArgs t, Arrays out, RateOut ro) {
  extern __shared__ uint32_t s_list[];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < t.N;
  uint2 m = valid ? t.a.meta[i] : make_uint2(0u, 0u);
  const bool fluid = valid && !(m.x & kWallBit);
  const int seg = (int)m.y;
  SweepBody<D, KERN> body;
  body.s = t.segs + seg;
  body.a = t.a;
  body.c1 = body.c2 = 0.f;
  body.npair = 0;
  PD<D> me;
  if (valid) {
    me = load_pd<D>(t.a, i);
    for (int k = 0; k < D; ++k) {
      body.xi[k] = me.x[k];
      body.vi[k] = me.v[k];
      body.acc[k] = 0.f;
    }
    body.rho_i = me.rho;
    body.p_i = me.p;
  }
  uint32_t* list = s_list + (threadIdx.x >> 5) * (kListCap * 32) + (threadIdx.x & 31);
  traverse<D, false>(t.segs, t.a.A, t.a, t.keys, t.cell_off, i, fluid, seg, list, body);
  // pair count (fluid i) for the throughput metric
  int np = body.npair;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) np += __shfl_down_sync(kFull, np, o);
  if ((threadIdx.x & 31) == 0 && np && t.pair_count) atomicAdd(t.pair_count, (unsigned long long)np);
  if (!valid) return;
  const DevSeg& s = *body.s;
  float acc_a[D];
  float inv_rho = 1.f / me.rho;
#pragma unroll
  for (int k = 0; k < D; ++k) acc_a[k] = fmaf(body.acc[k], inv_rho, s.g[k]);
  float drho = fmaf(me.rho, body.c1, -2.f * s.Cdel * body.c2);
  if (!INTEGRATE) {
    if (fluid) {
      int o = (int)(m.x & ~kWallBit) + ro.orig_base[seg];
#pragma unroll
      for (int k = 0; k < D; ++k) ro.a[(size_t)o * D + k] = acc_a[k];
      ro.drho[o] = drho;
      ro.rho[o] = me.rho;
    }
    return;
  }
  Cold c = load_cold<D>(t.a, i);
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
      me.V = fabsf(me.m) / me.rho;
    }
    bool bad = !(me.rho > 0.5f * s.rho0 && me.rho < 2.f * s.rho0);
#pragma unroll
    for (int k = 0; k < D; ++k) bad |= !isfinite(c.hi[k]) || !isfinite(me.v[k]);
    if (bad) atomicOr(t.status, 1);
  }
  store_pd<D>(out, i, me);
  store_cold<D>(out, i, c);
  out.meta[i] = m;
}

// ================================================================== pair export (exact)
template <int D>
struct PairBody {
  uint32_t id_i;
  const uint2* meta;
  int32_t* pi;
  int32_t* pj;
  unsigned long long* count;
  long long cap;
  __device__ void pair(uint32_t j) {
    unsigned long long k = atomicAdd(count, 1ull);
    if ((long long)k < cap) {
      pi[k] = (int32_t)id_i;
      pj[k] = (int32_t)(meta[j].x & ~kWallBit);
    }
  }
};

template <int D>
__global__ void __launch_bounds__(256) k_pairs(TravArgs t, int32_t* pi, int32_t* pj, unsigned long long* count,
                                               long long cap) {
  extern __shared__ uint32_t s_list[];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < t.N;
  uint2 m = valid ? t.a.meta[i] : make_uint2(0u, 0u);
  PairBody<D> body;
  body.id_i = m.x & ~kWallBit;
  body.meta = t.a.meta;
  body.pi = pi;
  body.pj = pj;
  body.count = count;
  body.cap = cap;
  uint32_t* list = s_list + (threadIdx.x >> 5) * (kListCap * 32) + (threadIdx.x & 31);
  traverse<D, true>(t.segs, t.a.A, t.a, t.keys, t.cell_off, i, valid, (int)m.y, list, body);
}

// ================================================================== state in/out
template <int D>
__global__ void k_upload(const DevSeg* __restrict__ segs, int seg, int n, int nf, int p0, const float* __restrict__ x,
                         const float* __restrict__ v, const float* __restrict__ rho, const float* __restrict__ mass,
                         Arrays a) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const DevSeg& s = segs[seg];
  PD<D> r;
  Cold c;
  bool wall = k >= nf;
  for (int q = 0; q < 3; ++q) {
    c.hi[q] = (q < D) ? x[(size_t)k * D + q] : 0.f;
    c.lo[q] = 0.f;
    c.off[q] = 0.f;
  }
  c.rlo = 0.f;
  for (int q = 0; q < D; ++q) {
    r.x[q] = c.hi[q];
    r.v[q] = wall ? 0.f : v[(size_t)k * D + q];
  }
  r.rho = rho[k];
  r.m = wall ? -mass[k] : mass[k];
  r.p = tait_p(s, r.rho);
  r.V = mass[k] / r.rho;
  int j = p0 + k;
  store_pd<D>(a, j, r);
  store_cold<D>(a, j, c);
  a.meta[j] = make_uint2((uint32_t)k | (wall ? kWallBit : 0u), (uint32_t)seg);
}

template <int D>
__global__ void k_download(int N, Arrays a, const int* __restrict__ orig_base, float* __restrict__ x,
                           float* __restrict__ v, float* __restrict__ rho) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  uint2 m = a.meta[k];
  int o = (int)(m.x & ~kWallBit) + orig_base[m.y];
  PD<D> r = load_pd<D>(a, k);
  Cold c = load_cold<D>(a, k);
  for (int q = 0; q < D; ++q) {
    if (x) x[(size_t)o * D + q] = __fadd_rn(c.hi[q], c.lo[q]);
    if (v) v[(size_t)o * D + q] = r.v[q];
  }
  if (rho) rho[o] = __fadd_rn(r.rho, c.rlo);
}

// ================================================================== adjoint (Sec. 2.2)
// Adjoint state per particle (sorted order of the step): XB = (xbar, rhobar), VB = (vbar, -).
// Seeds for the pair terms: abar = dt (vbar' + dt xbar'), bbar = dt rhobar', and P' = dp/drho.
template <int D>
__global__ void k_adj_seed(const DevSeg* __restrict__ segs, int N, Arrays fw, const float4* __restrict__ XB,
                           const float4* __restrict__ VB, float4* __restrict__ S, float* __restrict__ Pp) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const DevSeg& s = segs[fw.meta[k].y];
  PD<D> r = load_pd<D>(fw, k);
  float4 xb = XB[k], vb = VB[k];
  float xbs[3] = {xb.x, xb.y, xb.z}, vbs[3] = {vb.x, vb.y, vb.z}, ab[3];
  for (int q = 0; q < 3; ++q) ab[q] = (q < D) ? s.dt * fmaf(s.dt, xbs[q], vbs[q]) : 0.f;
  float bb = s.dt * xb.w;
  float pp = tait_slope(s, r.rho, r.p);
  if (D == 2) {
    S[k] = make_float4(ab[0], ab[1], bb, pp);
  } else {
    S[k] = make_float4(ab[0], ab[1], ab[2], bb);
    Pp[k] = pp;
  }
}

template <int D, int KERN>
struct AdjBody {
  const DevSeg* s;
  Arrays a;
  const float4* S;
  const float* Pp;
  float xi[D], vi[D], rho_i, p_i, V_i, P_i;
  float ab_i[D], bb_i;
  float gx[D], gv[D], grho, gnu;
  __device__ void pair(uint32_t jj) {
    const int j = (int)jj;
    PD<D> pj = load_pd<D>(a, j);
    float4 Sj = __ldg(S + j);
    float ab_j[3], bb_j, P_j;
    if (D == 2) {
      ab_j[0] = Sj.x; ab_j[1] = Sj.y; ab_j[2] = 0.f; bb_j = Sj.z; P_j = Sj.w;
    } else {
      ab_j[0] = Sj.x; ab_j[1] = Sj.y; ab_j[2] = Sj.z; bb_j = Sj.w; P_j = __ldg(Pp + j);
    }
    const DevSeg& c = *s;
    float r[D], u[D];
    float r2 = separation<D>(c, xi, pj.x, r);
    float q = safe_q(r2, c.invH);
    float gK = c.Kg * kern_gt<KERN>(q);
    float hK = c.Kh * kern_ht<KERN>(q);
    float sd = __frcp_rn(r2 + c.eH2);
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
    const float X = fmaf(c.Cv, ws, -(p_i + pj.p));          // -(p_a + p_b) + Cv w s (same for both orders)
    const float r2s = r2 * sd;
    const float S1 = hK * r2s + 2.f * gK * sd * (c.eH2 * sd);  // hK r2 s + 2 gK s (1 - r2 s)
    const float CvsgK = c.Cv * sd * gK;
    const float XhR = fmaf(X, hK, -2.f * gK * c.Cv * w * sd * sd);
    // own term (a = i, b = j, seeds of i)
    float cR, cU, alpha_ab;
    {
      const float Vb_ra = pj.V / rho_i;
      const float alpha = Vb_ra * gK * X;
      const float beta = rho_i * pj.V * gK * w - 2.f * c.Cdel * pj.V * (pj.rho - rho_i) * gK * r2s;
      const float cRa = Vb_ra * XhR;
      const float cUa = Vb_ra * CvsgK;
      const float cRb = rho_i * pj.V * hK * w - 2.f * c.Cdel * pj.V * (pj.rho - rho_i) * S1;
      const float cUb = rho_i * pj.V * gK;
      cR = e_i * cRa + bb_i * cRb;
      cU = e_i * cUa + bb_i * cUb;
      alpha_ab = alpha;
      grho += e_i * (-pj.V * gK * P_i / rho_i - alpha / rho_i) +
              bb_i * (pj.V * gK * w + 2.f * c.Cdel * pj.V * gK * r2s);
      gnu += e_i * Vb_ra * gK * c.dCv_dnu * ws;
      (void)beta;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      gx[k] += alpha_ab * ab_i[k] + cR * r[k] + cU * u[k];
      gv[k] += cU * r[k];
    }
    // transposed term (a = j, b = i, seeds of j), contributes -d/dr_ji, -d/du_ji, d/drho_b
    {
      const float Va_rb = V_i / pj.rho;  // V_b / rho_a with b = i, a = j
      const float alpha = Va_rb * gK * X;
      const float beta = pj.rho * V_i * gK * w - 2.f * c.Cdel * V_i * (rho_i - pj.rho) * gK * r2s;
      const float cRa = Va_rb * XhR;
      const float cUa = Va_rb * CvsgK;
      const float cRb = pj.rho * V_i * hK * w - 2.f * c.Cdel * V_i * (rho_i - pj.rho) * S1;
      const float cUb = pj.rho * V_i * gK;
      cR = e_j * cRa + bb_j * cRb;
      cU = e_j * cUa + bb_j * cUb;
      alpha_ab = alpha;
      grho += e_j * (-alpha / rho_i - V_i * gK * P_i / pj.rho) +
              bb_j * (-beta / rho_i - 2.f * c.Cdel * V_i * gK * r2s);
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      gx[k] += -alpha_ab * ab_j[k] + cR * r[k] + cU * u[k];
      gv[k] += cU * r[k];
    }
  }
};

template <int D, int KERN>
__global__ void __launch_bounds__(256) k_adj_sweep(TravArgs t, const float4* __restrict__ S, const float* __restrict__ Pp,
                                                   const float4* __restrict__ XBin, const float4* __restrict__ VBin,
                                                   float4* __restrict__ XBout, float4* __restrict__ VBout,
                                                   double* __restrict__ nu_partial) {
  extern __shared__ uint32_t s_list[];
  __shared__ double s_red[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < t.N;
  uint2 m = valid ? t.a.meta[i] : make_uint2(0u, 0u);
  const bool fluid = valid && !(m.x & kWallBit);
  const int seg = (int)m.y;
  AdjBody<D, KERN> body;
  body.s = t.segs + seg;
  body.a = t.a;
  body.S = S;
  body.Pp = Pp;
  body.grho = body.gnu = 0.f;
  for (int k = 0; k < D; ++k) body.gx[k] = body.gv[k] = 0.f;
  if (valid) {
    PD<D> me = load_pd<D>(t.a, i);
    for (int k = 0; k < D; ++k) {
      body.xi[k] = me.x[k];
      body.vi[k] = me.v[k];
    }
    body.rho_i = me.rho;
    body.p_i = me.p;
    body.V_i = me.V;
    float4 Si = S[i];
    if (D == 2) {
      body.ab_i[0] = Si.x; body.ab_i[1] = Si.y; body.bb_i = Si.z; body.P_i = Si.w;
    } else {
      body.ab_i[0] = Si.x; body.ab_i[1] = Si.y; body.ab_i[2] = Si.z; body.bb_i = Si.w; body.P_i = Pp[i];
    }
  }
  uint32_t* list = s_list + (threadIdx.x >> 5) * (kListCap * 32) + (threadIdx.x & 31);
  traverse<D, false>(t.segs, t.a.A, t.a, t.keys, t.cell_off, i, fluid, seg, list, body);
  double nu_b = 0.0;
  if (valid) {
    const DevSeg& s = *body.s;
    float4 xb = XBin[i], vb = VBin[i];
    float xbs[3] = {xb.x, xb.y, xb.z}, vbs[3] = {vb.x, vb.y, vb.z};
    float ox[3] = {0.f, 0.f, 0.f}, ov[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < D; ++k) {
      float vt = fmaf(s.dt, xbs[k], vbs[k]);
      ox[k] = xbs[k] + body.gx[k];
      ov[k] = vt + body.gv[k];
    }
    XBout[i] = make_float4(ox[0], ox[1], ox[2], xb.w + body.grho);
    VBout[i] = make_float4(ov[0], ov[1], ov[2], 0.f);
    nu_b = (double)body.gnu;
  }
  double tot = block_sum(nu_b, s_red);
  if (threadIdx.x == 0) nu_partial[blockIdx.x] = tot;
}

// Adjoint of the permutation of a rebuild: out[perm[k]] = in[k].
__global__ void k_adj_unpermute(int N, const uint32_t* __restrict__ perm, const float4* __restrict__ XBin,
                                const float4* __restrict__ VBin, float4* __restrict__ XBout, float4* __restrict__ VBout) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int d = (int)perm[k];
  XBout[d] = XBin[k];
  VBout[d] = VBin[k];
}

// Deterministic sum of the per-block viscosity partials into acc (fixed order).
__global__ void k_sum_partials(const double* __restrict__ part, int n, double* __restrict__ acc) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += part[k];
  double t = block_sum(v, sh);
  if (threadIdx.x == 0) *acc += t;
}

// adjoint state of the final step from original-order inputs: scatter into sorted order
template <int D>
__global__ void k_adj_load(int N, const uint2* __restrict__ meta, const int* __restrict__ orig_base,
                           const float* __restrict__ xb, const float* __restrict__ vb, const float* __restrict__ rb,
                           float4* __restrict__ XB, float4* __restrict__ VB) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  uint2 m = meta[k];
  int o = (int)(m.x & ~kWallBit) + orig_base[m.y];
  float a[3] = {0.f, 0.f, 0.f}, b[3] = {0.f, 0.f, 0.f};
  for (int q = 0; q < D; ++q) {
    if (xb) a[q] = xb[(size_t)o * D + q];
    if (vb) b[q] = vb[(size_t)o * D + q];
  }
  XB[k] = make_float4(a[0], a[1], a[2], rb ? rb[o] : 0.f);
  VB[k] = make_float4(b[0], b[1], b[2], 0.f);
}

// adjoint of the initial state, delivered in original order through the storage map
template <int D>
__global__ void k_adj_store(int N, const uint2* __restrict__ meta, const int* __restrict__ orig_base,
                            const float4* __restrict__ XB, const float4* __restrict__ VB, float* __restrict__ xb,
                            float* __restrict__ vb, float* __restrict__ rb) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  uint2 m = meta[k];
  int o = (int)(m.x & ~kWallBit) + orig_base[m.y];
  float4 a = XB[k], b = VB[k];
  float as[3] = {a.x, a.y, a.z}, bs[3] = {b.x, b.y, b.z};
  for (int q = 0; q < D; ++q) {
    if (xb) xb[(size_t)o * D + q] = as[q];
    if (vb) vb[(size_t)o * D + q] = bs[q];
  }
  if (rb) rb[o] = a.w;
}

// ================================================================== launchers
template <int D>
void launch_keys(const DevSeg* segs, int N, const Arrays& a, uint32_t* keys, uint32_t* vals, cudaStream_t st) {
  if (N > 0) k_keys<D><<<(N + 255) / 256, 256, 0, st>>>(segs, N, a, keys, vals);
}

void launch_sort_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, int N, int shift,
                      uint32_t* hist, uint32_t* sums, cudaStream_t st) {
  int nb = (N + kSortTile - 1) / kSortTile;
  k_sort_hist<<<nb, kSortThreads, 0, st>>>(kin, N, shift, hist, nb);
  int n = 256 * nb;
  int sb = (n + 2047) / 2048;
  k_scan_blocks<<<sb, 1024, 0, st>>>(hist, n, sb > 1 ? sums : nullptr);
  if (sb > 1) {
    k_scan_blocks<<<1, 1024, 0, st>>>(sums, sb, nullptr);
    k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(hist, n, sums);
  }
  k_sort_scatter<<<nb, kSortThreads, 0, st>>>(kin, vin, kout, vout, N, shift, hist, nb);
}

int sort_scratch_words(int N) {
  int nb = (N + kSortTile - 1) / kSortTile;
  return 256 * nb + 2048 + 64;
}

void launch_cell_offsets(const uint32_t* keys, int N, int C, int* off, cudaStream_t st) {
  k_cell_offsets<<<(N + 1 + 255) / 256, 256, 0, st>>>(keys, N, C, off);
}

template <int D>
void launch_permute(const DevSeg* segs, int N, const uint32_t* perm, const Arrays& in, const Arrays& out,
                    cudaStream_t st) {
  if (N > 0) k_permute<D><<<(N + 255) / 256, 256, 0, st>>>(segs, N, perm, in, out);
}

size_t trav_smem() { return (size_t)8 * kListCap * 32 * sizeof(uint32_t); }

template <int D, int KERN>
void launch_walls(const TravArgs& t, cudaStream_t st) {
  if (t.N > 0) k_walls<D, KERN><<<(t.N + 255) / 256, 256, trav_smem(), st>>>(t);
}
template <int D, int KERN>
void launch_density(const TravArgs& t, cudaStream_t st) {
  if (t.N > 0) k_density<D, KERN><<<(t.N + 255) / 256, 256, trav_smem(), st>>>(t);
}
template <int D, int KERN>
void launch_sweep(const TravArgs& t, const Arrays& out, cudaStream_t st) {
  if (t.N > 0) k_sweep<D, KERN, true><<<(t.N + 255) / 256, 256, trav_smem(), st>>>(t, out, RateOut{});
}
template <int D, int KERN>
void launch_rates(const TravArgs& t, const RateOut& ro, cudaStream_t st) {
  if (t.N > 0) k_sweep<D, KERN, false><<<(t.N + 255) / 256, 256, trav_smem(), st>>>(t, Arrays{}, ro);
}
template <int D>
void launch_pairs(const TravArgs& t, int32_t* pi, int32_t* pj, unsigned long long* count, long long cap,
                  cudaStream_t st) {
  if (t.N > 0) k_pairs<D><<<(t.N + 255) / 256, 256, trav_smem(), st>>>(t, pi, pj, count, cap);
}
template <int D>
void launch_upload(const DevSeg* segs, int seg, int n, int nf, int p0, const float* x, const float* v, const float* rho,
                   const float* mass, const Arrays& a, cudaStream_t st) {
  if (n > 0) k_upload<D><<<(n + 255) / 256, 256, 0, st>>>(segs, seg, n, nf, p0, x, v, rho, mass, a);
}
template <int D>
void launch_download(int N, const Arrays& a, const int* orig_base, float* x, float* v, float* rho, cudaStream_t st) {
  if (N > 0) k_download<D><<<(N + 255) / 256, 256, 0, st>>>(N, a, orig_base, x, v, rho);
}
template <int D>
void launch_adj_seed(const DevSeg* segs, int N, const Arrays& fw, const float4* XB, const float4* VB, float4* S,
                     float* Pp, cudaStream_t st) {
  if (N > 0) k_adj_seed<D><<<(N + 255) / 256, 256, 0, st>>>(segs, N, fw, XB, VB, S, Pp);
}
template <int D, int KERN>
int launch_adj_sweep(const TravArgs& t, const float4* S, const float* Pp, const float4* XBin, const float4* VBin,
                     float4* XBout, float4* VBout, double* nu_partial, cudaStream_t st) {
  int nb = (t.N + 255) / 256;
  if (t.N > 0) k_adj_sweep<D, KERN><<<nb, 256, trav_smem(), st>>>(t, S, Pp, XBin, VBin, XBout, VBout, nu_partial);
  return nb;
}
void launch_adj_unpermute(int N, const uint32_t* perm, const float4* XBin, const float4* VBin, float4* XBout,
                          float4* VBout, cudaStream_t st) {
  if (N > 0) k_adj_unpermute<<<(N + 255) / 256, 256, 0, st>>>(N, perm, XBin, VBin, XBout, VBout);
}
void launch_sum_partials(const double* part, int n, double* acc, cudaStream_t st) {
  k_sum_partials<<<1, 256, 0, st>>>(part, n, acc);
}
template <int D>
void launch_adj_load(int N, const uint2* meta, const int* orig_base, const float* xb, const float* vb, const float* rb,
                     float4* XB, float4* VB, cudaStream_t st) {
  if (N > 0) k_adj_load<D><<<(N + 255) / 256, 256, 0, st>>>(N, meta, orig_base, xb, vb, rb, XB, VB);
}
template <int D>
void launch_adj_store(int N, const uint2* meta, const int* orig_base, const float4* XB, const float4* VB, float* xb,
                      float* vb, float* rb, cudaStream_t st) {
  if (N > 0) k_adj_store<D><<<(N + 255) / 256, 256, 0, st>>>(N, meta, orig_base, XB, VB, xb, vb, rb);
}

cudaError_t configure_kernels() {
  size_t sm = trav_smem();
  cudaError_t e = cudaSuccess;
#define SPH_ATTR(fn)                                                                   \
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  SPH_ATTR((k_walls<2, 0>)) SPH_ATTR((k_walls<2, 1>)) SPH_ATTR((k_walls<3, 0>)) SPH_ATTR((k_walls<3, 1>))
  SPH_ATTR((k_density<2, 0>)) SPH_ATTR((k_density<2, 1>)) SPH_ATTR((k_density<3, 0>)) SPH_ATTR((k_density<3, 1>))
  SPH_ATTR((k_sweep<2, 0, true>)) SPH_ATTR((k_sweep<2, 1, true>)) SPH_ATTR((k_sweep<3, 0, true>))
  SPH_ATTR((k_sweep<3, 1, true>)) SPH_ATTR((k_sweep<2, 0, false>)) SPH_ATTR((k_sweep<2, 1, false>))
  SPH_ATTR((k_sweep<3, 0, false>)) SPH_ATTR((k_sweep<3, 1, false>))
  SPH_ATTR((k_pairs<2>)) SPH_ATTR((k_pairs<3>))
  SPH_ATTR((k_adj_sweep<2, 0>)) SPH_ATTR((k_adj_sweep<2, 1>)) SPH_ATTR((k_adj_sweep<3, 0>)) SPH_ATTR((k_adj_sweep<3, 1>))
#undef SPH_ATTR
  return e;
}

#define SPH_INST_D(D)                                                                                          \
  template void launch_keys<D>(const DevSeg*, int, const Arrays&, uint32_t*, uint32_t*, cudaStream_t);           \
  template void launch_permute<D>(const DevSeg*, int, const uint32_t*, const Arrays&, const Arrays&, cudaStream_t); \
  template void launch_pairs<D>(const TravArgs&, int32_t*, int32_t*, unsigned long long*, long long, cudaStream_t); \
  template void launch_upload<D>(const DevSeg*, int, int, int, int, const float*, const float*, const float*,   \
                                 const float*, const Arrays&, cudaStream_t);                                   \
  template void launch_download<D>(int, const Arrays&, const int*, float*, float*, float*, cudaStream_t);       \
  template void launch_adj_seed<D>(const DevSeg*, int, const Arrays&, const float4*, const float4*, float4*, float*, \
                                   cudaStream_t);                                                              \
  template void launch_adj_load<D>(int, const uint2*, const int*, const float*, const float*, const float*, float4*, \
                                   float4*, cudaStream_t);                                                     \
  template void launch_adj_store<D>(int, const uint2*, const int*, const float4*, const float4*, float*, float*, \
                                    float*, cudaStream_t);
SPH_INST_D(2)
SPH_INST_D(3)
#define SPH_INST_DK(D, K)                                                                                     \
  template void launch_walls<D, K>(const TravArgs&, cudaStream_t);                                            \
  template void launch_density<D, K>(const TravArgs&, cudaStream_t);                                          \
  template void launch_sweep<D, K>(const TravArgs&, const Arrays&, cudaStream_t);                             \
  template void launch_rates<D, K>(const TravArgs&, const RateOut&, cudaStream_t);                            \
  template int launch_adj_sweep<D, K>(const TravArgs&, const float4*, const float*, const float4*, const float4*, \
                                      float4*, float4*, double*, cudaStream_t);
SPH_INST_DK(2, 0)
SPH_INST_DK(2, 1)
SPH_INST_DK(3, 0)
SPH_INST_DK(3, 1)

}  // namespace sph
